// encode.cu -- GPU construction of the linearized sparse encoding.
//
// Sec. 3.3 of the paper: a linearized tensor is the collection of nonzeros
// <v_i, p_i> ordered by the position p, whose l(p) bits interleave the
// coordinates' bits; Sec. 3.3.1-3.3.2 fix the semantics of a bit order (the
// mode named at b^t gives its next low bit). Here:
//   K1 build_keys   coordinates -> p, by precomputed bit runs per mode
//   K2 radix sort   stable LSD sort of (p, original index), 8-bit digits
//   K3 make_words   p -> stored word (coordinates as concatenated fields)
//      gather       values permuted into encoded order
//      stats        equal-work partitions, per-partition [lo, hi] per mode,
//                   per-mode run counts and histograms (Sec. 4.1.3, 4.2)
// All integer work; results are bit-exact with the CPU oracle.
#include <cstring>

#include "internal.cuh"

namespace relate {

namespace {

using u128 = unsigned __int128;

__device__ __forceinline__ W128 to_w128(u128 p) {
    W128 w;
    w.lo = (uint64_t)p;
    w.hi = (uint64_t)(p >> 64);
    return w;
}
__device__ __forceinline__ u128 from_w128(W128 w) { return ((u128)w.hi << 64) | (u128)w.lo; }

__device__ __forceinline__ uint32_t digit_of(uint32_t k, int shift) { return (k >> shift) & 0xffu; }
__device__ __forceinline__ uint32_t digit_of(unsigned long long k, int shift) {
    return (uint32_t)(k >> shift) & 0xffu;
}
__device__ __forceinline__ uint32_t digit_of(W128 k, int shift) {
    return shift < 64 ? (uint32_t)(k.lo >> shift) & 0xffu : (uint32_t)(k.hi >> (shift - 64)) & 0xffu;
}

// Integer type wide enough for a position of KW 32-bit limbs: 64-bit
// arithmetic whenever l(p) <= 64, 128-bit only for the wider keys.
template <int KW> struct Pos { using T = unsigned long long; };
template <> struct Pos<4> { using T = u128; };

template <typename P> __device__ __forceinline__ P low_bits(int len) {
    return len >= (int)(8 * sizeof(P)) ? ~(P)0 : (((P)1 << len) - 1);
}
template <int KW> __device__ __forceinline__ typename WordT<KW>::T to_word_p(typename Pos<KW>::T p);
template <> __device__ __forceinline__ uint32_t to_word_p<1>(unsigned long long p) { return (uint32_t)p; }
template <> __device__ __forceinline__ unsigned long long to_word_p<2>(unsigned long long p) { return p; }
template <> __device__ __forceinline__ W128 to_word_p<4>(u128 p) { return to_w128(p); }
template <int KW> __device__ __forceinline__ typename Pos<KW>::T from_word_p(typename WordT<KW>::T w);
template <> __device__ __forceinline__ unsigned long long from_word_p<1>(uint32_t w) { return w; }
template <> __device__ __forceinline__ unsigned long long from_word_p<2>(unsigned long long w) { return w; }
template <> __device__ __forceinline__ u128 from_word_p<4>(W128 w) { return from_w128(w); }

template <int KW>
__global__ void __launch_bounds__(kThreads) k_words_to_keys(const typename WordT<KW>::T *__restrict__ words,
                                                            int64_t n, BitRuns runs,
                                                            unsigned long long *__restrict__ out2) {
    using P = typename Pos<KW>::T;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const P w = from_word_p<KW>(words[e]);
        P p = 0;
        for (int m = 0; m < kMaxModes; m++) {
            for (int r = runs.mode_begin[m]; r < runs.mode_begin[m + 1]; r++) {
                const P bits = (w >> (runs.field_off[m] + runs.src[r])) & low_bits<P>(runs.len[r]);
                p |= bits << runs.dst[r];
            }
        }
        const u128 q = (u128)p;
        out2[2 * e] = (unsigned long long)q;
        out2[2 * e + 1] = (unsigned long long)(q >> 64);
    }
}

template <int KW>
__device__ __forceinline__ uint32_t field_of(typename WordT<KW>::T w, int shift, uint32_t mask);
template <> __device__ __forceinline__ uint32_t field_of<1>(uint32_t w, int shift, uint32_t mask) {
    return (uint32_t)((uint64_t)w >> shift) & mask;
}
template <> __device__ __forceinline__ uint32_t field_of<2>(unsigned long long w, int shift, uint32_t mask) {
    return (uint32_t)(w >> shift) & mask;
}
template <> __device__ __forceinline__ uint32_t field_of<4>(W128 w, int shift, uint32_t mask) {
    uint64_t x;
    if (shift >= 64)
        x = w.hi >> (shift - 64);
    else if (shift == 0)
        x = w.lo;
    else
        x = (w.lo >> shift) | (w.hi << (64 - shift));
    return (uint32_t)x & mask;
}

template <int KW>
__global__ void __launch_bounds__(kThreads) k_decode_words(const typename WordT<KW>::T *__restrict__ words,
                                                           int64_t n, int N, Fields f,
                                                           uint32_t *__restrict__ coords) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        auto w = words[e];
        for (int m = 0; m < N; m++) coords[(int64_t)m * n + e] = field_of<KW>(w, f.shift[m], f.mask[m]);
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_gather(const T *__restrict__ in, const uint32_t *__restrict__ perm,
                                                     int64_t n, T *__restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = __ldg(in + perm[e]);
}

// ------------------------------------------------------------------ K2
// One LSD pass = histogram (per tile, per digit) -> flat exclusive scan of
// the digit-major table -> stable scatter through a shared-memory stage.
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = kThreads * RS_ITEMS;  // 4096 keys per tile
constexpr int RS_WARPS = kThreads / 32;
constexpr int RADIX = 256;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename K>
__global__ void __launch_bounds__(kThreads) k_rs_hist(const K *__restrict__ keys, int64_t n, int shift,
                                                      uint32_t mask, uint32_t *__restrict__ hist,
                                                      int ntiles) {
    __shared__ uint32_t cnt[RS_WARPS][RADIX];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RADIX; i += kThreads) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * (32 * RS_ITEMS);
#pragma unroll 4
    for (int i = 0; i < RS_ITEMS; i++) {
        int64_t e = base + i * 32 + lane;
        uint32_t d = e < n ? (digit_of(keys[e], shift) & mask) : RADIX;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        int leader = 31 - __clz(peers);
        if (d < RADIX && lane == leader) cnt[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += kThreads) {
        uint32_t s = 0;
        for (int w = 0; w < RS_WARPS; w++) s += cnt[w][d];
        hist[(int64_t)d * ntiles + blockIdx.x] = s;
    }
}

// flat exclusive scan, three kernels: per-chunk sums, scan of sums, apply
constexpr int SCAN_CHUNK = 4096;

__global__ void __launch_bounds__(kThreads) k_scan_reduce(const uint32_t *__restrict__ in, int64_t n,
                                                          uint32_t *__restrict__ sums) {
    __shared__ uint32_t red[RS_WARPS];
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
    uint32_t s = 0;
    for (int i = threadIdx.x; i < SCAN_CHUNK; i += kThreads) {
        int64_t e = base + i;
        if (e < n) s += in[e];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < RS_WARPS; w++) t += red[w];
        sums[blockIdx.x] = t;
    }
}

// single block: exclusive scan of `sums` (nchunks entries) in place
__global__ void __launch_bounds__(1024) k_scan_sums(uint32_t *sums, int nchunks) {
    __shared__ uint32_t buf[1024];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nchunks; base += 1024) {
        int i = base + threadIdx.x;
        uint32_t v = i < nchunks ? sums[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            uint32_t t = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        uint32_t incl = buf[threadIdx.x];
        if (i < nchunks) sums[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) k_scan_apply(uint32_t *__restrict__ data, int64_t n,
                                                         const uint32_t *__restrict__ sums) {
    // each block scans one chunk of SCAN_CHUNK with RS_ITEMS-style blocking
    __shared__ uint32_t wsum[RS_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int PER = SCAN_CHUNK / kThreads;  // 16 consecutive items per thread
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * PER;
    uint32_t v[PER];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < PER; i++) {
        v[i] = base + i < n ? data[base + i] : 0;
        s += v[i];
    }
    uint32_t incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; w++) wpre += wsum[w];
    uint32_t run = sums[blockIdx.x] + wpre + incl - s;
#pragma unroll
    for (int i = 0; i < PER; i++) {
        if (base + i < n) data[base + i] = run;
        run += v[i];
    }
}

template <typename K>
__global__ void __launch_bounds__(kThreads) k_rs_scatter(const K *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                         K *__restrict__ kout, uint32_t *__restrict__ vout,
                                                         int64_t n, int shift, uint32_t mask,
                                                         const uint32_t *__restrict__ offsets, int ntiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K *skey = reinterpret_cast<K *>(smem_raw);
    uint32_t *sval = reinterpret_cast<uint32_t *>(smem_raw + sizeof(K) * RS_TILE);
    __shared__ uint32_t wcnt[RS_WARPS][RADIX];
    __shared__ uint32_t bdo[RADIX];  // block digit offsets (exclusive over digits)
    __shared__ uint32_t gofs[RADIX];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RADIX; i += kThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();

    const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * (32 * RS_ITEMS);
    K k[RS_ITEMS];
    uint32_t v[RS_ITEMS];
    uint32_t dig[RS_ITEMS];
    uint32_t rank[RS_ITEMS];
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < RS_ITEMS; i++) {
        int64_t e = base + i * 32 + lane;
        bool ok = e < n;
        if (ok) {
            k[i] = kin[e];
            v[i] = vin[e];
        }
        uint32_t d = ok ? (digit_of(k[i], shift) & mask) : RADIX;
        dig[i] = d;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = d < RADIX ? wcnt[warp][d] : 0;
        rank[i] = before + __popc(peers & lt);
        __syncwarp();
        if (d < RADIX && lane == 31 - __clz(peers)) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, block total
    uint32_t total = 0;
    if (threadIdx.x < RADIX) {
        const int d = threadIdx.x;
        for (int w = 0; w < RS_WARPS; w++) {
            uint32_t c = wcnt[w][d];
            wcnt[w][d] = total;
            total += c;
        }
        gofs[d] = offsets[(int64_t)d * ntiles + blockIdx.x];
    }
    // exclusive scan of totals over digits (kThreads == RADIX)
    {
        __shared__ uint32_t ws[RS_WARPS];
        uint32_t incl = total;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) ws[warp] = incl;
        __syncthreads();
        uint32_t pre = 0;
        for (int w = 0; w < warp; w++) pre += ws[w];
        if (threadIdx.x < RADIX) bdo[threadIdx.x] = pre + incl - total;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS_ITEMS; i++) {
        uint32_t d = dig[i];
        if (d < RADIX) {
            uint32_t pos = bdo[d] + wcnt[warp][d] + rank[i];
            skey[pos] = k[i];
            sval[pos] = v[i];
        }
    }
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
    const int cnt = (int)min((int64_t)RS_TILE, n - tile0);
    for (int j = threadIdx.x; j < cnt; j += kThreads) {
        K kk = skey[j];
        uint32_t d = digit_of(kk, shift) & mask;
        int64_t g = (int64_t)gofs[d] + (j - (int)bdo[d]);
        kout[g] = kk;
        vout[g] = sval[j];
    }
}

// ------------------------------------------------------------------ K3
template <int KW>
__global__ void __launch_bounds__(kThreads) k_partition_stats(const typename WordT<KW>::T *__restrict__ words,
                                                              int64_t n, int N, Fields f, int64_t S,
                                                              uint32_t *__restrict__ plo, uint32_t *__restrict__ phi,
                                                              unsigned long long *__restrict__ runs,
                                                              CountPtrs counts_tbl) {
    // one block per partition: [lo_n, hi_n] and runs of each mode, then each
    // mode's histogram of the partition, in shared memory when the
    // partition's rows of the mode span at most kStatBins (one global
    // addition per distinct row), else with warp-aggregated global atomics
    constexpr int kStatBins = 4096;
    __shared__ uint32_t s_lo[kMaxModes][RS_WARPS], s_hi[kMaxModes][RS_WARPS], s_rn[kMaxModes][RS_WARPS];
    __shared__ uint32_t s_blo[kMaxModes], s_bhi[kMaxModes];
    __shared__ uint32_t hist[kStatBins];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t q = blockIdx.x;
    const int64_t b = q * S, e = min(b + S, n);
    uint32_t lo[kMaxModes], hi[kMaxModes], rn[kMaxModes];
#pragma unroll
    for (int m = 0; m < kMaxModes; m++) {
        lo[m] = 0xffffffffu;
        hi[m] = 0;
        rn[m] = 0;
    }
    for (int64_t j = b + threadIdx.x; j < e; j += kThreads) {
        const typename WordT<KW>::T w = words[j];
        typename WordT<KW>::T wp{};
        if (j > b) wp = words[j - 1];
#pragma unroll
        for (int m = 0; m < kMaxModes; m++) {
            if (m < N) {
                const uint32_t c = field_of<KW>(w, f.shift[m], f.mask[m]);
                lo[m] = min(lo[m], c);
                hi[m] = max(hi[m], c);
                if (j == b || c != field_of<KW>(wp, f.shift[m], f.mask[m])) rn[m]++;
            }
        }
    }
#pragma unroll
    for (int m = 0; m < kMaxModes; m++) {
        if (m < N) {
            uint32_t a = lo[m], z = hi[m], r = rn[m];
            for (int o = 16; o > 0; o >>= 1) {
                a = min(a, __shfl_xor_sync(0xffffffffu, a, o));
                z = max(z, __shfl_xor_sync(0xffffffffu, z, o));
                r += __shfl_xor_sync(0xffffffffu, r, o);
            }
            if (lane == 0) {
                s_lo[m][warp] = a;
                s_hi[m][warp] = z;
                s_rn[m][warp] = r;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < N) {
        const int m = threadIdx.x;
        uint32_t a = 0xffffffffu, z = 0, r = 0;
        for (int w2 = 0; w2 < RS_WARPS; w2++) {
            a = min(a, s_lo[m][w2]);
            z = max(z, s_hi[m][w2]);
            r += s_rn[m][w2];
        }
        s_blo[m] = a;
        s_bhi[m] = z;
        plo[q * N + m] = a;
        phi[q * N + m] = z;
        atomicAdd(runs + m, (unsigned long long)r);
    }
    __syncthreads();
    for (int m = 0; m < N; m++) {
        const uint32_t mlo = s_blo[m], span = s_bhi[m] - mlo + 1;  // uniform
        uint32_t *cm = counts_tbl.p[m];
        const uint64_t len = counts_tbl.len[m];
        if (span <= (uint32_t)kStatBins) {
            for (uint32_t i = threadIdx.x; i < span; i += kThreads) hist[i] = 0;
            __syncthreads();
            for (int64_t j = b + threadIdx.x; j < e; j += kThreads) {
                const uint32_t c = field_of<KW>(words[j], f.shift[m], f.mask[m]);
                atomicAdd(hist + (c - mlo), 1u);
            }
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < span; i += kThreads)
                if (hist[i] && (uint64_t)mlo + i < len) atomicAdd(cm + mlo + i, hist[i]);
            __syncthreads();  // hist is reused by the next mode
        } else {
            // whole-warp steps so that __match_any_sync sees full warps
            for (int64_t j0 = b; j0 < e; j0 += kThreads) {
                const int64_t j = j0 + threadIdx.x;
                const bool ok = j < e;
                const uint32_t c = ok ? field_of<KW>(words[j], f.shift[m], f.mask[m]) : 0xffffffffu;
                // lanes past the end may share c's value: keep only valid peers
                const uint32_t peers = __match_any_sync(0xffffffffu, c) & __ballot_sync(0xffffffffu, ok);
                if (ok && lane == 31 - __clz(peers) && (uint64_t)c < len) atomicAdd(cm + c, (uint32_t)__popc(peers));
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_hist_summary(const uint32_t *__restrict__ counts, uint64_t len,
                                                           unsigned long long *__restrict__ out2) {
    unsigned long long d = 0, mx = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t c = counts[i];
        d += c != 0;
        mx = max(mx, (unsigned long long)c);
    }
    for (int o = 16; o > 0; o >>= 1) {
        d += __shfl_xor_sync(0xffffffffu, d, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (d) atomicAdd(out2, d);
        if (mx) atomicMax(out2 + 1, mx);
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_sumsq_partial(const T *__restrict__ v, int64_t n,
                                                            double *__restrict__ partial) {
    __shared__ double red[RS_WARPS];
    double s = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        double x = (double)v[e];
        s = fma(x, x, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < RS_WARPS; w++) t += red[w];
        partial[blockIdx.x] = t;
    }
}

__global__ void k_sum_fixed(const double *__restrict__ partial, int np, double *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < np; i++) s += partial[i];
        out[0] = s;
    }
}

// hot-row table: sort rows by decreasing population (stable), keep kHotMax
__global__ void __launch_bounds__(kThreads) k_count_keys(const uint32_t *__restrict__ counts, uint64_t I,
                                                         uint32_t *__restrict__ keys, uint32_t *__restrict__ idx) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < I; i += (uint64_t)gridDim.x * blockDim.x) {
        keys[i] = 0xffffffffu - counts[i];
        idx[i] = (uint32_t)i;
    }
}

__global__ void __launch_bounds__(kThreads) k_hot_rows(const uint32_t *__restrict__ sorted_keys,
                                                       const uint32_t *__restrict__ sorted_idx, uint64_t I,
                                                       uint32_t *__restrict__ hot_rows) {
    const int j = threadIdx.x + blockIdx.x * blockDim.x;
    if (j >= kHotMax) return;
    // count > 0 (key = ~count); 0xffffffff marks an unused entry
    hot_rows[j] = ((uint64_t)j < I && sorted_keys[j] != 0xffffffffu) ? sorted_idx[j] : 0xffffffffu;
}

// ---- table-driven bit permutations (K1 key build, p -> word packing)
template <int KW>
__global__ void __launch_bounds__(kThreads) k_build_keys_lut(const uint32_t *__restrict__ coords,
                                                             const uint64_t *__restrict__ dims, int64_t n, int N,
                                                             ByteLuts d, const typename Pos<KW>::T *__restrict__ tab,
                                                             typename WordT<KW>::T *__restrict__ keys,
                                                             uint32_t *__restrict__ idx, uint32_t *__restrict__ err) {
    using P = typename Pos<KW>::T;
    extern __shared__ __align__(16) unsigned char lut_raw[];
    P *lut = reinterpret_cast<P *>(lut_raw);
    for (int i = threadIdx.x; i < d.ntab * 256; i += blockDim.x) lut[i] = tab[i];
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        P p = 0;
        bool bad = false;
        for (int m = 0; m < N; m++) {
            const uint32_t c = __ldg(coords + (int64_t)m * n + e);
            bad |= (uint64_t)c >= dims[m];
            for (int t = d.src_begin[m]; t < d.src_begin[m + 1]; t++) p |= lut[t * 256 + ((c >> (8 * d.byte[t])) & 255u)];
        }
        if (bad) atomicOr(err, 1u);
        keys[e] = to_word_p<KW>(p);
        idx[e] = (uint32_t)e;
    }
}

template <int KW>
__global__ void __launch_bounds__(kThreads) k_make_words_lut(const typename WordT<KW>::T *__restrict__ keys, int64_t n,
                                                             ByteLuts d, const typename Pos<KW>::T *__restrict__ tab,
                                                             typename WordT<KW>::T *__restrict__ words) {
    using P = typename Pos<KW>::T;
    extern __shared__ __align__(16) unsigned char lut_raw[];
    P *lut = reinterpret_cast<P *>(lut_raw);
    for (int i = threadIdx.x; i < d.ntab * 256; i += blockDim.x) lut[i] = tab[i];
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const P p = from_word_p<KW>(keys[e]);
        P w = 0;
        for (int t = 0; t < d.ntab; t++) w |= lut[t * 256 + (uint32_t)((p >> (8 * d.byte[t])) & 255u)];
        words[e] = to_word_p<KW>(w);
    }
}

inline int grid_for(int64_t n, int per_block = kThreads, int cap = 152 * 32) {
    int64_t g = (n + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

template <typename K>
cudaError_t rs_passes(K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt, int64_t n, int lp,
                      void *temp, cudaStream_t st, bool *in_alt) {
    *in_alt = false;
    if (n <= 1 || lp <= 0) return cudaSuccess;
    const int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
    const int64_t hlen = (int64_t)RADIX * ntiles;
    const int nchunks = (int)((hlen + SCAN_CHUNK - 1) / SCAN_CHUNK);
    uint32_t *hist = reinterpret_cast<uint32_t *>(temp);
    uint32_t *sums = hist + hlen;
    const size_t smem = sizeof(K) * RS_TILE + sizeof(uint32_t) * RS_TILE;
    cudaError_t e = allow_max_dynamic_smem(k_rs_scatter<K>);
    if (e != cudaSuccess) return e;
    K *ki = keys, *ko = keys_alt;
    uint32_t *vi = vals, *vo = vals_alt;
    for (int shift = 0; shift < lp; shift += 8) {
        const int bits = lp - shift < 8 ? lp - shift : 8;
        const uint32_t mask = (1u << bits) - 1u;
        k_rs_hist<K><<<ntiles, kThreads, 0, st>>>(ki, n, shift, mask, hist, ntiles);
        k_scan_reduce<<<nchunks, kThreads, 0, st>>>(hist, hlen, sums);
        k_scan_sums<<<1, 1024, 0, st>>>(sums, nchunks);
        k_scan_apply<<<nchunks, kThreads, 0, st>>>(hist, hlen, sums);
        k_rs_scatter<K><<<ntiles, kThreads, smem, st>>>(ki, vi, ko, vo, n, shift, mask, hist, ntiles);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        K *tk = ki; ki = ko; ko = tk;
        uint32_t *tv = vi; vi = vo; vo = tv;
        *in_alt = !*in_alt;
    }
    return cudaSuccess;
}

}  // namespace

size_t radix_sort_temp_bytes(int64_t n) {
    const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    const int64_t hlen = (int64_t)RADIX * (ntiles > 0 ? ntiles : 1);
    const int64_t nchunks = (hlen + SCAN_CHUNK - 1) / SCAN_CHUNK;
    return sizeof(uint32_t) * (size_t)(hlen + nchunks + 16);
}

cudaError_t radix_sort_pairs(int KW, void *keys, uint32_t *vals, void *keys_alt, uint32_t *vals_alt, int64_t n,
                             int lp, void *temp, size_t temp_bytes, cudaStream_t st, bool *in_alt) {
    if (temp_bytes < radix_sort_temp_bytes(n)) return cudaErrorInvalidValue;
    switch (KW) {
    case 1: return rs_passes<uint32_t>((uint32_t *)keys, vals, (uint32_t *)keys_alt, vals_alt, n, lp, temp, st, in_alt);
    case 2: return rs_passes<unsigned long long>((unsigned long long *)keys, vals, (unsigned long long *)keys_alt, vals_alt, n, lp, temp, st, in_alt);
    default: return rs_passes<W128>((W128 *)keys, vals, (W128 *)keys_alt, vals_alt, n, lp, temp, st, in_alt);
    }
}

cudaError_t launch_words_to_keys(int KW, const void *words, int64_t n, const BitRuns &runs, uint64_t *out2,
                                 cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int g = grid_for(n);
    auto o = reinterpret_cast<unsigned long long *>(out2);
    switch (KW) {
    case 1: k_words_to_keys<1><<<g, kThreads, 0, st>>>((const uint32_t *)words, n, runs, o); break;
    case 2: k_words_to_keys<2><<<g, kThreads, 0, st>>>((const unsigned long long *)words, n, runs, o); break;
    default: k_words_to_keys<4><<<g, kThreads, 0, st>>>((const W128 *)words, n, runs, o); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_decode_words(int KW, const void *words, int64_t n, int N, const Fields &f, uint32_t *coords,
                                cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int g = grid_for(n);
    switch (KW) {
    case 1: k_decode_words<1><<<g, kThreads, 0, st>>>((const uint32_t *)words, n, N, f, coords); break;
    case 2: k_decode_words<2><<<g, kThreads, 0, st>>>((const unsigned long long *)words, n, N, f, coords); break;
    default: k_decode_words<4><<<g, kThreads, 0, st>>>((const W128 *)words, n, N, f, coords); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_gather(const void *vals_in, const uint32_t *perm, int64_t n, int elem_bytes, void *vals_out,
                          cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int g = grid_for(n);
    if (elem_bytes == 8)
        k_gather<unsigned long long><<<g, kThreads, 0, st>>>((const unsigned long long *)vals_in, perm, n,
                                                              (unsigned long long *)vals_out);
    else
        k_gather<uint32_t><<<g, kThreads, 0, st>>>((const uint32_t *)vals_in, perm, n, (uint32_t *)vals_out);
    return cudaGetLastError();
}

cudaError_t launch_partition_stats(int KW, const void *words, int64_t n, int N, const Fields &f, int64_t S,
                                   uint32_t *plo, uint32_t *phi, unsigned long long *runs,
                                   const CountPtrs &counts, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int64_t P = (n + S - 1) / S;
    if (P > 0x7fffffff) return cudaErrorInvalidValue;
    switch (KW) {
    case 1: k_partition_stats<1><<<(unsigned)P, kThreads, 0, st>>>((const uint32_t *)words, n, N, f, S, plo, phi, runs, counts); break;
    case 2: k_partition_stats<2><<<(unsigned)P, kThreads, 0, st>>>((const unsigned long long *)words, n, N, f, S, plo, phi, runs, counts); break;
    default: k_partition_stats<4><<<(unsigned)P, kThreads, 0, st>>>((const W128 *)words, n, N, f, S, plo, phi, runs, counts); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_hist_summary(const uint32_t *counts, uint64_t len, unsigned long long *out2, cudaStream_t st) {
    if (len == 0) return cudaSuccess;
    k_hist_summary<<<grid_for((int64_t)len), kThreads, 0, st>>>(counts, len, out2);
    return cudaGetLastError();
}

namespace {
// table entries have the width of the arithmetic type: 8 bytes for keys of
// up to 64 bits, 16 bytes beyond
inline size_t entry_bytes(int KW) { return KW == 4 ? 16 : 8; }
// sets bit `bit` of table entry `e` (little-endian 32-bit limbs)
inline void set_bit(unsigned char *tables, int KW, size_t e, int bit) {
    uint32_t *limbs = reinterpret_cast<uint32_t *>(tables + e * entry_bytes(KW));
    limbs[bit >> 5] |= 1u << (bit & 31);
}
}  // namespace

void build_key_luts(int N, const int *lbits, const int8_t *order, int lp, int KW, ByteLuts &d, void *host_tables) {
    // bit s of coordinate m lands at position pos[m][s] of p
    int pos[kMaxModes][32];
    int next[kMaxModes] = {};
    for (int t = 0; t < lp; t++) pos[order[t]][next[order[t]]++] = t;
    unsigned char *tab = static_cast<unsigned char *>(host_tables);
    d.ntab = 0;
    for (int m = 0; m < kMaxModes; m++) {
        d.src_begin[m] = d.ntab;
        if (m >= N) continue;
        for (int b = 0; b * 8 < lbits[m]; b++) {
            const int t = d.ntab++;
            d.byte[t] = (uint8_t)b;
            memset(tab + (size_t)t * 256 * entry_bytes(KW), 0, 256 * entry_bytes(KW));
            for (int v = 0; v < 256; v++)
                for (int i = 0; i < 8; i++) {
                    const int s = 8 * b + i;
                    if (s < lbits[m] && ((v >> i) & 1)) set_bit(tab, KW, (size_t)t * 256 + v, pos[m][s]);
                }
        }
    }
    d.src_begin[kMaxModes] = d.ntab;
}

void build_word_luts(int N, const int *field_off, const int8_t *order, int lp, int KW, ByteLuts &d,
                     void *host_tables) {
    // bit t of p is bit c_t of mode a_t, which sits at field_off[a_t] + c_t
    int dst[RELATE_MAX_KEY_BITS];
    int next[kMaxModes] = {};
    for (int t = 0; t < lp; t++) {
        const int m = order[t];
        dst[t] = field_off[m] + next[m]++;
    }
    (void)N;
    unsigned char *tab = static_cast<unsigned char *>(host_tables);
    d.ntab = 0;
    for (int b = 0; b * 8 < lp; b++) {
        const int t = d.ntab++;
        d.byte[t] = (uint8_t)b;
        memset(tab + (size_t)t * 256 * entry_bytes(KW), 0, 256 * entry_bytes(KW));
        for (int v = 0; v < 256; v++)
            for (int i = 0; i < 8; i++) {
                const int bit = 8 * b + i;
                if (bit < lp && ((v >> i) & 1)) set_bit(tab, KW, (size_t)t * 256 + v, dst[bit]);
            }
    }
    for (int m = 0; m <= kMaxModes; m++) d.src_begin[m] = 0;
}

cudaError_t launch_build_keys_lut(int KW, const uint32_t *coords, const uint64_t *dims_dev, int64_t n, int N,
                                  const ByteLuts &d, const void *tables, void *keys, uint32_t *idx, uint32_t *err,
                                  cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int g = grid_for(n, kThreads, 152 * 8);
    const size_t smem = (size_t)d.ntab * 256 * entry_bytes(KW);
    switch (KW) {
    case 1: k_build_keys_lut<1><<<g, kThreads, smem, st>>>(coords, dims_dev, n, N, d, (const unsigned long long *)tables, (uint32_t *)keys, idx, err); break;
    case 2: k_build_keys_lut<2><<<g, kThreads, smem, st>>>(coords, dims_dev, n, N, d, (const unsigned long long *)tables, (unsigned long long *)keys, idx, err); break;
    default: {
        cudaError_t e = allow_max_dynamic_smem(k_build_keys_lut<4>);
        if (e != cudaSuccess) return e;
        k_build_keys_lut<4><<<g, kThreads, smem, st>>>(coords, dims_dev, n, N, d, (const u128 *)tables, (W128 *)keys, idx, err);
    }
    }
    return cudaGetLastError();
}

cudaError_t launch_make_words_lut(int KW, const void *keys, int64_t n, const ByteLuts &d, const void *tables,
                                  void *words, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int g = grid_for(n, kThreads, 152 * 8);
    const size_t smem = (size_t)d.ntab * 256 * entry_bytes(KW);
    switch (KW) {
    case 1: k_make_words_lut<1><<<g, kThreads, smem, st>>>((const uint32_t *)keys, n, d, (const unsigned long long *)tables, (uint32_t *)words); break;
    case 2: k_make_words_lut<2><<<g, kThreads, smem, st>>>((const unsigned long long *)keys, n, d, (const unsigned long long *)tables, (unsigned long long *)words); break;
    default: {
        cudaError_t e = allow_max_dynamic_smem(k_make_words_lut<4>);
        if (e != cudaSuccess) return e;
        k_make_words_lut<4><<<g, kThreads, smem, st>>>((const W128 *)keys, n, d, (const u128 *)tables, (W128 *)words);
    }
    }
    return cudaGetLastError();
}

size_t hot_table_temp_bytes(uint64_t I) {
    return 16 * (size_t)I + radix_sort_temp_bytes((int64_t)I) + 64;
}

cudaError_t launch_hot_table(const uint32_t *counts, uint64_t I, uint32_t *hot_rows, void *temp, cudaStream_t st) {
    uint32_t *keys = reinterpret_cast<uint32_t *>(temp);
    uint32_t *idx = keys + I;
    uint32_t *keys2 = idx + I;
    uint32_t *idx2 = keys2 + I;
    void *sort_tmp = idx2 + I;
    k_count_keys<<<grid_for((int64_t)I), kThreads, 0, st>>>(counts, I, keys, idx);
    bool in_alt = false;
    cudaError_t e = rs_passes<uint32_t>(keys, idx, keys2, idx2, (int64_t)I, 32, sort_tmp, st, &in_alt);
    if (e != cudaSuccess) return e;
    k_hot_rows<<<1, kHotMax, 0, st>>>(in_alt ? keys2 : keys, in_alt ? idx2 : idx, I, hot_rows);
    return cudaGetLastError();
}

cudaError_t launch_sum_squares(const void *vals, int64_t n, int elem_bytes, double *partial, double *out,
                               cudaStream_t st) {
    const int g = 1024;
    if (elem_bytes == 8)
        k_sumsq_partial<double><<<g, kThreads, 0, st>>>((const double *)vals, n, partial);
    else
        k_sumsq_partial<float><<<g, kThreads, 0, st>>>((const float *)vals, n, partial);
    k_sum_fixed<<<1, 32, 0, st>>>(partial, g, out);
    return cudaGetLastError();
}

}  // namespace relate
