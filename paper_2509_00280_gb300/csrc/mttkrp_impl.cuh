// mttkrp_impl.cuh -- the mode-n MTTKRP kernel over the linearized encoding.
//
// Sec. 2.2 and Fig. 2 of the paper: every nonzero (i_0..i_{N-1}, v) reads
// rows i_k of the factors A_k (k != n), multiplies them element-wise, scales
// by v and adds the result into row i_n of the output; writes to one row
// from many nonzeros must be synchronised (Sec. 2.2; Sec. 4.1.3 picks
// reduction or atomics per mode from fiber reuse).
//
// GB300 mapping:
//  * A block walks 2048-nonzero tiles of the sorted stream (grid-stride, so
//    neighbouring blocks work on neighbouring partitions and share factor
//    rows in L2); a tile's words and values arrive by a TMA bulk copy.
//  * The tile is ordered by output row in shared memory (a counting sort,
//    or the mode's precomputed tile order) and each nonzero is decoded once
//    into a record {value, i_n, i_k (k != n)}.
//  * A "group" of G lanes owns one nonzero at a time; each lane holds 16
//    bytes of the R-wide row (VEC elements), so a factor-row gather is G
//    coalesced 16-byte loads (one 128-byte line for R = 32 FP32).
//  * Each group walks a contiguous slice of the records. Consecutive
//    nonzeros with the same output row are summed in registers; a run is
//    flushed once:
//      ATOMIC      -> global vector atomics (red.global.add.v4.f32 / f64), the
//                     mode's hottest rows into shared-memory accumulators,
//      SEGMENTED   -> global vector atomics after the sort (the hottest rows of
//                     a skewed mode into the block's copy in global scratch),
//      PRIVATIZED  -> shared-memory atomics into a block-private copy of the
//                     whole output, flushed once per block.
#pragma once

#include "internal.cuh"

namespace relate {
namespace mk {

template <typename FT> struct Prec;
template <> struct Prec<double> {
    using C = double;
    static constexpr int VEC = 2;
};
template <> struct Prec<float> {
    using C = float;
    static constexpr int VEC = 4;
};
template <> struct Prec<__nv_bfloat16> {
    using C = float;
    static constexpr int VEC = 4;  // 8-byte loads: 8 lanes per nonzero for R = 32
};

template <int KW> __device__ __forceinline__ typename WordT<KW>::T load_word(const void *p, int64_t j);
template <> __device__ __forceinline__ uint32_t load_word<1>(const void *p, int64_t j) {
    return __ldg(reinterpret_cast<const unsigned int *>(p) + j);
}
template <> __device__ __forceinline__ unsigned long long load_word<2>(const void *p, int64_t j) {
    return __ldg(reinterpret_cast<const unsigned long long *>(p) + j);
}
template <> __device__ __forceinline__ W128 load_word<4>(const void *p, int64_t j) {
    uint4 u = __ldg(reinterpret_cast<const uint4 *>(p) + j);
    W128 w;
    w.lo = ((uint64_t)u.y << 32) | u.x;
    w.hi = ((uint64_t)u.w << 32) | u.z;
    return w;
}

__device__ __forceinline__ uint32_t fld(uint32_t w, int s, uint32_t m) { return (uint32_t)((uint64_t)w >> s) & m; }
__device__ __forceinline__ uint32_t fld(unsigned long long w, int s, uint32_t m) { return (uint32_t)(w >> s) & m; }
__device__ __forceinline__ uint32_t fld(W128 w, int s, uint32_t m) {
    uint64_t x;
    if (s >= 64)
        x = w.hi >> (s - 64);
    else if (s == 0)
        x = w.lo;
    else
        x = (w.lo >> s) | (w.hi << (64 - s));
    return (uint32_t)x & m;
}

// Load of VEC consecutive elements of a factor row at p (16-byte aligned for
// the vector forms), converted to C.
template <typename FT, int VEC> struct VecLoadP;
template <> struct VecLoadP<double, 2> {
    static __device__ __forceinline__ void run(const void *p, double (&x)[2]) {
        const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
        x[0] = v.x;
        x[1] = v.y;
    }
};
template <> struct VecLoadP<float, 4> {
    static __device__ __forceinline__ void run(const void *p, float (&x)[4]) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        x[0] = v.x;
        x[1] = v.y;
        x[2] = v.z;
        x[3] = v.w;
    }
};
template <> struct VecLoadP<__nv_bfloat16, 4> {
    static __device__ __forceinline__ void run(const void *p, float (&x)[4]) {
        const uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
        x[0] = __uint_as_float(u.x << 16);
        x[1] = __uint_as_float(u.x & 0xffff0000u);
        x[2] = __uint_as_float(u.y << 16);
        x[3] = __uint_as_float(u.y & 0xffff0000u);
    }
};
template <typename FT> struct VecLoadP<FT, 1> {
    using C = typename Prec<FT>::C;
    static __device__ __forceinline__ void run(const void *p, C (&x)[1]) { x[0] = (C)*reinterpret_cast<const FT *>(p); }
};

template <bool B> struct Tail {
    static constexpr bool value = B;
};

// global accumulation of one vector (VEC elements) at out + off
template <typename C, int VEC> struct GAdd;
template <> struct GAdd<float, 4> {
    static __device__ __forceinline__ void run(float *p, const float (&a)[4]) {
        atomicAdd(reinterpret_cast<float4 *>(p), make_float4(a[0], a[1], a[2], a[3]));
    }
};
template <> struct GAdd<float, 8> {
    static __device__ __forceinline__ void run(float *p, const float (&a)[8]) {
        atomicAdd(reinterpret_cast<float4 *>(p), make_float4(a[0], a[1], a[2], a[3]));
        atomicAdd(reinterpret_cast<float4 *>(p) + 1, make_float4(a[4], a[5], a[6], a[7]));
    }
};
template <> struct GAdd<double, 2> {
    static __device__ __forceinline__ void run(double *p, const double (&a)[2]) {
        atomicAdd(p, a[0]);
        atomicAdd(p + 1, a[1]);
    }
};
template <typename C> struct GAdd<C, 1> {
    static __device__ __forceinline__ void run(C *p, const C (&a)[1]) { atomicAdd(p, a[0]); }
};

// Nonzeros a group keeps in flight: all factor-row loads of U nonzeros are
// issued before any of them is consumed.
template <typename FT, int VPL> struct Unroll { static constexpr int U = 4; };

constexpr int kTile = 2048;       // nonzeros per tile
constexpr int kTileBits = 11;     // log2(kTile): a tile position in a tile-order entry
static_assert((1 << kTileBits) == kTile, "tile positions take kTileBits bits");
constexpr int kTagMax = (1 << (16 - kTileBits)) - 1;  // hot slots a 16-bit tile-order entry can tag
static_assert(kTagMax == kHotTagMax, "the AUTO rule counts on the tag range");
constexpr int kItems = kTile / kThreads;
constexpr int kSortBins = 2048;   // widest row range a tile may span to be sorted
constexpr int kSortBinBits = 11;  // log2(kSortBins): hashed bins take this many bits
static_assert((1 << kSortBinBits) == kSortBins, "sort bins must be a power of two");
constexpr int kSnap = 16;         // records a slice boundary may move to reach a run boundary

// A decoded nonzero in shared memory: its value (compute type) and all N
// indices; records are padded to a multiple of 16 bytes.
template <int NT, typename C> struct __align__(16) Rec {
    static constexpr int NI = NT ? NT : kMaxModes;
    C val;
    uint32_t idx[NI];
};
template <int NT, typename C> struct RecStride {
    static constexpr int B = (int)((sizeof(Rec<NT, C>) + 15) / 16 * 16);
};

__device__ __forceinline__ uint32_t lane_lt_mask() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Open-addressing hash set of the hot rows in shared memory (row -> slot).
constexpr int kHotHash = 2 * kHotMax;
__device__ __forceinline__ uint32_t hot_hash(uint32_t row) { return (row * 2654435761u) >> 23; }  // 9 bits

// Shared-memory bytes of the per-tile area: raw stage (words, values of vb
// bytes), records, row counters, hot-row hash, mbarrier. The compile-time
// SEGMENTED kernel (precomputed tile order, hot rows tagged there) needs no
// row counters and no hash.
template <int NT, int KW, typename C, bool SEG = false> constexpr size_t tile_bytes(int vb) {
    return (size_t)kTile * (4 * KW) + (size_t)kTile * vb + (size_t)kTile * RecStride<NT, C>::B +
           (SEG ? (size_t)0 : (size_t)kSortBins * 4 + (size_t)kHotHash * 8) + 16;
}

// ---- TMA bulk copy (global -> shared) completing on an mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after `limit` SM clock cycles and reports it.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// SEG = true: the SEGMENTED strategy fixed at compile time, with the mode's
// precomputed tile order (a.tperm, k_tile_order) in place of the in-kernel
// sort and no privatised output, so the flush and the record build carry no
// strategy branches. Runs go to global memory. Runs of the mode's hottest rows (hot_n >
// 0, tagged when the records are built) go to the block's own copy of those
// rows in global scratch (a.hot_scratch, zeroed by the block, same vector
// atomics), which the block adds into the output once at its end: a row
// present in tens of thousands of tiles would otherwise take one FP32 global
// addition per tile, and the rounding of that many additions to one large sum
// exceeds the FP32 tolerance.
template <int NT, int KW, typename FT, int VEC, int VPL, bool SEG>
__global__ void __launch_bounds__(kThreads, 3) k_mttkrp(const MttkrpArgs a, const int log2G) {
    using C = typename Prec<FT>::C;
    using Word = typename WordT<KW>::T;
    using R_t = Rec<NT, C>;
    constexpr int RB = RecStride<NT, C>::B;
    static_assert(sizeof(R_t) == RB, "records are indexed as an array of R_t");
    // nonzeros in flight per group: one more for the FP32/BF16 SEGMENTED
    // kernel of 2-3 modes, whose records and row registers leave room for it
    constexpr int U = (SEG && NT >= 2 && NT <= 3 && sizeof(C) == 4) ? Unroll<FT, VPL>::U + 1 : Unroll<FT, VPL>::U;
    constexpr int NI = R_t::NI;
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int N = NT ? NT : a.N;
    const int G = 1 << log2G;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int gid = threadIdx.x >> log2G;
    const int ngroups = kThreads >> log2G;
    const int R = a.R;
    const int nvec = (R + VEC - 1) / VEC;
    const int mode = a.mode;
    const int mshift = a.fields.shift[mode];
    const uint32_t mmask = a.fields.mask[mode];
    C *__restrict__ out = reinterpret_cast<C *>(a.out);
    const int strat = a.strategy;
    const bool priv = !SEG && strat == RELATE_CONFLICT_PRIVATIZED;
    const bool sort_tiles = SEG || strat != RELATE_CONFLICT_ATOMIC;
    const int hot_n = priv ? 0 : a.hot_n;
    const int vb = a.vals_f64 ? 8 : 4;

    // shared layout: accumulators | raw words | raw values | records | hot slots | row counters | mbarrier
    const int64_t acc_elems = priv ? (int64_t)a.In * R : SEG ? 0 : (int64_t)hot_n * R;
    // SEG: this block's copy of the hot rows in global scratch
    C *__restrict__ hrep = SEG && hot_n ? reinterpret_cast<C *>(a.hot_scratch) + (int64_t)blockIdx.x * hot_n * R
                                        : nullptr;
    C *sacc = reinterpret_cast<C *>(smem_raw);
    unsigned char *tarea = smem_raw + ((acc_elems * (int64_t)sizeof(C) + 15) & ~(int64_t)15);
    Word *sw = reinterpret_cast<Word *>(tarea);
    unsigned char *sv = tarea + (size_t)kTile * sizeof(Word);
    unsigned char *srec = sv + (size_t)kTile * vb;
    uint32_t *bins = reinterpret_cast<uint32_t *>(srec + (size_t)kTile * RB);
    uint32_t *hkey = bins + kSortBins;     // hot-row hash: keys (row ids)
    uint32_t *hval = hkey + kHotHash;      // and their slots
    // SEG uses neither: the mbarrier follows the records
    uint64_t *bar = SEG ? reinterpret_cast<uint64_t *>(srec + (size_t)kTile * RB)
                        : reinterpret_cast<uint64_t *>(hval + kHotHash);
    __shared__ uint32_t wsum[kThreads / 32];

    int vj[VPL];
    bool act[VPL];
#pragma unroll
    for (int v = 0; v < VPL; v++) {
        vj[v] = gl + v * G;
        act[v] = vj[v] < nvec;
    }
    for (int64_t i = threadIdx.x; i < acc_elems; i += kThreads) sacc[i] = C(0);
    if (SEG && hot_n)  // ordered before this block's atomics by the barriers that follow
        for (int i = threadIdx.x; i < hot_n * R; i += kThreads) hrep[i] = C(0);
    if (!SEG && hot_n) {  // hash set of this mode's hot rows (most populated first); SEG reads tags
        for (int i = threadIdx.x; i < kHotHash; i += kThreads) hkey[i] = 0xffffffffu;
        __syncthreads();
        for (int t = threadIdx.x; t < hot_n; t += kThreads) {
            const uint32_t row = __ldg(a.hot_rows + t);
            if (row == 0xffffffffu) continue;
            uint32_t h = hot_hash(row);
            for (int probe = 0; probe < kHotHash; probe++, h = (h + 1) & (kHotHash - 1)) {
                const uint32_t prev = atomicCAS(hkey + h, 0xffffffffu, row);
                if (prev == 0xffffffffu) {
                    hval[h] = (uint32_t)t;
                    break;
                }
                if (prev == row) break;
            }
        }
        __syncthreads();
    }
    // slot of a hot row, or 0xffffffff: a few shared-memory probes
    auto hot_slot_of = [&](uint32_t row) -> uint32_t {
        uint32_t h = hot_hash(row);
        for (int probe = 0; probe < kHotHash; probe++, h = (h + 1) & (kHotHash - 1)) {
            const uint32_t k = hkey[h];
            if (k == row) return hval[h];
            if (k == 0xffffffffu) return 0xffffffffu;
        }
        return 0xffffffffu;
    };

    const int64_t tiles_per_part = (a.S + kTile - 1) / kTile;
    const int64_t ntiles = a.P * tiles_per_part;
    // TMA needs 16-byte aligned tile starts: partitions of a multiple of 4 nonzeros
    const bool use_tma = (a.S % 4) == 0;
    auto tile_span = [&](int64_t tq, int64_t &b, int &nt) {
        const int64_t q = tq / tiles_per_part;
        b = q * a.S + (tq - q * tiles_per_part) * kTile;
        const int64_t pe = min(q * a.S + a.S, a.nnz);
        nt = (int)max((int64_t)0, min((int64_t)kTile, pe - b));
    };
    auto issue = [&](int64_t tq) {  // one thread: stage tile tq through TMA
        int64_t b;
        int nt;
        tile_span(tq, b, nt);
        if (nt == 0) return;
        const uint32_t wbytes = (uint32_t)((nt * sizeof(Word) + 15) & ~(size_t)15);
        const uint32_t vbytes = (uint32_t)((nt * vb + 15) & ~15);
        mbar_expect_tx(bar, wbytes + vbytes);
        bulk_g2s(sw, reinterpret_cast<const Word *>(a.words) + b, wbytes, bar);
        bulk_g2s(sv, reinterpret_cast<const unsigned char *>(a.vals) + b * vb, vbytes, bar);
    };
    if (use_tma) {
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        // fault_skip_copy (a test hook): the first tile's copy is never issued,
        // so its bounded wait runs out and the launch reports a timeout
        if (threadIdx.x == 0 && blockIdx.x < ntiles && !a.fault_skip_copy) issue(blockIdx.x);
    }
    uint32_t phase = 0;

    for (int64_t tq = blockIdx.x; tq < ntiles; tq += gridDim.x) {
        int64_t b;
        int nt;
        tile_span(tq, b, nt);
        if (nt == 0) {  // uniform; no copy was issued for an empty tile, stage the next one
            if (use_tma && threadIdx.x == 0 && tq + gridDim.x < ntiles) issue(tq + gridDim.x);
            continue;
        }
        const int64_t q = tq / tiles_per_part;
        if (use_tma) {
            const bool ok = mbar_wait_bounded(bar, phase, a.wait_cycles);
            phase ^= 1;
            if (__syncthreads_or(!ok)) {  // a copy never landed: report and stop
                if (threadIdx.x == 0) atomicOr(a.err, 1);
                return;
            }
        } else {
            __syncthreads();  // the previous tile is fully consumed
            for (int j = threadIdx.x; j < nt; j += kThreads) {
                sw[j] = load_word<KW>(a.words, b + j);
                if (a.vals_f64)
                    reinterpret_cast<double *>(sv)[j] = __ldg(reinterpret_cast<const double *>(a.vals) + b + j);
                else
                    reinterpret_cast<float *>(sv)[j] = __ldg(reinterpret_cast<const float *>(a.vals) + b + j);
            }
            __syncthreads();
        }

        // ---- block-local counting sort of the tile by output row: bins are
        // rows - lo when the partition's rows span at most kSortBins, else a
        // 11-bit multiplicative hash of the row (equal rows share a bin, so
        // their nonzeros stay adjacent unless another row hashes alike)
        const uint32_t lo = a.plo[q * N + mode];
        const uint32_t span = a.phi[q * N + mode] - lo + 1;
        const bool direct = span <= (uint32_t)kSortBins;
        const uint32_t nb = direct ? span : (uint32_t)kSortBins;
        const bool sorted = sort_tiles;
        auto bin_of = [&](uint32_t row) -> uint32_t {
            return direct ? row - lo : (row * 2654435761u) >> (32 - kSortBinBits);
        };
        // pass 1 counts rows; the warp-aggregated atomic returns the bin's
        // running count, so each nonzero learns its offset inside its bin
        // SEG: the precomputed tile order replaces the sort; each nonzero
        // reads its sorted position and hot tag from it in pass 2
        uint32_t ibin[kItems], ioff[kItems];
        if (sorted && !SEG) {
            for (uint32_t i = threadIdx.x; i < nb; i += kThreads) bins[i] = 0;
            __syncthreads();
#pragma unroll
            for (int i = 0; i < kItems; i++) {
                const int j = i * kThreads + threadIdx.x;
                const uint32_t r = j < nt ? bin_of(fld(sw[j], mshift, mmask)) : 0xffffffffu;
                const uint32_t peers = __match_any_sync(0xffffffffu, r);
                const int leader = __ffs(peers) - 1;
                uint32_t base = 0;
                if (r != 0xffffffffu && lane == leader) base = atomicAdd(bins + r, (uint32_t)__popc(peers));
                base = __shfl_sync(0xffffffffu, base, leader);
                ibin[i] = r;
                ioff[i] = base + __popc(peers & lane_lt_mask());
            }
            __syncthreads();
            {   // exclusive scan of the nb counters, a contiguous slice per thread
                constexpr int PER = kSortBins / kThreads;
                const int base = threadIdx.x * PER;
                uint32_t loc[PER];
                uint32_t sum = 0;
#pragma unroll
                for (int i = 0; i < PER; i++) {
                    loc[i] = base + i < (int)nb ? bins[base + i] : 0u;
                    sum += loc[i];
                }
                uint32_t incl = sum;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += t;
                }
                if (lane == 31) wsum[threadIdx.x >> 5] = incl;
                __syncthreads();
                uint32_t run = incl - sum;
                for (int w = 0; w < (threadIdx.x >> 5); w++) run += wsum[w];
#pragma unroll
                for (int i = 0; i < PER; i++) {
                    if (base + i < (int)nb) {
                        // a direct bin is a single row: a hot row's slot + 1
                        // rides in bits 16..24 (offsets stay below 2^16), so
                        // each row of the tile is looked up once
                        uint32_t bv = run;
                        if (hot_n && direct && loc[i]) {
                            const uint32_t hs = hot_slot_of(lo + (uint32_t)(base + i));
                            if (hs != 0xffffffffu) bv |= (hs + 1u) << 16;
                        }
                        bins[base + i] = bv;
                    }
                    run += loc[i];
                }
            }
            __syncthreads();
        }
        // ---- pass 2: decode each nonzero once into its record at its (sorted) position
#pragma unroll
        for (int i = 0; i < kItems; i++) {
            const int j = i * kThreads + threadIdx.x;
            if (j >= nt) continue;
            const Word w = sw[j];
            uint32_t p = (uint32_t)j, hbin = 0;
            if (SEG) {
                const uint32_t e = __ldg(a.tperm + b + j);
                p = e & (kTile - 1);
                hbin = e >> kTileBits;
                if (hbin > (uint32_t)hot_n) hbin = 0;  // tagged for a larger hot set
            } else if (sorted) {
                const uint32_t bv = bins[ibin[i]];
                p = (bv & 0xffffu) + ioff[i];
                hbin = bv >> 16;
            }
            R_t rec;
            rec.val = a.vals_f64 ? (C)reinterpret_cast<const double *>(sv)[j]
                                 : (C)reinterpret_cast<const float *>(sv)[j];
#pragma unroll
            for (int k = 0; k < NI; k++) rec.idx[k] = k < N ? fld(w, a.rshift[k], a.rmask[k]) : 0u;
            if (hot_n) {  // slot 0 becomes the run's destination: 0x80000000|slot for a hot row
                if (SEG && a.full_copy) {
                    rec.idx[0] |= 0x80000000u;  // every row has its slot: the row itself
                } else if (SEG || (sorted && direct)) {
                    if (hbin) rec.idx[0] = 0x80000000u | (hbin - 1u);
                } else {
                    const uint32_t hs = hot_slot_of(rec.idx[0]);
                    if (hs != 0xffffffffu) rec.idx[0] = 0x80000000u | hs;
                }
            }
            *reinterpret_cast<R_t *>(srec + (size_t)p * RB) = rec;
        }
        __syncthreads();  // records complete; the raw stage is free
        if (use_tma && threadIdx.x == 0 && tq + gridDim.x < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(tq + gridDim.x);  // lands while this tile computes
        }

        // ---- each group walks a contiguous slice of the records; slice
        // boundaries move forward to the next change of output row (at most
        // kSnap records) so that short runs are not split between groups
        const int chunk = (nt + ngroups - 1) / ngroups;
        auto snap = [&](int x) -> int {  // monotone in x because chunk >= kSnap
            if (x <= 0 || x >= nt || chunk < kSnap) return min(max(x, 0), nt);
            const uint32_t prev = reinterpret_cast<const R_t *>(srec + (size_t)(x - 1) * RB)->idx[0];
            for (int y = x; y < nt && y < x + kSnap; y++)
                if (reinterpret_cast<const R_t *>(srec + (size_t)y * RB)->idx[0] != prev) return y;
            return x;
        };
        const int jb = snap(gid * chunk);
        const int je = snap((gid + 1) * chunk);
        uint32_t cur = 0xffffffffu;
        C acc[VPL][VEC];
#pragma unroll
        for (int v = 0; v < VPL; v++)
#pragma unroll
            for (int i = 0; i < VEC; i++) acc[v][i] = C(0);

        auto flush = [&](uint32_t row) {
            C *dst;
            bool shared_acc = true;
            if (SEG) {
                shared_acc = false;
                dst = (hot_n && (row & 0x80000000u)) ? hrep + (int64_t)(row & 0x7fffffffu) * R  // block's copy
                                                     : out + (int64_t)row * R;
            } else if (priv) {
                dst = sacc + (int64_t)row * R;
            } else if (row & 0x80000000u) {  // hot row: its shared-memory slot
                dst = sacc + (int64_t)(row & 0x7fffffffu) * R;
            } else {
                dst = out + (int64_t)row * R;
                shared_acc = false;
            }
#pragma unroll
            for (int v = 0; v < VPL; v++) {
                if (!act[v]) continue;
                C *p = dst + vj[v] * VEC;
                if (shared_acc) {
#pragma unroll
                    for (int i = 0; i < VEC; i++)
                        if (VEC == 1 || vj[v] * VEC + i < R) atomicAdd(p + i, acc[v][i]);
                } else if (VEC == 1 || (vj[v] + 1) * VEC <= R) {
                    GAdd<C, VEC>::run(p, acc[v]);
                } else {
#pragma unroll
                    for (int i = 0; i < VEC; i++)
                        if (vj[v] * VEC + i < R) atomicAdd(p + i, acc[v][i]);
                }
            }
        };

        // byte offset of this lane's first vector in a row; a row's address is
        // one 32 x 32 -> 64-bit multiply-add off the factor's base
        const uint32_t loff = (uint32_t)gl * VEC * (uint32_t)sizeof(FT);
        const uint32_t rbytes = (uint32_t)R * (uint32_t)sizeof(FT);
        const R_t *recs = reinterpret_cast<const R_t *>(srec);
        // U nonzeros per step; the tail step (fewer than U left) clamps its
        // record reads and skips the missing nonzeros
        auto step = [&](int p0, auto tail) {
            constexpr bool TAIL = decltype(tail)::value;
            R_t rec[U];
            C t[U][VPL][VEC];
#pragma unroll
            for (int u = 0; u < U; u++) rec[u] = recs[TAIL ? min(p0 + u, je - 1) : p0 + u];
            bool first = true;
#pragma unroll
            for (int k = 1; k < NI; k++) {  // record slots 1..N-1: the other modes
                if (k >= N) continue;
                C x[U][VPL][VEC];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const char *rowp = reinterpret_cast<const char *>(a.rfac[k]) +
                                       ((uint64_t)rec[u].idx[k] * rbytes + loff);
#pragma unroll
                    for (int v = 0; v < VPL; v++)
                        if (act[v]) VecLoadP<FT, VEC>::run(rowp + (size_t)v * G * VEC * sizeof(FT), x[u][v]);
                }
#pragma unroll
                for (int u = 0; u < U; u++)
#pragma unroll
                    for (int v = 0; v < VPL; v++)
#pragma unroll
                        for (int i = 0; i < VEC; i++) t[u][v][i] = first ? x[u][v][i] : t[u][v][i] * x[u][v][i];
                first = false;
            }
            if (first) {  // one-mode tensor slice (N == 1 never happens; keeps t defined)
#pragma unroll
                for (int u = 0; u < U; u++)
#pragma unroll
                    for (int v = 0; v < VPL; v++)
#pragma unroll
                        for (int i = 0; i < VEC; i++) t[u][v][i] = C(1);
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (TAIL && p0 + u >= je) continue;
                const uint32_t row = rec[u].idx[0];
                const C val = rec[u].val;
                if (row != cur) {
                    if (cur != 0xffffffffu) flush(cur);
                    cur = row;
#pragma unroll
                    for (int v = 0; v < VPL; v++)
#pragma unroll
                        for (int i = 0; i < VEC; i++) acc[v][i] = val * t[u][v][i];
                } else {
#pragma unroll
                    for (int v = 0; v < VPL; v++)
#pragma unroll
                        for (int i = 0; i < VEC; i++) acc[v][i] = fma(val, t[u][v][i], acc[v][i]);
                }
            }
        };
        for (int p0 = jb; p0 < je; p0 += U) step(p0, Tail<true>{});
        if (cur != 0xffffffffu) flush(cur);
    }

    __syncthreads();
    if (priv) {
        const int64_t tot = (int64_t)a.In * R;
        for (int64_t i = threadIdx.x; i < tot; i += kThreads) {
            C s = sacc[i];
            if (s != C(0)) atomicAdd(out + i, s);
        }
    } else if (hot_n) {
        const int tot = hot_n * R;
        if (SEG) __threadfence();  // this block's atomics on its copy are complete
        __syncthreads();
        for (int i = threadIdx.x; i < tot; i += kThreads) {
            const C s = SEG ? __ldcg(hrep + i) : sacc[i];
            const uint32_t row = (SEG && a.full_copy) ? (uint32_t)(i / R) : __ldg(a.hot_rows + i / R);
            if (s != C(0) && row != 0xffffffffu) atomicAdd(out + (int64_t)row * R + i % R, s);
        }
    }
}

// Tile order of one mode, computed once per handle and mode: for every
// nonzero, its position in its tile sorted by output row (the counting sort
// of k_mttkrp: direct bins row - lo, or the hashed bins) in bits 0..10, and
// 1 + the hot slot of its row (0 = not hot; slots < hot_n <= kTagMax) in
// bits 11..15. One block per tile.
template <int KW>
__global__ void __launch_bounds__(kThreads) k_tile_order(const MttkrpArgs a, uint16_t *__restrict__ tperm) {
    __shared__ uint32_t bins[kSortBins];
    __shared__ uint32_t hkey[kHotHash], hval[kHotHash];
    __shared__ uint32_t wsum[kThreads / 32];
    const int lane = threadIdx.x & 31;
    const int N = a.N, mode = a.mode, hot_n = a.hot_n;
    const int mshift = a.fields.shift[mode];
    const uint32_t mmask = a.fields.mask[mode];
    if (hot_n) {
        for (int i = threadIdx.x; i < kHotHash; i += kThreads) hkey[i] = 0xffffffffu;
        __syncthreads();
        for (int t = threadIdx.x; t < hot_n; t += kThreads) {
            const uint32_t row = __ldg(a.hot_rows + t);
            if (row == 0xffffffffu) continue;
            uint32_t h = hot_hash(row);
            for (int probe = 0; probe < kHotHash; probe++, h = (h + 1) & (kHotHash - 1)) {
                const uint32_t prev = atomicCAS(hkey + h, 0xffffffffu, row);
                if (prev == 0xffffffffu) {
                    hval[h] = (uint32_t)t;
                    break;
                }
                if (prev == row) break;
            }
        }
        __syncthreads();
    }
    auto hot_tag = [&](uint32_t row) -> uint32_t {  // 1 + slot, or 0
        uint32_t h = hot_hash(row);
        for (int probe = 0; probe < kHotHash; probe++, h = (h + 1) & (kHotHash - 1)) {
            const uint32_t k = hkey[h];
            if (k == row) return hval[h] + 1u;
            if (k == 0xffffffffu) return 0u;
        }
        return 0u;
    };
    const int64_t tiles_per_part = (a.S + kTile - 1) / kTile;
    const int64_t ntiles = a.P * tiles_per_part;
    for (int64_t tq = blockIdx.x; tq < ntiles; tq += gridDim.x) {
        const int64_t q = tq / tiles_per_part;
        const int64_t b = q * a.S + (tq - q * tiles_per_part) * kTile;
        const int64_t pe = min(q * a.S + a.S, a.nnz);
        const int nt = (int)max((int64_t)0, min((int64_t)kTile, pe - b));
        if (nt == 0) continue;
        const uint32_t lo = a.plo[q * N + mode];
        const uint32_t span = a.phi[q * N + mode] - lo + 1;
        const bool direct = span <= (uint32_t)kSortBins;
        const uint32_t nb = direct ? span : (uint32_t)kSortBins;
        __syncthreads();  // the previous tile's bins are consumed
        for (uint32_t i = threadIdx.x; i < nb; i += kThreads) bins[i] = 0;
        __syncthreads();
        uint32_t ibin[kItems], ioff[kItems], irow[kItems];
#pragma unroll
        for (int i = 0; i < kItems; i++) {
            const int j = i * kThreads + threadIdx.x;
            const uint32_t row = j < nt ? fld(load_word<KW>(a.words, b + j), mshift, mmask) : 0u;
            const uint32_t r = j < nt ? (direct ? row - lo : (row * 2654435761u) >> (32 - kSortBinBits)) : 0xffffffffu;
            const uint32_t peers = __match_any_sync(0xffffffffu, r);
            const int leader = __ffs(peers) - 1;
            uint32_t base = 0;
            if (r != 0xffffffffu && lane == leader) base = atomicAdd(bins + r, (uint32_t)__popc(peers));
            base = __shfl_sync(0xffffffffu, base, leader);
            ibin[i] = r;
            ioff[i] = base + __popc(peers & lane_lt_mask());
            irow[i] = row;
        }
        __syncthreads();
        {   // exclusive scan of the bins, a contiguous slice per thread
            constexpr int PER = kSortBins / kThreads;
            const int base = threadIdx.x * PER;
            uint32_t loc[PER];
            uint32_t sum = 0;
#pragma unroll
            for (int i = 0; i < PER; i++) {
                loc[i] = base + i < (int)nb ? bins[base + i] : 0u;
                sum += loc[i];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane == 31) wsum[threadIdx.x >> 5] = incl;
            __syncthreads();
            uint32_t run = incl - sum;
            for (int w = 0; w < (threadIdx.x >> 5); w++) run += wsum[w];
#pragma unroll
            for (int i = 0; i < PER; i++) {
                if (base + i < (int)nb) bins[base + i] = run;
                run += loc[i];
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kItems; i++) {
            const int j = i * kThreads + threadIdx.x;
            if (j >= nt) continue;
            const uint32_t p = bins[ibin[i]] + ioff[i];
            const uint32_t tag = hot_n ? hot_tag(irow[i]) : 0u;
            tperm[b + j] = (uint16_t)(p | (tag << kTileBits));
        }
    }
}

// Chooses lanes per group for R and launches one instantiation.
template <int NT, int KW, typename FT, int VEC, int VPL, bool SEG = false>
cudaError_t launch_one(const MttkrpArgs &a, size_t acc_bytes, int grid, cudaStream_t st) {
    const int nvec = (a.R + VEC - 1) / VEC;
    int G = 1, log2G = 0;
    while (G * VPL < nvec && G < 32) {
        G <<= 1;
        log2G++;
    }
    const size_t smem = ((acc_bytes + 15) & ~(size_t)15) + tile_bytes<NT, KW, typename Prec<FT>::C, SEG>(a.vals_f64 ? 8 : 4);
    auto kern = k_mttkrp<NT, KW, FT, VEC, VPL, SEG>;
    cudaError_t e = allow_max_dynamic_smem(kern);
    if (e != cudaSuccess) return e;
    kern<<<grid, kThreads, smem, st>>>(a, log2G);
    return cudaGetLastError();
}

// Dispatch over N (2..5 specialised, 6..8 generic) and word width for one FT.
template <typename FT>
cudaError_t dispatch_ft(const MttkrpArgs &a, int KW, bool vec_ok, size_t acc_bytes, int grid, cudaStream_t st) {
    constexpr int V = Prec<FT>::VEC;
#define RELATE_MK_KW_S(NT_, S_)                                                                  \
    (KW == 1 ? launch_one<NT_, 1, FT, V, 1, S_>(a, acc_bytes, grid, st)                          \
             : KW == 2 ? launch_one<NT_, 2, FT, V, 1, S_>(a, acc_bytes, grid, st)                \
                       : launch_one<NT_, 4, FT, V, 1, S_>(a, acc_bytes, grid, st))
#define RELATE_MK_KW(NT_) (seg ? RELATE_MK_KW_S(NT_, true) : RELATE_MK_KW_S(NT_, false))
    const bool seg = a.strategy == RELATE_CONFLICT_SEGMENTED && a.tperm != nullptr;
    if (!vec_ok) {
        return KW == 1 ? launch_one<0, 1, FT, 1, 2>(a, acc_bytes, grid, st)
                       : KW == 2 ? launch_one<0, 2, FT, 1, 2>(a, acc_bytes, grid, st)
                                 : launch_one<0, 4, FT, 1, 2>(a, acc_bytes, grid, st);
    }
    switch (a.N) {
    case 2: return RELATE_MK_KW(2);
    case 3: return RELATE_MK_KW(3);
    case 4: return RELATE_MK_KW(4);
    case 5: return RELATE_MK_KW(5);
    default: return RELATE_MK_KW_S(0, false);
    }
#undef RELATE_MK_KW
#undef RELATE_MK_KW_S
}

// Per-tile shared bytes of the instantiation a launch will use (seg: the
// compile-time SEGMENTED kernel).
template <int KW, bool SEG>
inline size_t tile_bytes_kw(int NT, bool f64, int vb) {
    switch (NT) {
    case 2: return f64 ? tile_bytes<2, KW, double, SEG>(vb) : tile_bytes<2, KW, float, SEG>(vb);
    case 3: return f64 ? tile_bytes<3, KW, double, SEG>(vb) : tile_bytes<3, KW, float, SEG>(vb);
    case 4: return f64 ? tile_bytes<4, KW, double, SEG>(vb) : tile_bytes<4, KW, float, SEG>(vb);
    case 5: return f64 ? tile_bytes<5, KW, double, SEG>(vb) : tile_bytes<5, KW, float, SEG>(vb);
    default: return f64 ? tile_bytes<0, KW, double, SEG>(vb) : tile_bytes<0, KW, float, SEG>(vb);
    }
}
inline size_t tile_bytes_for(int N, int KW, int factor_dtype, bool vec_ok, int vb, bool seg = false) {
    const bool f64 = factor_dtype == RELATE_F64;
    const int NT = (vec_ok && N >= 2 && N <= 5) ? N : 0;
    if (seg && NT)
        return KW == 1 ? tile_bytes_kw<1, true>(NT, f64, vb) : KW == 2 ? tile_bytes_kw<2, true>(NT, f64, vb)
                                                                      : tile_bytes_kw<4, true>(NT, f64, vb);
    return KW == 1 ? tile_bytes_kw<1, false>(NT, f64, vb) : KW == 2 ? tile_bytes_kw<2, false>(NT, f64, vb)
                                                                    : tile_bytes_kw<4, false>(NT, f64, vb);
}

#include "mttkrp_fac.cuh"
#include "mttkrp_batch.cuh"

}  // namespace mk

cudaError_t mttkrp_batch_f64(const mk::BatchParams &bp, int N, int KW, int num_sms, cudaStream_t st);
cudaError_t mttkrp_batch_f32(const mk::BatchParams &bp, int N, int KW, int num_sms, cudaStream_t st);
cudaError_t mttkrp_batch_bf16(const mk::BatchParams &bp, int N, int KW, int num_sms, cudaStream_t st);

cudaError_t mttkrp_fac_f64(const MttkrpArgs &a, int KW, int64_t tiles, int num_sms, cudaStream_t st);
cudaError_t mttkrp_fac_f32(const MttkrpArgs &a, int KW, int64_t tiles, int num_sms, cudaStream_t st);
cudaError_t mttkrp_fac_bf16(const MttkrpArgs &a, int KW, int64_t tiles, int num_sms, cudaStream_t st);

cudaError_t mttkrp_f64(const MttkrpArgs &a, int KW, bool vec_ok, size_t acc_bytes, int grid, cudaStream_t st);

cudaError_t mttkrp_f32(const MttkrpArgs &a, int KW, bool vec_ok, size_t acc_bytes, int grid, cudaStream_t st);
cudaError_t mttkrp_bf16(const MttkrpArgs &a, int KW, bool vec_ok, size_t acc_bytes, int grid, cudaStream_t st);

}  // namespace relate
