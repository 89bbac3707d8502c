// mttkrp.cu -- host-side launch configuration of the MTTKRP kernel:
// grid sizing in multiples of the SM count, shared-memory accumulators,
// vector-path eligibility.
#include <map>
#include <mutex>
#include <utility>

#include "mttkrp_impl.cuh"

namespace relate {

int max_dynamic_smem(const void *kern) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    const auto key = std::make_pair(dev, kern);
    {
        std::lock_guard<std::mutex> lock(mu);
        const auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int optin = 0;
    cudaFuncAttributes fa{};
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, kern) != cudaSuccess)
        return 0;
    const int lim = optin - (int)fa.sharedSizeBytes;
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = lim;
    return lim;
}

int mttkrp_acc_bytes(int factor_dtype) { return factor_dtype == RELATE_F64 ? 8 : 4; }

// Record slots of a launch: slot 0 = the output mode, slots 1..N-1 = the other
// modes, in a.level order when the mode is fiber-factored (depth >= 1), else
// in increasing order.
void fill_slots(MttkrpArgs &a) {
    a.rshift[0] = a.fields.shift[a.mode];
    a.rmask[0] = a.fields.mask[a.mode];
    a.rfac[0] = nullptr;
    bool use_level = a.depth >= 1;
    if (use_level) {  // a.level must name every other mode once
        unsigned seen = 0;
        for (int s = 0; s < a.N - 1; s++) {
            const int k = a.level[s];
            if (k < 0 || k >= a.N || k == a.mode || (seen >> k) & 1u) use_level = false;
            else seen |= 1u << k;
        }
        if (!use_level) a.depth = 0;
    }
    int j = 1;
    for (int s = 0; s < a.N - 1; s++) {
        int k;
        if (use_level) {
            k = a.level[s];
        } else {
            k = s < a.mode ? s : s + 1;
        }
        a.rshift[j] = a.fields.shift[k];
        a.rmask[j] = a.fields.mask[k];
        a.rfac[j] = a.factors[k];
        j++;
    }
    for (; j < kMaxModes; j++) {
        a.rshift[j] = 0;
        a.rmask[j] = 0;
        a.rfac[j] = nullptr;
    }
}

cudaError_t launch_mttkrp(const MttkrpArgs &a_in, int KW, int factor_dtype, int val_dtype, int smem_budget,
                          int num_sms, cudaStream_t st) {
    MttkrpArgs a = a_in;
    if (a.nnz == 0 || a.P == 0) return cudaSuccess;
    if (a.wait_cycles <= 0) a.wait_cycles = kWaitCycles;
    const int accb = mttkrp_acc_bytes(factor_dtype);
    const int fb = factor_dtype == RELATE_F64 ? 8 : factor_dtype == RELATE_F32 ? 4 : 2;

    // vector path (16-byte loads, 8-byte for BF16): every factor row starts
    // 16-byte aligned and the output rows take 16-byte vector atomics
    bool vec_ok = (a.R * fb) % 16 == 0 && (a.R * accb) % 16 == 0 && (reinterpret_cast<uintptr_t>(a.out) % 16) == 0;
    for (int k = 0; k < a.N; k++)
        if (k != a.mode && (reinterpret_cast<uintptr_t>(a.factors[k]) % 16) != 0) vec_ok = false;

    a.vals_f64 = val_dtype == RELATE_F64;
    fill_slots(a);
    const int V = factor_dtype == RELATE_F64 ? 2 : 4;  // elements per lane load
    if (a.col_passes < 1 || a.R % a.col_passes != 0 || (a.R / a.col_passes) % V != 0) a.col_passes = 1;
    if (a.strategy == RELATE_CONFLICT_SEGMENTED && a.tperm && vec_ok && a.depth >= 1 && a.N >= 3 && a.N <= 5 &&
        a.S % 4 == 0 && a.R % V == 0) {
        // the fiber-factored kernel (mttkrp_fac.cuh): per-block copies of the
        // hot rows as for the SEGMENTED kernel
        if (a.kr_table && a.kr_mul && a.depth >= 2 && a.N - 1 - a.depth == 1 &&
            (reinterpret_cast<uintptr_t>(a.kr_table) % 16) == 0) {
            // slots depth and depth + 1 as one slot over the Khatri-Rao rows
            a.rfac[a.N - 2] = a.kr_table;
            a.N -= 1;
            a.depth -= 1;
        } else {
            a.kr_mul = 0;
        }
        int hot = 0;
        a.full_copy = 0;
        if (a.hot_scratch && (size_t)a.In * a.R * accb <= kHotBlockBytes) {
            // a short mode: all its rows in the block's copy
            a.full_copy = 1;
            hot = (int)a.In;
        } else if (a.hot_rows && a.In < (1ull << 31) && a.maxcount >= kSegHotMinCount && a.hot_scratch) {
            hot = (int)(kHotBlockBytes / ((size_t)a.R * accb));
            if (hot > mk::kTagMax) hot = mk::kTagMax;
            if (hot > kHotMax) hot = kHotMax;
            if ((uint64_t)hot > a.In) hot = (int)a.In;
        }
        a.hot_n = hot;
        const int64_t tiles = a.P * ((a.S + mk::kTile - 1) / mk::kTile);
        switch (factor_dtype) {
        case RELATE_F64: return mttkrp_fac_f64(a, KW, tiles, num_sms, st);
        case RELATE_F32: return mttkrp_fac_f32(a, KW, tiles, num_sms, st);
        default: return mttkrp_fac_bf16(a, KW, tiles, num_sms, st);
        }
    }
    a.depth = 0;
    fill_slots(a);
    const size_t tile = mk::tile_bytes_for(a.N, KW, factor_dtype, vec_ok, a.vals_f64 ? 8 : 4);
    size_t acc_bytes = 0;
    if (a.strategy == RELATE_CONFLICT_PRIVATIZED && (size_t)a.In * a.R * accb + 16 + tile > (size_t)smem_budget)
        a.strategy = RELATE_CONFLICT_SEGMENTED;  // the whole output does not fit: sort tiles instead
    if (a.strategy == RELATE_CONFLICT_PRIVATIZED) {
        a.hot_n = 0;
        acc_bytes = (size_t)a.In * a.R * accb;
    } else {
        // hot rows: up to 16 KB of accumulators
        // Hot rows of unsorted tiles (ATOMIC) accumulate in shared memory:
        // their runs are short and would contend on the same global lines.
        // Sorted tiles (SEGMENTED) merge each row's run in registers first,
        // so their flushes go straight to global memory. Runs are tagged
        // 0x80000000|slot, so the hot path needs rows < 2^31.
        // SEGMENTED tiles keep their hottest rows in per-block copies in
        // global scratch (8 KB per block, no shared memory), and only in modes
        // whose hottest row has enough nonzeros for its global additions to
        // matter.
        int hot = 0;
        a.full_copy = 0;
        const bool seg_k = a.strategy == RELATE_CONFLICT_SEGMENTED && a.hot_scratch && a.tperm && vec_ok && a.N >= 2 &&
                           a.N <= 5;  // the compile-time SEGMENTED kernel
        if (seg_k && (size_t)a.In * a.R * accb <= kHotBlockBytes) {
            // a short mode: all its rows in the block's copy (slot = row)
            a.full_copy = 1;
            hot = (int)a.In;
        } else if (a.hot_rows && a.In < (1ull << 31)) {
            if (a.strategy == RELATE_CONFLICT_ATOMIC)
                hot = (16 * 1024) / (a.R * accb);
            else if (seg_k && a.maxcount >= kSegHotMinCount) {
                hot = (int)(kHotBlockBytes / ((size_t)a.R * accb));
                if (hot > mk::kTagMax) hot = mk::kTagMax;  // slots a tile-order entry can tag
            }
            if (hot > kHotMax) hot = kHotMax;
            if ((uint64_t)hot > a.In) hot = (int)a.In;
        }
        a.hot_n = hot;
        acc_bytes = a.strategy == RELATE_CONFLICT_ATOMIC ? (size_t)hot * a.R * accb : 0;
    }
    // the compile-time SEGMENTED kernel (tile order present, vector path, N <= 5) needs less shared memory
    const bool seg_kernel = a.strategy == RELATE_CONFLICT_SEGMENTED && a.tperm && vec_ok && a.N >= 2 && a.N <= 5;
    const size_t smem = acc_bytes + 16 +
                        (seg_kernel ? mk::tile_bytes_for(a.N, KW, factor_dtype, vec_ok, a.vals_f64 ? 8 : 4, true) : tile);
    int per_sm = (int)((227 * 1024) / (smem + 1024));
    if (per_sm > 3) per_sm = 3;
    if (per_sm < 1) per_sm = 1;
    const int64_t tiles = a.P * ((a.S + mk::kTile - 1) / mk::kTile);
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    if (a.strategy == RELATE_CONFLICT_SEGMENTED && a.hot_n && (size_t)grid * kHotBlockBytes > kHotScratchBytes) {
        a.hot_n = 0;  // more blocks than scratch copies (over 1024): no hot copies
        a.full_copy = 0;
    }
    switch (factor_dtype) {
    case RELATE_F64: return mttkrp_f64(a, KW, vec_ok, acc_bytes, (int)grid, st);
    case RELATE_F32: return mttkrp_f32(a, KW, vec_ok, acc_bytes, (int)grid, st);
    default: return mttkrp_bf16(a, KW, vec_ok, acc_bytes, (int)grid, st);
    }
}

template <typename T, typename V>
__global__ void __launch_bounds__(256) k_kr_rows(const T *__restrict__ A, const T *__restrict__ B, uint32_t Ib,
                                                 uint32_t rows, int nv, T *__restrict__ out) {
    constexpr int E = sizeof(V) / sizeof(T);
    const int lane = threadIdx.x & 31;
    const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t row = w0; row < rows; row += nw) {
        const uint32_t ia = row / Ib, ib = row - ia * Ib;
        for (int c = lane; c < nv; c += 32) {
            const V x = reinterpret_cast<const V *>(A + (size_t)ia * nv * E)[c];
            const V y = reinterpret_cast<const V *>(B + (size_t)ib * nv * E)[c];
            V z;
            const T *px = reinterpret_cast<const T *>(&x), *py = reinterpret_cast<const T *>(&y);
            T *pz = reinterpret_cast<T *>(&z);
#pragma unroll
            for (int i = 0; i < E; i++) pz[i] = px[i] * py[i];
            reinterpret_cast<V *>(out + (size_t)row * nv * E)[c] = z;
        }
    }
}

cudaError_t launch_kr_rows(const void *A, const void *B, uint64_t Ia, uint64_t Ib, int R, int dtype, void *out,
                           cudaStream_t st) {
    const uint64_t rows = Ia * Ib;
    if (rows == 0) return cudaSuccess;
    if (rows >= (1ull << 32) || R < 2 || R % 2 || (dtype != RELATE_F64 && dtype != RELATE_F32))
        return cudaErrorInvalidValue;
    const int threads = 256;
    int64_t blocks = (int64_t)((rows + 7) / 8);  // 8 warps per block, a row per warp and step
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (dtype == RELATE_F64)
        k_kr_rows<double, double2><<<(unsigned)blocks, threads, 0, st>>>(
            (const double *)A, (const double *)B, (uint32_t)Ib, (uint32_t)rows, R / 2, (double *)out);
    else if (R % 4 == 0)
        k_kr_rows<float, float4><<<(unsigned)blocks, threads, 0, st>>>(
            (const float *)A, (const float *)B, (uint32_t)Ib, (uint32_t)rows, R / 4, (float *)out);
    else
        k_kr_rows<float, float2><<<(unsigned)blocks, threads, 0, st>>>(
            (const float *)A, (const float *)B, (uint32_t)Ib, (uint32_t)rows, R / 2, (float *)out);
    return cudaGetLastError();
}

int tile_order_hot_rows(const MttkrpArgs &a) {
    if (!a.hot_rows || a.In >= (1ull << 31) || a.maxcount < kSegHotMinCount) return 0;
    uint64_t hot = mk::kTagMax;
    if (hot > (uint64_t)kHotMax) hot = kHotMax;
    if (hot > a.In) hot = a.In;
    return (int)hot;
}

cudaError_t launch_tile_order(const MttkrpArgs &a_in, int KW, int num_sms, uint16_t *tperm, cudaStream_t st) {
    MttkrpArgs a = a_in;
    if (a.nnz == 0 || a.P == 0) return cudaSuccess;
    a.hot_n = tile_order_hot_rows(a);
    const int64_t tiles = a.P * ((a.S + mk::kTile - 1) / mk::kTile);
    if (a.depth >= 1) {  // fiber-factored mode: tiles sorted by (i_n, slots 1..depth)
        fill_slots(a);
    }
    if (a.depth >= 1) {
        int64_t g = (int64_t)num_sms * 4;
        if (g > tiles) g = tiles;
        int bits = mk::kTileBits;  // key width: the row, the level fields, the position
        for (int s = 0; s <= a.depth; s++) bits += __builtin_popcount(a.rmask[s]);
        const bool k64 = bits <= 64;
#define RELATE_TOL(KW_)                                                                            \
    (k64 ? (mk::k_tile_order_lex<KW_, true><<<(unsigned)g, kThreads, 0, st>>>(a, tperm), 0)        \
         : (mk::k_tile_order_lex<KW_, false><<<(unsigned)g, kThreads, 0, st>>>(a, tperm), 0))
        switch (KW) {
        case 1: RELATE_TOL(1); break;
        case 2: RELATE_TOL(2); break;
        default: RELATE_TOL(4); break;
        }
#undef RELATE_TOL
        return cudaGetLastError();
    }
    int64_t grid = (int64_t)num_sms * 4;
    if (grid > tiles) grid = tiles;
    switch (KW) {
    case 1: mk::k_tile_order<1><<<(unsigned)grid, kThreads, 0, st>>>(a, tperm); break;
    case 2: mk::k_tile_order<2><<<(unsigned)grid, kThreads, 0, st>>>(a, tperm); break;
    default: mk::k_tile_order<4><<<(unsigned)grid, kThreads, 0, st>>>(a, tperm); break;
    }
    return cudaGetLastError();
}

}  // namespace relate

namespace relate {

bool batch_eligible(const MttkrpArgs &a, int factor_dtype) {
    const int accb = mttkrp_acc_bytes(factor_dtype);
    const int fb = factor_dtype == RELATE_F64 ? 8 : factor_dtype == RELATE_F32 ? 4 : 2;
    if (a.N < 2 || a.N > 5 || !a.tperm || a.S % 4 != 0 || a.nnz == 0 || a.P == 0) return false;
    if ((a.R * fb) % 16 != 0 || (a.R * accb) % 16 != 0 || (reinterpret_cast<uintptr_t>(a.out) % 16) != 0) return false;
    for (int k = 0; k < a.N; k++)
        if (k != a.mode && (reinterpret_cast<uintptr_t>(a.factors[k]) % 16) != 0) return false;
    return true;
}

cudaError_t launch_mttkrp_batch(const MttkrpArgs *items, int n, int KW, int factor_dtype, int num_sms,
                                cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (n > mk::kBatchMax) return cudaErrorInvalidValue;
    const int V = factor_dtype == RELATE_F64 ? 2 : 4;
    mk::BatchParams bp{};
    bp.n = n;
    bp.wait_cycles = items[0].wait_cycles > 0 ? items[0].wait_cycles : kWaitCycles;
    bp.fault_skip_copy = items[0].fault_skip_copy;
    bp.tile_begin[0] = 0;
    for (int i = 0; i < n; i++) {
        MttkrpArgs a = items[i];
        a.depth = 0;
        fill_slots(a);  // slot 0 = the output mode, then the other modes in increasing order
        mk::BatchItem &it = bp.it[i];
        it.words = a.words;
        it.vals = a.vals;
        it.tperm = a.tperm;
        it.nnz = a.nnz;
        it.S = a.S;
        it.P = a.P;
        it.tiles_per_part = (a.S + mk::kTile - 1) / mk::kTile;
        it.out = a.out;
        it.R = a.R;
        const int nvec = (a.R + V - 1) / V;
        int G = 1, log2G = 0;
        while (G < nvec && G < 32) {
            G <<= 1;
            log2G++;
        }
        it.log2G = log2G;
        it.vals_f64 = a.vals_f64;
        it.err = a.err;
        for (int k = 0; k < kMaxModes; k++) {
            it.rshift[k] = a.rshift[k];
            it.rmask[k] = a.rmask[k];
            it.rfac[k] = a.rfac[k];
        }
        bp.tile_begin[i + 1] = bp.tile_begin[i] + a.P * it.tiles_per_part;
    }
    switch (factor_dtype) {
    case RELATE_F64: return mttkrp_batch_f64(bp, items[0].N, KW, num_sms, st);
    case RELATE_F32: return mttkrp_batch_f32(bp, items[0].N, KW, num_sms, st);
    default: return mttkrp_batch_bf16(bp, items[0].N, KW, num_sms, st);
    }
}

}  // namespace relate
