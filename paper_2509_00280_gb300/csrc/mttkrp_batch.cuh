// mttkrp_batch.cuh -- one persistent MTTKRP launch over the tiles of several
// MTTKRPs (included by mttkrp_impl.cuh inside namespace relate::mk).
//
// The per-nonzero MTTKRP of Sec. 2.2 (Fig. 2), for a batch of small problems
// (the requests of a CP-ALS service): each item is one mode of one encoded
// tensor with its own factors, rank and output. The items' tiles are numbered
// one after the other; a resident grid walks the global tile range
// grid-stride, and each tile is processed as in the SEGMENTED kernel: TMA
// staging of the words and values, records at the positions of the item's
// precomputed tile order, runs of equal output rows merged in registers and
// added with vector atomics. Items share (N, key width, factor type); rank,
// sizes, strategy and pointers are per item. No per-block copies of hot rows
// (small items take few tiles per row) and no privatised outputs (a block
// moves between items).

constexpr int kBatchMax = kBatchItems;  // items per launch (kernel parameter space)

struct BatchItem {
    const void *words;
    const void *vals;
    const uint16_t *tperm;
    int64_t nnz, S, P;
    int64_t tiles_per_part;
    void *out;
    int R;
    int log2G;
    int vals_f64;
    int *err;
    int rshift[kMaxModes];
    uint32_t rmask[kMaxModes];
    const void *rfac[kMaxModes];
};

struct BatchParams {
    int n;
    long long wait_cycles;
    int fault_skip_copy;
    int64_t tile_begin[kBatchMax + 1];  // item i owns global tiles [tile_begin[i], tile_begin[i + 1])
    BatchItem it[kBatchMax];
};

template <int NT, int KW, typename FT, int VEC>
__global__ void __launch_bounds__(kThreads, 3) k_mttkrp_batch(const __grid_constant__ BatchParams bp) {
    using C = typename Prec<FT>::C;
    using Word = typename WordT<KW>::T;
    using R_t = Rec<NT, C>;
    constexpr int RB = RecStride<NT, C>::B;
    static_assert(sizeof(R_t) == RB, "records are indexed as an array of R_t");
    constexpr int U = Unroll<FT, 1>::U;
    constexpr int NI = R_t::NI;
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int lane = threadIdx.x & 31;
    const int64_t ntiles = bp.tile_begin[bp.n];
    // shared layout: raw words | raw values (8 bytes each, either dtype) | records | mbarrier
    Word *sw = reinterpret_cast<Word *>(smem_raw);
    unsigned char *sv = smem_raw + (size_t)kTile * sizeof(Word);
    unsigned char *srec = sv + (size_t)kTile * 8;
    uint64_t *bar = reinterpret_cast<uint64_t *>(srec + (size_t)kTile * RB);

    auto item_of = [&](int64_t tq) -> int {
        int i = 0;
        while (i + 1 < bp.n && bp.tile_begin[i + 1] <= tq) i++;
        return i;
    };
    // tile tq: its item, its first nonzero and its size
    auto tile_span = [&](int64_t tq, int &i, int64_t &b, int &nt) {
        i = item_of(tq);
        const BatchItem &it = bp.it[i];
        const int64_t lt = tq - bp.tile_begin[i];
        const int64_t q = lt / it.tiles_per_part;
        b = q * it.S + (lt - q * it.tiles_per_part) * kTile;
        const int64_t pe = min(q * it.S + it.S, it.nnz);
        nt = (int)max((int64_t)0, min((int64_t)kTile, pe - b));
    };
    auto issue = [&](int64_t tq) {  // one thread: stage tile tq through TMA
        int i, nt;
        int64_t b;
        tile_span(tq, i, b, nt);
        if (nt == 0) return;
        const BatchItem &it = bp.it[i];
        const int vb = it.vals_f64 ? 8 : 4;
        const uint32_t wbytes = (uint32_t)((nt * sizeof(Word) + 15) & ~(size_t)15);
        const uint32_t vbytes = (uint32_t)((nt * vb + 15) & ~15);
        mbar_expect_tx(bar, wbytes + vbytes);
        bulk_g2s(sw, reinterpret_cast<const Word *>(it.words) + b, wbytes, bar);
        bulk_g2s(sv, reinterpret_cast<const unsigned char *>(it.vals) + b * vb, vbytes, bar);
    };
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && blockIdx.x < ntiles && !bp.fault_skip_copy) issue(blockIdx.x);
    uint32_t phase = 0;

    for (int64_t tq = blockIdx.x; tq < ntiles; tq += gridDim.x) {
        int ii, nt;
        int64_t b;
        tile_span(tq, ii, b, nt);
        if (nt == 0) {
            if (threadIdx.x == 0 && tq + gridDim.x < ntiles) issue(tq + gridDim.x);
            continue;
        }
        const BatchItem &it = bp.it[ii];
        {
            const bool ok = mbar_wait_bounded(bar, phase, bp.wait_cycles);
            phase ^= 1;
            if (__syncthreads_or(!ok)) {  // a copy never landed: report and stop
                if (threadIdx.x == 0) atomicOr(it.err, 1);
                return;
            }
        }
        // ---- records at their positions in the item's tile order (rows contiguous)
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            const int j = k * kThreads + threadIdx.x;
            if (j >= nt) continue;
            const Word w = sw[j];
            const uint32_t p = __ldg(it.tperm + b + j) & (kTile - 1);
            R_t rec;
            rec.val = it.vals_f64 ? (C)reinterpret_cast<const double *>(sv)[j] : (C)reinterpret_cast<const float *>(sv)[j];
#pragma unroll
            for (int s = 0; s < NI; s++) rec.idx[s] = fld(w, it.rshift[s], it.rmask[s]);
            *reinterpret_cast<R_t *>(srec + (size_t)p * RB) = rec;
        }
        __syncthreads();  // records complete; the raw stage is free
        if (threadIdx.x == 0 && tq + gridDim.x < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(tq + gridDim.x);  // lands while this tile computes
        }
        // ---- groups of G lanes walk contiguous record slices (boundaries moved to row changes)
        const int log2G = it.log2G;
        const int G = 1 << log2G;
        const int gl = lane & (G - 1);
        const int gid = threadIdx.x >> log2G;
        const int ngroups = kThreads >> log2G;
        const int R = it.R;
        const bool act = gl * VEC < R;
        const R_t *recs = reinterpret_cast<const R_t *>(srec);
        const int chunk = (nt + ngroups - 1) / ngroups;
        auto snap = [&](int x) -> int {
            if (x <= 0 || x >= nt || chunk < kSnap) return min(max(x, 0), nt);
            const uint32_t prev = recs[x - 1].idx[0];
            for (int y = x; y < nt && y < x + kSnap; y++)
                if (recs[y].idx[0] != prev) return y;
            return x;
        };
        const int jb = snap(gid * chunk);
        const int je = snap((gid + 1) * chunk);
        C *__restrict__ out = reinterpret_cast<C *>(it.out);
        const uint32_t loff = (uint32_t)gl * VEC * (uint32_t)sizeof(FT);
        const uint32_t rbytes = (uint32_t)R * (uint32_t)sizeof(FT);
        uint32_t cur = 0xffffffffu;
        C acc[VEC];
#pragma unroll
        for (int i = 0; i < VEC; i++) acc[i] = C(0);
        auto flush = [&](uint32_t row) {
            if (act) GAdd<C, VEC>::run(out + (int64_t)row * R + gl * VEC, acc);
        };
        for (int p0 = jb; p0 < je; p0 += U) {
            R_t rec[U];
            C t[U][VEC];
#pragma unroll
            for (int u = 0; u < U; u++) rec[u] = recs[min(p0 + u, je - 1)];
#pragma unroll
            for (int k = 1; k < NI; k++) {
                C x[U][VEC];
#pragma unroll
                for (int u = 0; u < U; u++)
                    if (act)
                        VecLoadP<FT, VEC>::run(reinterpret_cast<const char *>(it.rfac[k]) +
                                                   ((uint64_t)rec[u].idx[k] * rbytes + loff),
                                               x[u]);
#pragma unroll
                for (int u = 0; u < U; u++)
#pragma unroll
                    for (int i = 0; i < VEC; i++) t[u][i] = k == 1 ? x[u][i] : t[u][i] * x[u][i];
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (p0 + u >= je) continue;
                const uint32_t row = rec[u].idx[0];
                const C v = rec[u].val;
                if (row != cur) {
                    if (cur != 0xffffffffu) flush(cur);
                    cur = row;
#pragma unroll
                    for (int i = 0; i < VEC; i++) acc[i] = v * t[u][i];
                } else {
#pragma unroll
                    for (int i = 0; i < VEC; i++) acc[i] = fma(v, t[u][i], acc[i]);
                }
            }
        }
        if (cur != 0xffffffffu) flush(cur);
        __syncthreads();  // the records are rewritten by the next tile
    }
}

template <int NT, int KW, typename FT>
cudaError_t launch_batch_one(const BatchParams &bp, int num_sms, cudaStream_t st) {
    using C = typename Prec<FT>::C;
    constexpr int V = Prec<FT>::VEC;
    const size_t smem = (size_t)kTile * (4 * KW) + (size_t)kTile * 8 + (size_t)kTile * RecStride<NT, C>::B + 16;
    auto kern = k_mttkrp_batch<NT, KW, FT, V>;
    cudaError_t e = allow_max_dynamic_smem(kern);
    if (e != cudaSuccess) return e;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem)) != cudaSuccess) return e;
    int64_t grid = (int64_t)num_sms * (occ > 0 ? occ : 1);
    if (grid > bp.tile_begin[bp.n]) grid = bp.tile_begin[bp.n];
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, kThreads, smem, st>>>(bp);
    return cudaGetLastError();
}

template <typename FT>
cudaError_t dispatch_batch(const BatchParams &bp, int N, int KW, int num_sms, cudaStream_t st) {
#define RELATE_BATCH_KW(NT_)                                                                      \
    (KW == 1 ? launch_batch_one<NT_, 1, FT>(bp, num_sms, st)                                      \
             : KW == 2 ? launch_batch_one<NT_, 2, FT>(bp, num_sms, st) : launch_batch_one<NT_, 4, FT>(bp, num_sms, st))
    switch (N) {
    case 2: return RELATE_BATCH_KW(2);
    case 3: return RELATE_BATCH_KW(3);
    case 4: return RELATE_BATCH_KW(4);
    case 5: return RELATE_BATCH_KW(5);
    default: return cudaErrorInvalidValue;
    }
#undef RELATE_BATCH_KW
}
