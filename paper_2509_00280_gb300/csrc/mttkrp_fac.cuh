// mttkrp_fac.cuh -- the fiber-factored SEGMENTED MTTKRP (included by
// mttkrp_impl.cuh inside namespace relate::mk).
//
// The per-nonzero MTTKRP of Sec. 2.2 (Fig. 2), regrouped by distributivity.
// Within a tile sorted by (i_n, i_{p1}, ..., i_{pD}) (p = the mode's level
// order of the other modes), the nonzeros sharing (i_n, i_{p1..pl}) form a
// fiber of level l, and
//   M(i_n, :) = sum_{i_p1} A_p1(i_p1, :) * ( sum_{i_p2} A_p2(i_p2, :) * ( ...
//               sum_{nonzeros of the level-D fiber} v * prod_{s > D} A_ps(i_ps, :) ))
// so a level-l factor row is gathered and multiplied once per level-l fiber
// instead of once per nonzero. With no repeated fibers the arithmetic is one
// fused multiply-add per mode and element, as the flat loop's multiplies
// plus one addition; every repeat saves a gather and a multiply. The sums are
// the same terms as the flat loop's, in another association order (FP64:
// rounding differences only).
//
// With a Khatri-Rao pair (MttkrpArgs::kr_table) the launcher hands this
// kernel N - 1 slots and depth - 1 levels: the last slot then indexes the
// rows of A_a (.) A_b of the deepest level's mode a and the innermost mode b,
// so v * (A_a (.) A_b)(i_a, i_b) is summed straight into the next level out
// (the tile order, sorted by mode a too, keeps those rows together).
//
// Layout as the SEGMENTED kernel: 2048-nonzero tiles staged by TMA, records
// {value, i_n, i_p1, ..., i_p(N-1)} at their sorted positions from the
// mode's precomputed tile order; per record the lowest slot at which it
// differs from the next record ("end level", 0 = the output row changes) is
// computed once per tile in shared memory. A group of G lanes walks a slice
// of records keeping one running sum per level (VEC elements per lane) and
// closes the levels a record ends. col_passes > 1 walks the records once per
// chunk of R / col_passes columns (narrower groups, half the row bytes per
// gather per pass).

// 128-bit key builder: (hi, lo) <- (hi, lo) << w | v, for 1 <= w <= 32.
__device__ __forceinline__ void push_bits(unsigned long long &hi, unsigned long long &lo, uint32_t v, int w) {
    hi = (hi << w) | (lo >> (64 - w));
    lo = (lo << w) | (unsigned long long)v;
}

// Bits of a coordinate field (its mask is 2^l - 1).
__device__ __forceinline__ int field_width(uint32_t mask) { return __popc(mask); }

// Tile order of a fiber-factored mode: every tile sorted by (i_n, slot 1, ...,
// slot depth, position in the tile), a bitonic sort of the concatenated keys
// in shared memory (64-bit when the fields and the 11 position bits fit, else
// 128-bit); entries as k_tile_order's (sorted position | (1 + hot slot) << 11).
// One block per tile, grid-stride.
template <int KW, bool K64>
__global__ void __launch_bounds__(kThreads) k_tile_order_lex(const MttkrpArgs a, uint16_t *__restrict__ tperm) {
    __shared__ unsigned long long klo[kTile];
    __shared__ unsigned long long khi[K64 ? 1 : kTile];
    __shared__ uint32_t srow[kTile];
    __shared__ uint32_t hkey[kHotHash], hval[kHotHash];
    const int hot_n = a.hot_n, D = a.depth;
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
        __syncthreads();  // the previous tile's keys are consumed
        for (int j = threadIdx.x; j < kTile; j += kThreads) {
            unsigned long long hi = ~0ull, lo = ~0ull;  // padding sorts last
            if (j < nt) {
                const auto w = load_word<KW>(a.words, b + j);
                hi = lo = 0ull;
                const uint32_t row = fld(w, a.rshift[0], a.rmask[0]);
                srow[j] = row;
                if (a.rmask[0]) push_bits(hi, lo, row, field_width(a.rmask[0]));
                for (int s = 1; s <= D; s++)
                    if (a.rmask[s]) push_bits(hi, lo, fld(w, a.rshift[s], a.rmask[s]), field_width(a.rmask[s]));
                push_bits(hi, lo, (uint32_t)j, kTileBits);
            }
            klo[j] = lo;
            if (!K64) khi[j] = hi;
        }
        __syncthreads();
        for (int k = 2; k <= kTile; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int i = threadIdx.x; i < kTile; i += kThreads) {
                    const int ixj = i ^ jj;
                    if (ixj > i) {
                        const unsigned long long alo = klo[i], blo = klo[ixj];
                        if (K64) {
                            if ((alo > blo) == ((i & k) == 0)) {
                                klo[i] = blo;
                                klo[ixj] = alo;
                            }
                        } else {
                            const unsigned long long ahi = khi[i], bhi = khi[ixj];
                            const bool gt = ahi > bhi || (ahi == bhi && alo > blo);
                            if (gt == ((i & k) == 0)) {
                                khi[i] = bhi;
                                klo[i] = blo;
                                khi[ixj] = ahi;
                                klo[ixj] = alo;
                            }
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int p = threadIdx.x; p < nt; p += kThreads) {
            const int j = (int)(klo[p] & (kTile - 1));
            const uint32_t tag = hot_n ? hot_tag(srow[j]) : 0u;
            tperm[b + j] = (uint16_t)((uint32_t)p | (tag << kTileBits));
        }
    }
}

// Blocks per SM the register budget aims at: 3 for 3-mode FP32 / BF16 rows
// (4 records of two 16-byte row slices in flight fit 80 registers), else 2.
template <int NT, typename FT> struct FacCfg {
    static constexpr int MinBlocks = (sizeof(FT) < 8 && NT == 3) ? 3 : 2;
    static constexpr int U = 4;
};

template <int NT, int KW, typename FT, int VEC, int D>
__global__ void __launch_bounds__(kThreads, FacCfg<NT, FT>::MinBlocks) k_mttkrp_fac(const MttkrpArgs a, const int log2G) {
    using C = typename Prec<FT>::C;
    using Word = typename WordT<KW>::T;
    using R_t = Rec<NT, C>;
    constexpr int RB = RecStride<NT, C>::B;
    static_assert(sizeof(R_t) == RB, "records are indexed as an array of R_t");
    static_assert(D >= 1 && D <= NT - 2, "factored levels: 1 .. N-2");
    constexpr int NI = NT;
    constexpr int U = FacCfg<NT, FT>::U;  // records in flight per group
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int next_chunk;       // the next unclaimed chunk of the tile (G = 32)
    constexpr int kChunk = 64;       // records per claimed chunk

    const int G = 1 << log2G;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int gid = threadIdx.x >> log2G;
    const int ngroups = kThreads >> log2G;
    const int R = a.R;
    const int passes = a.col_passes;
    const int Rc = R / passes;  // columns per pass (the launcher keeps R % passes == 0 and Rc % VEC == 0)
    const bool act = gl * VEC < Rc;
    const int hot_n = a.hot_n;
    const int vb = a.vals_f64 ? 8 : 4;
    C *__restrict__ out = reinterpret_cast<C *>(a.out);
    C *__restrict__ hrep = hot_n ? reinterpret_cast<C *>(a.hot_scratch) + (int64_t)blockIdx.x * hot_n * R : nullptr;

    // shared layout: raw words | raw values | records | end levels | mbarrier
    Word *sw = reinterpret_cast<Word *>(smem_raw);
    unsigned char *sv = smem_raw + (size_t)kTile * sizeof(Word);
    unsigned char *srec = sv + (size_t)kTile * vb;
    uint8_t *rend = srec + (size_t)kTile * RB;
    uint64_t *bar = reinterpret_cast<uint64_t *>(rend + kTile);

    if (hot_n)  // ordered before this block's atomics by the barriers that follow
        for (int i = threadIdx.x; i < hot_n * R; i += kThreads) hrep[i] = C(0);

    const int64_t tiles_per_part = (a.S + kTile - 1) / kTile;
    const int64_t ntiles = a.P * tiles_per_part;
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
    // the launcher guarantees partitions of a multiple of 4 nonzeros (16-byte tile starts)
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && blockIdx.x < ntiles && !a.fault_skip_copy) issue(blockIdx.x);
    uint32_t phase = 0;

    for (int64_t tq = blockIdx.x; tq < ntiles; tq += gridDim.x) {
        int64_t b;
        int nt;
        tile_span(tq, b, nt);
        if (nt == 0) {
            if (threadIdx.x == 0 && tq + gridDim.x < ntiles) issue(tq + gridDim.x);
            continue;
        }
        {
            const bool ok = mbar_wait_bounded(bar, phase, a.wait_cycles);
            phase ^= 1;
            if (__syncthreads_or(!ok)) {  // a copy never landed: report and stop
                if (threadIdx.x == 0) atomicOr(a.err, 1);
                return;
            }
        }
        // ---- decode each nonzero once into its record at its sorted position
#pragma unroll
        for (int i = 0; i < kItems; i++) {
            const int j = i * kThreads + threadIdx.x;
            if (j >= nt) continue;
            const Word w = sw[j];
            const uint32_t e = __ldg(a.tperm + b + j);
            const uint32_t p = e & (kTile - 1);
            uint32_t hbin = e >> kTileBits;
            if (hbin > (uint32_t)hot_n) hbin = 0;  // tagged for a larger hot set
            R_t rec;
            rec.val = a.vals_f64 ? (C)reinterpret_cast<const double *>(sv)[j] : (C)reinterpret_cast<const float *>(sv)[j];
#pragma unroll
            for (int k = 0; k < NI; k++) rec.idx[k] = fld(w, a.rshift[k], a.rmask[k]);
            if (a.kr_mul)  // the last slot indexes the Khatri-Rao rows of two modes
                rec.idx[NI - 1] = rec.idx[NI - 1] * a.kr_mul + fld(w, a.rshift[NI], a.rmask[NI]);
            if (a.full_copy) rec.idx[0] |= 0x80000000u;  // every row has its slot: the row itself
            else if (hbin) rec.idx[0] = 0x80000000u | (hbin - 1u);
            *reinterpret_cast<R_t *>(srec + (size_t)p * RB) = rec;
        }
        __syncthreads();  // records complete; the raw stage is free
        if (threadIdx.x == 0 && tq + gridDim.x < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(tq + gridDim.x);  // lands while this tile computes
        }
        const R_t *recs = reinterpret_cast<const R_t *>(srec);
        // ---- end level of every record: the lowest slot (0..D) at which it
        // differs from the next record, D + 1 if none, 0 for the tile's last
        for (int p = threadIdx.x; p < nt; p += kThreads) {
            int e = 0;
            if (p + 1 < nt) {
                e = D + 1;
#pragma unroll
                for (int s = D; s >= 0; s--)
                    if (recs[p].idx[s] != recs[p + 1].idx[s]) e = s;
            }
            rend[p] = (uint8_t)e;
        }
        if (threadIdx.x == 0) next_chunk = 0;
        __syncthreads();

        // ---- slices: contiguous record ranges, boundaries moved forward to
        // the next change of output row (at most kSnap records). A group of a
        // whole warp (G = 32) takes kChunk-record chunks from a shared counter
        // until the tile is done, so that warps whose records close more
        // fibers (more FP64 work) do not hold the others at the tile's end;
        // narrower groups take one equal slice each.
        auto snap_to = [&](int x, int ch) -> int {
            if (x <= 0 || x >= nt || ch < kSnap) return min(max(x, 0), nt);
            for (int y = x - 1; y < nt - 1 && y < x - 1 + kSnap; y++)
                if (rend[y] == 0) return y + 1;
            return x;
        };
        auto process = [&](const int jb, const int je) {
        for (int pass = 0; pass < passes; pass++) {
            const int c0 = pass * Rc;  // first column of this pass
            const uint32_t loff = (uint32_t)(c0 + gl * VEC) * (uint32_t)sizeof(FT);
            const uint32_t rbytes = (uint32_t)R * (uint32_t)sizeof(FT);
            C s[D + 1][VEC];  // s[0]: the output row; s[l]: the open level-l fiber
#pragma unroll
            for (int l = 0; l <= D; l++)
#pragma unroll
                for (int i = 0; i < VEC; i++) s[l][i] = C(0);
            auto rowp = [&](int slot, uint32_t idx) -> const char * {
                return reinterpret_cast<const char *>(a.rfac[slot]) + ((uint64_t)idx * rbytes + loff);
            };
            auto flush = [&](uint32_t row) {
                if (!act) return;
                C *dst = (hot_n && (row & 0x80000000u)) ? hrep + (int64_t)(row & 0x7fffffffu) * R
                                                        : out + (int64_t)row * R;
                GAdd<C, VEC>::run(dst + c0 + gl * VEC, s[0]);
            };
            for (int p0 = jb; p0 < je; p0 += U) {
                R_t rec[U];
                int e[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int p = min(p0 + u, je - 1);
                    rec[u] = recs[p];
                    e[u] = (p0 + u >= je - 1) ? 0 : (int)rend[p];  // a slice closes every level at its end
                }
                // gathers of all U records first: the unfactored slots always,
                // a level's row only where the record ends that level's fiber
                C x[U][NI - 1 - D][VEC];
                C y[U][D][VEC];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    if (!act) continue;
#pragma unroll
                    for (int k = D + 1; k < NI; k++) VecLoadP<FT, VEC>::run(rowp(k, rec[u].idx[k]), x[u][k - D - 1]);
#pragma unroll
                    for (int l = 1; l <= D; l++)
                        if (e[u] <= l && p0 + u < je) VecLoadP<FT, VEC>::run(rowp(l, rec[u].idx[l]), y[u][l - 1]);
                }
#pragma unroll
                for (int u = 0; u < U; u++) {
                    if (p0 + u >= je) continue;
                    const C v = rec[u].val;
                    // innermost: s[D] += v * prod of the unfactored rows
                    C t[VEC];
#pragma unroll
                    for (int i = 0; i < VEC; i++) t[i] = x[u][0][i];
#pragma unroll
                    for (int k = 1; k < NI - 1 - D; k++)
#pragma unroll
                        for (int i = 0; i < VEC; i++) t[i] *= x[u][k][i];
#pragma unroll
                    for (int i = 0; i < VEC; i++) s[D][i] = fma(v, t[i], s[D][i]);
                    // close the levels this record ends, innermost first. An
                    // FP64 instruction with its lanes predicated off still takes
                    // its slots in the narrow FP64 pipe, so when the warp is one
                    // group (G = 32, the condition is the same in every lane) a
                    // vote makes the close a branch that an open fiber skips
#pragma unroll
                    for (int l = D; l >= 1; l--) {
                        // a record that leaves level l open leaves every outer level open
                        const bool c = e[u] <= l;
                        if (!((sizeof(C) == 8 && G == 32) ? __any_sync(0xffffffffu, c) : c)) break;
#pragma unroll
                        for (int i = 0; i < VEC; i++) {
                            s[l - 1][i] = fma(s[l][i], y[u][l - 1][i], s[l - 1][i]);
                            s[l][i] = C(0);
                        }
                    }
                    if (e[u] == 0) {
                        flush(rec[u].idx[0]);
#pragma unroll
                        for (int i = 0; i < VEC; i++) s[0][i] = C(0);
                    }
                }
            }
        }
        };
        for (int round = 0;; round++) {  // one place that runs process(), so it is compiled once
            int x0, x1, ch;
            if (G == 32) {
                int ci = 0;
                if (lane == 0) ci = atomicAdd(&next_chunk, 1);
                ci = __shfl_sync(0xffffffffu, ci, 0);
                ch = kChunk;
                x0 = ci * kChunk;
                x1 = min(x0 + kChunk, nt);
            } else {
                ch = (nt + ngroups - 1) / ngroups;
                x0 = round == 0 ? gid * ch : nt;
                x1 = (gid + 1) * ch;
            }
            if (x0 >= nt) break;
            process(snap_to(x0, ch), snap_to(x1, ch));
        }
        __syncthreads();  // records and end levels are rewritten by the next tile
    }

    if (hot_n) {
        const int tot = hot_n * R;
        __threadfence();  // this block's atomics on its copy are complete
        __syncthreads();
        for (int i = threadIdx.x; i < tot; i += kThreads) {
            const C v = __ldcg(hrep + i);
            const uint32_t row = a.full_copy ? (uint32_t)(i / R) : __ldg(a.hot_rows + i / R);
            if (v != C(0) && row != 0xffffffffu) atomicAdd(out + (int64_t)row * R + i % R, v);
        }
    }
}

// Shared-memory bytes of the factored kernel's tile area.
template <int NT, int KW, typename C> constexpr size_t fac_tile_bytes(int vb) {
    return (size_t)kTile * (4 * KW) + (size_t)kTile * vb + (size_t)kTile * RecStride<NT, C>::B + kTile + 16;
}

// Launches the factored kernel: N = 3..5 on the vector path, depth 1..N-2.
template <int NT, int KW, typename FT, int D>
cudaError_t launch_fac_one(const MttkrpArgs &a_in, int64_t tiles, int num_sms, cudaStream_t st) {
    MttkrpArgs a = a_in;
    using C = typename Prec<FT>::C;
    constexpr int V = Prec<FT>::VEC;
    const int Rc = a.R / a.col_passes;
    const int nvec = (Rc + V - 1) / V;
    int G = 1, log2G = 0;
    while (G < nvec && G < 32) {
        G <<= 1;
        log2G++;
    }
    const size_t smem = fac_tile_bytes<NT, KW, C>(a.vals_f64 ? 8 : 4);
    auto kern = k_mttkrp_fac<NT, KW, FT, V, D>;
    cudaError_t e = allow_max_dynamic_smem(kern);
    if (e != cudaSuccess) return e;
    // one wave of resident blocks, walking the tiles grid-stride
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem)) != cudaSuccess) return e;
    int64_t grid = (int64_t)num_sms * (occ > 0 ? occ : 1);
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    if (a.hot_n && (size_t)grid * kHotBlockBytes > kHotScratchBytes) {  // more blocks than copies
        a.hot_n = 0;
        a.full_copy = 0;
    }
    kern<<<(unsigned)grid, kThreads, smem, st>>>(a, log2G);
    return cudaGetLastError();
}

template <int NT, typename FT, int D>
cudaError_t launch_fac_kw(const MttkrpArgs &a, int KW, int64_t tiles, int num_sms, cudaStream_t st) {
    return KW == 1 ? launch_fac_one<NT, 1, FT, D>(a, tiles, num_sms, st)
                   : KW == 2 ? launch_fac_one<NT, 2, FT, D>(a, tiles, num_sms, st)
                             : launch_fac_one<NT, 4, FT, D>(a, tiles, num_sms, st);
}

template <typename FT>
cudaError_t dispatch_fac(const MttkrpArgs &a, int KW, int64_t tiles, int num_sms, cudaStream_t st) {
    switch (a.N) {
    case 3: return launch_fac_kw<3, FT, 1>(a, KW, tiles, num_sms, st);
    case 4:
        return a.depth >= 2 ? launch_fac_kw<4, FT, 2>(a, KW, tiles, num_sms, st)
                            : launch_fac_kw<4, FT, 1>(a, KW, tiles, num_sms, st);
    case 5:
        return a.depth >= 3 ? launch_fac_kw<5, FT, 3>(a, KW, tiles, num_sms, st)
                            : a.depth == 2 ? launch_fac_kw<5, FT, 2>(a, KW, tiles, num_sms, st)
                                           : launch_fac_kw<5, FT, 1>(a, KW, tiles, num_sms, st);
    default: return cudaErrorInvalidValue;
    }
}

// Shared-memory bytes of the factored kernel's tile area for a launch.
inline size_t fac_tile_bytes_for(int N, int KW, int factor_dtype, int vb) {
    const bool f64 = factor_dtype == RELATE_F64;
#define RELATE_FAC_TB(NT_)                                                                            \
    (KW == 1 ? (f64 ? fac_tile_bytes<NT_, 1, double>(vb) : fac_tile_bytes<NT_, 1, float>(vb))        \
             : KW == 2 ? (f64 ? fac_tile_bytes<NT_, 2, double>(vb) : fac_tile_bytes<NT_, 2, float>(vb)) \
                       : (f64 ? fac_tile_bytes<NT_, 4, double>(vb) : fac_tile_bytes<NT_, 4, float>(vb)))
    switch (N) {
    case 3: return RELATE_FAC_TB(3);
    case 4: return RELATE_FAC_TB(4);
    default: return RELATE_FAC_TB(5);
    }
#undef RELATE_FAC_TB
}
