// dense.cu -- the dense remainder of CP-ALS around the MTTKRP.
//
// The paper accelerates CP decomposition (Sec. 2.2) and cites the standard
// ALS of Kolda & Bader for it; per mode n the update is
//   V = Hadamard_{k != n} (A_k^T A_k),  A_n = M V^{-1},
//   lambda_r = ||A_n(:, r)||_2, columns normalised,
// and after a sweep the fit uses ||X||^2 + lambda^T (Hadamard_k G_k) lambda
// - 2 <M, A_{N-1} diag(lambda)>. The normal-equations factorisation, the
// normalisation and the fit run in FP64 on the GPU (R <= 64, one block);
// the tall-skinny Gram and the row passes stream the I x R matrices.
#include "internal.cuh"

namespace relate {
namespace {

constexpr int GR_ROWS = 32;    // rows per staged tile of the Gram kernel
constexpr int GR_BLOCKS = 304; // 2 blocks per SM on 152 SMs
constexpr int MAXR = RELATE_MAX_RANK;
constexpr int MAXPAIRS = MAXR * (MAXR + 1) / 2;
constexpr int PAIRS_PER_THREAD = (MAXPAIRS + kThreads - 1) / kThreads;

template <typename FT> struct GramAcc { using T = float; };
template <> struct GramAcc<double> { using T = double; };

template <typename FT> __device__ __forceinline__ typename GramAcc<FT>::T ld_as(const FT *p) { return *p; }
template <> __device__ __forceinline__ float ld_as<__nv_bfloat16>(const __nv_bfloat16 *p) {
    return __bfloat162float(*p);
}

__device__ __forceinline__ void pair_of(int p, int R, int &r, int &s) {
    int row = 0, left = p;
    while (left >= R - row) {
        left -= R - row;
        row++;
    }
    r = row;
    s = row + left;
}

// Per-block partial of the upper triangle of A^T A. FP32/BF16 inputs
// accumulate in FP32 over the block's rows (at most a few thousand), FP64
// inputs in FP64; blocks are combined in FP64.
template <typename FT>
__global__ void __launch_bounds__(kThreads) k_gram_partial(const FT *__restrict__ A, int64_t I, int R,
                                                           double *__restrict__ partial) {
    using T = typename GramAcc<FT>::T;
    __shared__ T tile[GR_ROWS][MAXR + 1];
    const int npairs = R * (R + 1) / 2;
    int pr[PAIRS_PER_THREAD], ps[PAIRS_PER_THREAD];
    T acc[PAIRS_PER_THREAD];
#pragma unroll
    for (int u = 0; u < PAIRS_PER_THREAD; u++) {
        const int p = threadIdx.x + u * kThreads;
        pr[u] = ps[u] = 0;
        if (p < npairs) pair_of(p, R, pr[u], ps[u]);
        acc[u] = T(0);
    }
    // the next tile's elements are loaded into registers while this one computes
    constexpr int LD = (GR_ROWS * MAXR + kThreads - 1) / kThreads;
    T pre[LD];
    auto fetch = [&](int64_t r0) {
#pragma unroll
        for (int u = 0; u < LD; u++) {
            const int idx = threadIdx.x + u * kThreads;
            const int i = idx / R, c = idx - i * R;
            const int64_t row = r0 + i;
            pre[u] = (idx < GR_ROWS * R && row < I) ? ld_as<FT>(A + row * R + c) : T(0);
        }
    };
    fetch((int64_t)blockIdx.x * GR_ROWS);
    for (int64_t r0 = (int64_t)blockIdx.x * GR_ROWS; r0 < I; r0 += (int64_t)gridDim.x * GR_ROWS) {
#pragma unroll
        for (int u = 0; u < LD; u++) {
            const int idx = threadIdx.x + u * kThreads;
            if (idx < GR_ROWS * R) tile[idx / R][idx % R] = pre[u];
        }
        __syncthreads();
        fetch(r0 + (int64_t)gridDim.x * GR_ROWS);
#pragma unroll
        for (int u = 0; u < PAIRS_PER_THREAD; u++) {
            if (threadIdx.x + u * kThreads < npairs) {
                T s = acc[u];
#pragma unroll 8
                for (int i = 0; i < GR_ROWS; i++) s = fma(tile[i][pr[u]], tile[i][ps[u]], s);
                acc[u] = s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < PAIRS_PER_THREAD; u++) {
        const int p = threadIdx.x + u * kThreads;
        if (p < npairs) partial[(int64_t)blockIdx.x * npairs + p] = (double)acc[u];
    }
}

// Deterministic warp sum: lane l adds partials l, l+32, ... in order, then a
// fixed xor tree combines the lanes.
__device__ __forceinline__ double warp_sum_strided(const double *__restrict__ base, int n, int stride) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < n; b += 32) s += base[(int64_t)b * stride];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

__global__ void __launch_bounds__(kThreads) k_gram_reduce(const double *__restrict__ partial, int nblocks, int R,
                                                          double *__restrict__ G) {
    const int npairs = R * (R + 1) / 2;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int p = warp; p < npairs; p += nwarps) {
        const double s = warp_sum_strided(partial + p, nblocks, npairs);
        if ((threadIdx.x & 31) == 0) {
            int r, c;
            pair_of(p, R, r, c);
            G[r * R + c] = s;
            G[c * R + r] = s;
        }
    }
}

// V = Hadamard_{k != n} G_k, Cholesky (FP64, one ridge retry), V^{-1}.
// FP64 is a narrow pipe on GB300: square roots and reciprocals are computed
// once per column by one thread, the O(R^3) parts are spread over the block,
// and for FP32 / BF16 factors V^{-1} = L^{-T} L^{-1} is formed in FP32 from
// the FP64 L^{-1} (it is applied in FP32). V itself is kept (Vsave) for the
// fit's inner products.
__global__ void __launch_bounds__(kThreads) k_normal_eq(const double *__restrict__ G_all, int N, int n, int R,
                                                        double *__restrict__ Vinv, float *__restrict__ Vinv32,
                                                        double *__restrict__ Vsave, int f64_apply,
                                                        int *__restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double(*L)[MAXR + 1] = reinterpret_cast<double(*)[MAXR + 1]>(smem_raw);
    double(*Li)[MAXR + 1] = reinterpret_cast<double(*)[MAXR + 1]>(smem_raw + sizeof(double) * MAXR * (MAXR + 1));
    __shared__ double rdiag[MAXR];
    __shared__ int fail;
    __shared__ double ridge;
    const int RR = R * R;
    for (int attempt = 0; attempt < 2; attempt++) {
        for (int idx = threadIdx.x; idx < RR; idx += kThreads) {
            double v = 1.0;
            for (int k = 0; k < N; k++)
                if (k != n) v *= G_all[(int64_t)k * RR + idx];
            L[idx / R][idx % R] = v;
            if (attempt == 0) Vsave[idx] = v;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            double tr = 0.0;
            for (int r = threadIdx.x; r < R; r += 32) tr += L[r][r];
            for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
            if (threadIdx.x == 0) {
                fail = 0;
                if (attempt == 0) ridge = 1e-12 * tr / R;
            }
        }
        __syncthreads();
        if (attempt == 1)
            for (int r = threadIdx.x; r < R; r += kThreads) L[r][r] += ridge;
        __syncthreads();
        for (int j = 0; j < R; j++) {
            if (threadIdx.x == 0) {
                const double d = L[j][j];
                if (!(d > 0.0)) {
                    fail = 1;
                } else {
                    const double ljj = sqrt(d);
                    L[j][j] = ljj;
                    rdiag[j] = 1.0 / ljj;
                }
            }
            __syncthreads();
            if (fail) break;
            const double inv = rdiag[j];
            for (int i = j + 1 + threadIdx.x; i < R; i += kThreads) L[i][j] *= inv;
            __syncthreads();
            const int m = R - j - 1;
            for (int t = threadIdx.x; t < m * m; t += kThreads) {
                const int i = j + 1 + t / m, k = j + 1 + t % m;
                if (k <= i) L[i][k] = fma(-L[i][j], L[k][j], L[i][k]);
            }
            __syncthreads();
        }
        __syncthreads();
        if (!fail) break;
        if (threadIdx.x == 0 && attempt == 0) status[0] += 1;
        __syncthreads();
    }
    if (fail) {
        if (threadIdx.x == 0) status[1] = 1;
        for (int idx = threadIdx.x; idx < RR; idx += kThreads) {
            Vinv[idx] = 0.0;
            Vinv32[idx] = 0.0f;
        }
        return;
    }
    // L^{-1} column by column (forward substitution on unit vectors, FP64)
    for (int c = threadIdx.x; c < R; c += kThreads) {
        for (int i = 0; i < c; i++) Li[i][c] = 0.0;
        Li[c][c] = rdiag[c];
        for (int i = c + 1; i < R; i++) {
            double s = 0.0;
            for (int k = c; k < i; k++) s = fma(L[i][k], Li[k][c], s);
            Li[i][c] = -s * rdiag[i];
        }
    }
    __syncthreads();
    // V^{-1} = L^{-T} L^{-1}: FP64 for FP64 factors; otherwise L^{-1} is
    // rounded to FP32 once (reusing L's storage) and the product runs in FP32
    if (f64_apply) {
        for (int idx = threadIdx.x; idx < RR; idx += kThreads) {
            const int i = idx / R, j = idx % R;
            double s = 0.0;
            for (int k = max(i, j); k < R; k++) s = fma(Li[k][i], Li[k][j], s);
            Vinv[idx] = s;
            Vinv32[idx] = (float)s;
        }
    } else {
        float(*Lf)[MAXR + 1] = reinterpret_cast<float(*)[MAXR + 1]>(smem_raw);
        __syncthreads();  // L is no longer read
        for (int idx = threadIdx.x; idx < RR; idx += kThreads) Lf[idx / R][idx % R] = (float)Li[idx / R][idx % R];
        __syncthreads();
        for (int idx = threadIdx.x; idx < RR; idx += kThreads) {
            const int i = idx / R, j = idx % R;
            float s = 0.0f;
            for (int k = max(i, j); k < R; k++) s = fmaf(Lf[k][i], Lf[k][j], s);
            Vinv32[idx] = s;
        }
    }
}

// In place M <- M V^{-1}: one thread per row, V^{-1} broadcast from shared
// memory (zero-padded to RP columns), CC independent accumulators per
// thread; the row's inputs are re-read from L1 for each output chunk.
template <typename C, int RP>
__global__ void __launch_bounds__(kThreads) k_solve_rows(C *__restrict__ M, int64_t I, int R,
                                                         const C *__restrict__ Vinv) {
    constexpr int CC = sizeof(C) == 8 ? 16 : 32;  // output columns per pass
    constexpr int NC = (RP + CC - 1) / CC;
    __shared__ __align__(16) C Vs[MAXR][NC * CC];
    for (int idx = threadIdx.x; idx < MAXR * NC * CC; idx += kThreads) {
        const int r = idx / (NC * CC), c = idx % (NC * CC);
        Vs[r][c] = (r < R && c < R) ? Vinv[r * R + c] : C(0);
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < I; i += (int64_t)gridDim.x * kThreads) {
        C *row = M + i * R;
        C y[NC][CC];
#pragma unroll
        for (int q = 0; q < NC; q++)
#pragma unroll
            for (int c = 0; c < CC; c++) y[q][c] = C(0);
#pragma unroll 1
        for (int r = 0; r < R; r++) {
            const C xr = row[r];
#pragma unroll
            for (int q = 0; q < NC; q++)
#pragma unroll
                for (int c = 0; c < CC; c++) y[q][c] = fma(xr, Vs[r][q * CC + c], y[q][c]);
        }
#pragma unroll
        for (int q = 0; q < NC; q++)
#pragma unroll
            for (int c = 0; c < CC; c++)
                if (q * CC + c < R) row[q * CC + c] = y[q][c];
    }
}

// lambda_r = sqrt(Ghat_rr); G_n = Ghat / (lambda lambda^T); inner_r =
// <M(:,r), A_n(:,r)> for the normalised A_n. Since M = Ahat V (Ahat = M V^{-1}),
// <M(:,r), Ahat(:,r)> = sum_s Ghat[r][s] V[s][r], so no pass over the rows
// is needed.
__global__ void __launch_bounds__(kThreads) k_finish_mode(const double *__restrict__ V, int R,
                                                          double *__restrict__ lambda, double *__restrict__ G,
                                                          double *__restrict__ inner) {
    __shared__ double lam[MAXR];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < R; r += kThreads / 32) {
        double s = 0.0;
        for (int q = lane; q < R; q += 32) s = fma(G[r * R + q], V[q * R + r], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const double l = sqrt(G[r * R + r]);
            lam[r] = l;
            lambda[r] = l;
            inner[r] = l > 0.0 ? s / l : 0.0;
        }
    }
    __syncthreads();
    if (threadIdx.x < R) {  // reciprocals once per column
        const double l = lam[threadIdx.x];
        lam[threadIdx.x] = l > 0.0 ? 1.0 / l : 0.0;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < R * R; idx += kThreads) {
        const int r = idx / R, s = idx % R;
        G[idx] = G[idx] * lam[r] * lam[s];
    }
}

// Per-block column sums of squares of Ahat (FP32 rows, FP64 partials): the
// column norms lambda of the BF16 path, before its factor is rounded.
__global__ void __launch_bounds__(kThreads) k_colsq_partial(const float *__restrict__ M, int64_t I, int R,
                                                            double *__restrict__ partial) {
    __shared__ float red[kThreads / 32][MAXR];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0 = lane, c1 = lane + 32;
    float s0 = 0.f, s1 = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * (kThreads / 32) + warp; i < I; i += (int64_t)gridDim.x * (kThreads / 32)) {
        const float *row = M + i * R;
        if (c0 < R) s0 = fmaf(row[c0], row[c0], s0);
        if (c1 < R) s1 = fmaf(row[c1], row[c1], s1);
    }
    red[warp][c0] = s0;
    red[warp][c1] = s1;
    __syncthreads();
    for (int c = threadIdx.x; c < R; c += kThreads) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; w++) t += (double)red[w][c];
        partial[(int64_t)blockIdx.x * MAXR + c] = t;
    }
}

__global__ void __launch_bounds__(kThreads) k_colnorm_finish(const double *__restrict__ partial, int nblocks, int R,
                                                             double *__restrict__ lambda) {
    const int warp = threadIdx.x >> 5;
    for (int r = warp; r < R; r += kThreads / 32) {
        const double s = warp_sum_strided(partial + r, nblocks, MAXR);
        if ((threadIdx.x & 31) == 0) lambda[r] = sqrt(s);
    }
}

// inner_r = <M(:,r), A_n(:,r)> from the Gram G_n of the stored (normalised)
// A_n: M = Ahat V and Ahat = A_n diag(lambda), so inner_r = sum_s lambda_s
// G_n[r][s] V[s][r].
__global__ void __launch_bounds__(kThreads) k_inner_from_gram(const double *__restrict__ V, const double *__restrict__ G,
                                                              const double *__restrict__ lambda, int R,
                                                              double *__restrict__ inner) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < R; r += kThreads / 32) {
        double s = 0.0;
        for (int q = lane; q < R; q += 32) s = fma(lambda[q] * G[r * R + q], V[q * R + r], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) inner[r] = s;
    }
}

template <typename C, typename FT> __device__ __forceinline__ FT store_as(C x);
template <> __device__ __forceinline__ double store_as<double, double>(double x) { return x; }
template <> __device__ __forceinline__ float store_as<float, float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 store_as<float, __nv_bfloat16>(float x) {
    return __float2bfloat16_rn(x);
}

template <typename C, typename FT>
__global__ void __launch_bounds__(kThreads) k_scale_store(const C *__restrict__ Mh, int64_t I, int R,
                                                          const double *__restrict__ lambda, FT *__restrict__ A) {
    // thread t owns column t % R of rows t / R, t / R + rows_per_pass, ...:
    // coalesced, and no division or remainder per element (1 / lambda_r is
    // formed once per thread)
    const int rows_per_pass = kThreads / R;  // R <= 64 <= kThreads
    const int t = threadIdx.x;
    if (t >= rows_per_pass * R) return;
    const int r = t % R;
    const double l = lambda[r];
    const C inv = l > 0.0 ? (C)(1.0 / l) : C(1);
    for (int64_t row = (int64_t)blockIdx.x * rows_per_pass + t / R; row < I;
         row += (int64_t)gridDim.x * rows_per_pass) {
        const int64_t idx = row * R + r;
        A[idx] = store_as<C, FT>(Mh[idx] * inv);
    }
}

__global__ void __launch_bounds__(kThreads) k_fit(const double *__restrict__ G_all, int N, int R,
                                                  const double *__restrict__ lambda, const double *__restrict__ inner,
                                                  const double *__restrict__ normX2, double *__restrict__ fit) {
    __shared__ double red[kThreads / 32];
    double s = 0.0;
    const int RR = R * R;
    for (int idx = threadIdx.x; idx < RR; idx += kThreads) {
        double h = 1.0;
        for (int k = 0; k < N; k++) h *= G_all[(int64_t)k * RR + idx];
        s += lambda[idx / R] * h * lambda[idx % R];
    }
    for (int r = threadIdx.x; r < R; r += kThreads) s -= 2.0 * lambda[r] * inner[r];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; w++) t += red[w];
        const double res = normX2[0] + t;
        fit[0] = 1.0 - sqrt(res > 0.0 ? res : 0.0) / sqrt(normX2[0]);
    }
}

// Records the fit of a graph-replayed iteration: trace[counter[0]++] = fit;
// counter[1] = the first iteration (1-based) whose normal equations were not
// positive definite.
__global__ void k_record_fit(const double *__restrict__ fit, const int *__restrict__ status,
                             double *__restrict__ trace, int *__restrict__ counter) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int it = counter[0];
        trace[it] = fit[0];
        if (status[1] && counter[1] == 0) counter[1] = it + 1;
        counter[0] = it + 1;
    }
}

inline int rows_grid(int64_t I, int rows_per_block) {
    int64_t g = (I + rows_per_block - 1) / rows_per_block;
    if (g > GR_BLOCKS) g = GR_BLOCKS;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

size_t dense_scratch_doubles(int R) {
    (void)R;
    return (size_t)GR_BLOCKS * MAXPAIRS + (size_t)GR_BLOCKS * MAXR + 64;
}

int *gram_err_word(double *scratch) {
    return reinterpret_cast<int *>(scratch + (size_t)GR_BLOCKS * MAXPAIRS + (size_t)GR_BLOCKS * MAXR);
}

int *gram_colexp_word(double *scratch) { return reinterpret_cast<int *>(scratch + (size_t)GR_BLOCKS * MAXPAIRS); }

bool gram_uses_tc(const void *A, int R, int dtype) {
    if (dtype == RELATE_F64 || dtype == RELATE_F32) return R >= 1 && R <= MAXR;
    return dtype == RELATE_BF16 && gram_tc_supported(R) && (reinterpret_cast<uintptr_t>(A) % 16) == 0;
}

bool dense_f64_small(int64_t I, int R) { return (double)I * R * (3 * R + 1) / 2 <= 8e6; }

cudaError_t launch_gram(const void *A, int64_t I, int R, int dtype, double *scratch, double *G, int *err,
                        cudaStream_t st, long long wait_cycles, int fault_skip, bool simt_f64) {
    if (R < 1 || R > MAXR) return cudaErrorInvalidValue;
    if (I == 0) return cudaMemsetAsync(G, 0, sizeof(double) * R * R, st);
    if (gram_uses_tc(A, R, dtype) && !(simt_f64 && dtype == RELATE_F64)) {
        // tcgen05 tensor cores: BF16 inputs directly, FP32 inputs as three
        // BF16 terms (gram_f32.cu), FP64 inputs as exact 7-bit slices (gram_oz.cu)
        const int npairs_tc = R * (R + 1) / 2;
        int *e_word = err ? err : gram_err_word(scratch);
        int g;
        cudaError_t e;
        if (dtype == RELATE_F64) {
            g = gram_oz_blocks(I);
            e = launch_gram_oz(A, I, R, dtype, scratch, gram_colexp_word(scratch), e_word, wait_cycles, fault_skip, st);
        } else if (dtype == RELATE_F32) {
            g = gram_f32_blocks(I);
            e = launch_gram_f32((const float *)A, I, R, scratch, e_word, wait_cycles, fault_skip, st);
        } else {
            g = gram_tc_blocks(I);
            e = launch_gram_tc((const __nv_bfloat16 *)A, I, R, scratch, e_word, wait_cycles, fault_skip, st);
        }
        if (e != cudaSuccess) return e;
        k_gram_reduce<<<(npairs_tc + kThreads / 32 - 1) / (kThreads / 32), kThreads, 0, st>>>(scratch, g, R, G);
        return cudaGetLastError();
    }
    const int g = rows_grid(I, GR_ROWS);
    switch (dtype) {
    case RELATE_F64: k_gram_partial<double><<<g, kThreads, 0, st>>>((const double *)A, I, R, scratch); break;
    case RELATE_F32: k_gram_partial<float><<<g, kThreads, 0, st>>>((const float *)A, I, R, scratch); break;
    default: k_gram_partial<__nv_bfloat16><<<g, kThreads, 0, st>>>((const __nv_bfloat16 *)A, I, R, scratch); break;
    }
    const int npairs = R * (R + 1) / 2;
    k_gram_reduce<<<(npairs + kThreads / 32 - 1) / (kThreads / 32), kThreads, 0, st>>>(scratch, g, R, G);
    return cudaGetLastError();
}

cudaError_t launch_normal_eq(const double *G_all, int N, int n, int R, double *Vinv, float *Vinv32, double *Vsave,
                             int f64_apply, int *status, cudaStream_t st) {
    const size_t smem = 2 * sizeof(double) * MAXR * (MAXR + 1);
    cudaError_t e = allow_max_dynamic_smem(k_normal_eq);
    if (e != cudaSuccess) return e;
    k_normal_eq<<<1, kThreads, smem, st>>>(G_all, N, n, R, Vinv, Vinv32, Vsave, f64_apply, status);
    return cudaGetLastError();
}

template <typename C>
static void solve_rows_rp(C *M, int64_t I, int R, const C *Vinv, int g, cudaStream_t st) {
    if (R <= 16)
        k_solve_rows<C, 16><<<g, kThreads, 0, st>>>(M, I, R, Vinv);
    else if (R <= 32)
        k_solve_rows<C, 32><<<g, kThreads, 0, st>>>(M, I, R, Vinv);
    else if (R <= 48)
        k_solve_rows<C, 48><<<g, kThreads, 0, st>>>(M, I, R, Vinv);
    else
        k_solve_rows<C, 64><<<g, kThreads, 0, st>>>(M, I, R, Vinv);
}

cudaError_t launch_solve_rows(void *M, int64_t I, int R, int acc_dtype, const double *Vinv, const float *Vinv32,
                              int *err, cudaStream_t st, long long wait_cycles, int fault_skip, bool simt_f64) {
    if (I == 0) return cudaSuccess;
    int64_t g64 = (I + kThreads - 1) / kThreads;
    const int g = (int)(g64 > 152 * 8 ? 152 * 8 : g64);
    if (acc_dtype == RELATE_F64) {
        if (!simt_f64)  // tensor cores, exact integer slices (solve_oz.cu)
            return launch_solve_oz((double *)M, I, R, Vinv, err, wait_cycles, fault_skip, st);
        solve_rows_rp<double>((double *)M, I, R, Vinv, g, st);  // FP64 pipe
        return cudaGetLastError();
    }
    solve_rows_rp<float>((float *)M, I, R, Vinv32, g, st);
    return cudaGetLastError();
}

__global__ void k_to_float(const double *__restrict__ x, int n, float *__restrict__ y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = (float)x[i];
}

cudaError_t launch_to_float(const double *x, int n, float *y, cudaStream_t st) {
    k_to_float<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(x, n, y);
    return cudaGetLastError();
}

cudaError_t launch_colnorms(const float *M, int64_t I, int R, double *scratch, double *lambda, cudaStream_t st) {
    const int g = rows_grid(I, kThreads / 32);
    double *partial = scratch + (size_t)GR_BLOCKS * MAXPAIRS;
    k_colsq_partial<<<g, kThreads, 0, st>>>(M, I, R, partial);
    k_colnorm_finish<<<1, kThreads, 0, st>>>(partial, g, R, lambda);
    return cudaGetLastError();
}

cudaError_t launch_inner_from_gram(const double *Vsave, const double *G_n, const double *lambda, int R, double *inner,
                                   cudaStream_t st) {
    k_inner_from_gram<<<1, kThreads, 0, st>>>(Vsave, G_n, lambda, R, inner);
    return cudaGetLastError();
}

cudaError_t launch_finish_mode(const double *Vsave, int R, double *lambda, double *G_n, double *inner,
                               cudaStream_t st) {
    k_finish_mode<<<1, kThreads, 0, st>>>(Vsave, R, lambda, G_n, inner);
    return cudaGetLastError();
}

cudaError_t launch_scale_store(const void *Mh, int64_t I, int R, int acc_dtype, const double *lambda, void *A,
                               int factor_dtype, cudaStream_t st) {
    if (I == 0) return cudaSuccess;
    const int64_t rows_per_block = kThreads / R;
    int64_t g64 = (I + rows_per_block - 1) / rows_per_block;
    const int g = (int)(g64 > 152 * 16 ? 152 * 16 : g64);
    if (factor_dtype == RELATE_F64)
        k_scale_store<double, double><<<g, kThreads, 0, st>>>((const double *)Mh, I, R, lambda, (double *)A);
    else if (factor_dtype == RELATE_F32)
        k_scale_store<float, float><<<g, kThreads, 0, st>>>((const float *)Mh, I, R, lambda, (float *)A);
    else
        k_scale_store<float, __nv_bfloat16><<<g, kThreads, 0, st>>>((const float *)Mh, I, R, lambda,
                                                                     (__nv_bfloat16 *)A);
    (void)acc_dtype;
    return cudaGetLastError();
}

cudaError_t launch_record_fit(const double *fit, const int *status, double *trace, int *counter, cudaStream_t st) {
    k_record_fit<<<1, 32, 0, st>>>(fit, status, trace, counter);
    return cudaGetLastError();
}

cudaError_t launch_fit(const double *G_all, int N, int R, const double *lambda, const double *inner,
                       const double *normX2, double *fit, cudaStream_t st) {
    k_fit<<<1, kThreads, 0, st>>>(G_all, N, R, lambda, inner, normX2, fit);
    return cudaGetLastError();
}

}  // namespace relate
