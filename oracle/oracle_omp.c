/*
 * oracle_omp.c -- OpenMP build of the oracle's COO MTTKRP, for the CPU
 * baseline's timing only.
 *
 * THIS IS TEST / BENCHMARK INFRASTRUCTURE. Only the CPU-baseline leg of the
 * benchmark calls it; correctness comparisons always use the single-threaded,
 * compensated orc_mttkrp of oracle.c. The product library never links it.
 *
 * The arithmetic per nonzero is the oracle's (Sec. 2.2, Fig. 2 of the paper):
 * t_r = v * prod_{k != n} A_k(i_k, r) with the factors multiplied in mode
 * order, added into row i_n of the output. The nonzeros are split into
 * contiguous chunks, one per thread (static schedule). A short output mode
 * (I_n x R at most priv_limit entries) is accumulated in one private copy
 * per thread, summed afterwards; a long one with atomic additions. The sums
 * are plain (not compensated), so the result differs from orc_mttkrp by
 * rounding only.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int orc_omp_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int orc_mttkrp_omp(const uint32_t *coords, const double *vals, const uint64_t *dims, int64_t nnz, int N,
                   int mode, const double *const *factors, int R, double *out, int nthreads,
                   int64_t priv_limit)
{
    if (mode < 0 || mode >= N || R < 1 || R > 64 || nthreads < 1) return -1;
    const uint64_t In = dims[mode];
    const uint64_t total = In * (uint64_t)R;
    memset(out, 0, total * sizeof(double));
    const int priv = (int64_t)total <= priv_limit;
    double *copies = NULL;
    if (priv) {
        copies = (double *)calloc((size_t)nthreads * (total ? total : 1), sizeof(double));
        if (!copies) return -6;
    }
#pragma omp parallel num_threads(nthreads)
    {
#ifdef _OPENMP
        const int tid = omp_get_thread_num(), nt = omp_get_num_threads();
#else
        const int tid = 0, nt = 1;
#endif
        const int64_t b = nnz * tid / nt, e = nnz * (tid + 1) / nt;
        double *mine = priv ? copies + (size_t)tid * total : NULL;
        double t[64];
        for (int64_t x = b; x < e; x++) {
            const uint32_t row = coords[(int64_t)mode * nnz + x];
            for (int r = 0; r < R; r++) t[r] = vals[x];
            for (int k = 0; k < N; k++) {
                if (k == mode) continue;
                const double *a = factors[k] + (uint64_t)coords[(int64_t)k * nnz + x] * R;
                for (int r = 0; r < R; r++) t[r] *= a[r];
            }
            if (priv) {
                double *o = mine + (uint64_t)row * R;
                for (int r = 0; r < R; r++) o[r] += t[r];
            } else {
                double *o = out + (uint64_t)row * R;
                for (int r = 0; r < R; r++) {
#pragma omp atomic
                    o[r] += t[r];
                }
            }
        }
        if (priv) {
#pragma omp barrier
            /* each thread sums a contiguous range of entries over the copies */
            const uint64_t lo = total * tid / nt, hi = total * (tid + 1) / nt;
            for (int c = 0; c < nt; c++) {
                const double *src = copies + (size_t)c * total;
                for (uint64_t j = lo; j < hi; j++) out[j] += src[j];
            }
        }
    }
    free(copies);
    return 0;
}
