/*
 * oracle.c -- plain, slow, obviously correct CPU oracle for the ReLATE hot path
 * (linearized sparse encoding, mode-n MTTKRP, CP-ALS).
 *
 * THIS IS TEST INFRASTRUCTURE. Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may call it. The product library never
 * links or calls it, and it shares no code, header or table with the CUDA
 * path.
 *
 * Everything is single-threaded, in the order the paper states the method,
 * in FP64 for floating point and with 128-bit integers for positions.
 *
 * Paper: "ReLATE: Accelerating Tensor Decomposition via Safe and Efficient
 * Learning of Sparse Encodings" (arXiv 2509.00280).
 *   - Sec. 2.1 (Tensor Notations): modes, 0-based indices i_n in [0, I_n).
 *   - Sec. 2.2 (Tensor Decomposition) + Fig. 2: mode-n MTTKRP, per nonzero.
 *   - Sec. 3.3 (Problem Formulation): linearized tensor {<v_i, p_i>} ordered
 *     by p; bit budget l(n) = ceil(log2 I_n), l(p) = sum_n l(n); ALTO default
 *     interleave "starting with the shortest mode" (Fig. 4).
 *   - Sec. 3.3.1-3.3.2 (Environment States, Actions): column j of the
 *     encoding matrix names the mode whose NEXT LOW bit goes to b^j; the bits
 *     of each mode keep their internal order; Eq. 1 counts the interleavings.
 *   - Sec. 3.4 (Alg. 1, masking): an order is valid iff mode n occurs exactly
 *     l(n) times.
 *   - Sec. 4.1.3: partitions of equal work; "minimum fiber reuse".
 * CP-ALS: the paper cites Kolda & Bader for the algorithm and prints no
 * equations; the standard Gauss-Seidel ALS with column 2-norm normalisation
 * is written out below (readings listed in the design notes).
 *
 * Parity pins for each function live in tests/test_oracle_*.py. The ALTO
 * tie-break between modes with equal l(n) beyond the paper's 4x8x2 example
 * and the exact ALS variant of the paper's TD library are "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_ORDER -2
#define ORC_ERR_WIDE -3
#define ORC_ERR_RANGE -4
#define ORC_ERR_NOT_PD -5
#define ORC_ERR_OOM -6

/* ---------------------------------------------------------------------- */
/* Sec. 3.3: l(n) = ceil(log2 I_n), computed by an integer loop:          */
/* the smallest b with 2^b >= I_n (so I_n = 1 gives 0 bits).              */
/* ---------------------------------------------------------------------- */
int orc_bits_for_dim(uint64_t I)
{
    int b = 0;
    while (b < 64 && ((uint64_t)1 << b) < I) b++;
    return b;
}

/* l(p) = sum_n l(n); lbits[n] receives l(n). */
int orc_bit_budget(const uint64_t *dims, int N, int *lbits)
{
    int lp = 0;
    for (int n = 0; n < N; n++) {
        lbits[n] = orc_bits_for_dim(dims[n]);
        lp += lbits[n];
    }
    return lp;
}

/* Sec. 3.4 masking rule: every entry names a mode in [0, N) and mode n
 * occurs exactly l(n) times. Returns 0 if valid. */
int orc_check_order(const uint64_t *dims, int N, const int8_t *order, int len)
{
    int lbits[64];
    if (N < 1 || N > 64) return ORC_ERR_ARG;
    int lp = orc_bit_budget(dims, N, lbits);
    if (len != lp) return ORC_ERR_ORDER;
    int used[64];
    for (int n = 0; n < N; n++) used[n] = 0;
    for (int t = 0; t < len; t++) {
        int n = order[t];
        if (n < 0 || n >= N) return ORC_ERR_ORDER;
        used[n]++;
    }
    for (int n = 0; n < N; n++)
        if (used[n] != lbits[n]) return ORC_ERR_ORDER;
    return ORC_OK;
}

/* ALTO default order (Sec. 3.3, Fig. 4): interleave the modes' bits from b^0
 * upward, starting with the shortest mode; modes with equal l(n) are taken by
 * increasing mode id; a mode whose bits are all placed is skipped.
 * Writes l(p) entries into order and returns l(p). */
int orc_alto_order(const uint64_t *dims, int N, int8_t *order)
{
    int lbits[64], rank[64], left[64];
    int lp = orc_bit_budget(dims, N, lbits);
    /* modes sorted by (l(n), n): simple selection sort */
    for (int n = 0; n < N; n++) rank[n] = n;
    for (int a = 0; a < N; a++)
        for (int b = a + 1; b < N; b++) {
            int ma = rank[a], mb = rank[b];
            if (lbits[mb] < lbits[ma] || (lbits[mb] == lbits[ma] && mb < ma)) {
                rank[a] = mb;
                rank[b] = ma;
            }
        }
    for (int n = 0; n < N; n++) left[n] = lbits[n];
    int t = 0;
    while (t < lp) {
        for (int a = 0; a < N; a++) {
            int n = rank[a];
            if (left[n] > 0) {
                order[t++] = (int8_t)n;
                left[n]--;
            }
        }
    }
    return lp;
}

/* ---------------------------------------------------------------------- */
/* Position p of one nonzero, bit by bit (Sec. 3.3.1-3.3.2): for t = 0..   */
/* l(p)-1, mode a_t contributes its next unused low bit to b^t.            */
/* ---------------------------------------------------------------------- */
static u128 position_of(const uint32_t *coords, int64_t nnz, int64_t e, int N,
                        const int8_t *order, int lp)
{
    int next[64];
    for (int n = 0; n < N; n++) next[n] = 0;
    u128 p = 0;
    for (int t = 0; t < lp; t++) {
        int n = order[t];
        uint32_t i_n = coords[(int64_t)n * nnz + e];
        u128 bit = (u128)((i_n >> next[n]) & 1u);
        p |= bit << t;
        next[n]++;
    }
    return p;
}

/* coords: SoA, coords[n*nnz + e]. Writes p as two 64-bit halves.
 * Returns ORC_ERR_RANGE if some i_n >= I_n, ORC_ERR_WIDE if l(p) > 128. */
int orc_encode(const uint32_t *coords, const uint64_t *dims, int64_t nnz, int N,
               const int8_t *order, uint64_t *key_lo, uint64_t *key_hi)
{
    int lbits[64];
    int lp = orc_bit_budget(dims, N, lbits);
    if (lp > 128) return ORC_ERR_WIDE;
    int rc = orc_check_order(dims, N, order, lp);
    if (rc) return rc;
    for (int n = 0; n < N; n++)
        for (int64_t e = 0; e < nnz; e++)
            if ((uint64_t)coords[(int64_t)n * nnz + e] >= dims[n]) return ORC_ERR_RANGE;
    for (int64_t e = 0; e < nnz; e++) {
        u128 p = position_of(coords, nnz, e, N, order, lp);
        key_lo[e] = (uint64_t)p;
        key_hi[e] = (uint64_t)(p >> 64);
    }
    return ORC_OK;
}

/* Inverse of the position: bit b^t goes back to the next low bit of mode a_t. */
int orc_decode(const uint64_t *key_lo, const uint64_t *key_hi, const uint64_t *dims,
               int64_t nnz, int N, const int8_t *order, uint32_t *coords)
{
    int lbits[64];
    int lp = orc_bit_budget(dims, N, lbits);
    if (lp > 128) return ORC_ERR_WIDE;
    int rc = orc_check_order(dims, N, order, lp);
    if (rc) return rc;
    for (int64_t e = 0; e < nnz; e++) {
        u128 p = ((u128)key_hi[e] << 64) | (u128)key_lo[e];
        int next[64];
        uint32_t c[64];
        for (int n = 0; n < N; n++) {
            next[n] = 0;
            c[n] = 0;
        }
        for (int t = 0; t < lp; t++) {
            int n = order[t];
            uint32_t bit = (uint32_t)((p >> t) & 1u);
            c[n] |= bit << next[n];
            next[n]++;
        }
        for (int n = 0; n < N; n++) coords[(int64_t)n * nnz + e] = c[n];
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* "Ordered collection" (Sec. 3.3): a stable ascending sort by position.   */
/* qsort on (p, original index) is a total order, so its result is the     */
/* stable sort; the library sort is the step, nothing more.                */
/* ---------------------------------------------------------------------- */
static const uint64_t *g_lo, *g_hi; /* single-threaded oracle */

static int cmp_pos(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    if (g_hi[x] != g_hi[y]) return g_hi[x] < g_hi[y] ? -1 : 1;
    if (g_lo[x] != g_lo[y]) return g_lo[x] < g_lo[y] ? -1 : 1;
    return x < y ? -1 : (x > y ? 1 : 0);
}

void orc_sort_perm(const uint64_t *key_lo, const uint64_t *key_hi, int64_t nnz, uint32_t *perm)
{
    for (int64_t e = 0; e < nnz; e++) perm[e] = (uint32_t)e;
    g_lo = key_lo;
    g_hi = key_hi;
    qsort(perm, (size_t)nnz, sizeof(uint32_t), cmp_pos);
    g_lo = g_hi = NULL;
}

/* ---------------------------------------------------------------------- */
/* Equal-work partitions of the ordered stream (Sec. 4.2: workload balance */
/* of linearized formats). Partition q covers [qS, min((q+1)S, nnz)).      */
/* lo/hi[q*N + n] = min/max of i_n over the partition.                     */
/* coords_sorted is SoA in encoded order.                                  */
/* ---------------------------------------------------------------------- */
int64_t orc_partitions(const uint32_t *coords_sorted, int64_t nnz, int N, int64_t S,
                       uint32_t *lo, uint32_t *hi)
{
    if (S <= 0) return ORC_ERR_ARG;
    int64_t P = (nnz + S - 1) / S;
    for (int64_t q = 0; q < P; q++) {
        int64_t b = q * S, e = b + S < nnz ? b + S : nnz;
        for (int n = 0; n < N; n++) {
            uint32_t mn = 0xffffffffu, mx = 0;
            for (int64_t j = b; j < e; j++) {
                uint32_t c = coords_sorted[(int64_t)n * nnz + j];
                if (c < mn) mn = c;
                if (c > mx) mx = c;
            }
            lo[q * N + n] = mn;
            hi[q * N + n] = mx;
        }
    }
    return P;
}

/* Fiber statistics per mode (Sec. 4.1.3 "minimum fiber reuse", Sec. 4.2.1:
 * the synchronisation choice follows the tensor's shape, not the order):
 *   runs[n]     = number of maximal runs of equal i_n in encoded order, a run
 *                 never crossing a partition boundary;
 *   distinct[n] = number of distinct values of i_n;
 *   maxcount[n] = largest number of nonzeros sharing one value of i_n.
 * counts (optional, may be NULL): per-mode histograms, laid out mode after
 * mode, dims[n] entries each. */
int orc_mode_stats(const uint32_t *coords_sorted, const uint64_t *dims, int64_t nnz, int N,
                   int64_t S, uint64_t *runs, uint64_t *distinct, uint64_t *maxcount,
                   uint64_t *counts)
{
    if (S <= 0) return ORC_ERR_ARG;
    uint64_t off = 0;
    for (int n = 0; n < N; n++) {
        const uint32_t *c = coords_sorted + (int64_t)n * nnz;
        uint64_t r = 0;
        for (int64_t j = 0; j < nnz; j++)
            if (j % S == 0 || c[j] != c[j - 1]) r++;
        runs[n] = r;
        uint64_t *h = (uint64_t *)calloc(dims[n] ? dims[n] : 1, sizeof(uint64_t));
        if (!h) return ORC_ERR_OOM;
        for (int64_t j = 0; j < nnz; j++) h[c[j]]++;
        uint64_t d = 0, m = 0;
        for (uint64_t i = 0; i < dims[n]; i++) {
            if (h[i]) d++;
            if (h[i] > m) m = h[i];
        }
        distinct[n] = d;
        maxcount[n] = m;
        if (counts) memcpy(counts + off, h, dims[n] * sizeof(uint64_t));
        off += dims[n];
        free(h);
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Mode-n MTTKRP (Sec. 2.2, Fig. 2): for every nonzero (i_1..i_N, v), the  */
/* rows i_k of C^(k), k != n, are multiplied element-wise, scaled by v and */
/* added into row i_n of the output. Direct COO loop in input order; each  */
/* output entry is a Neumaier-compensated sum (Neumaier 1974), so the      */
/* oracle's own rounding error stays near 2u whatever the row length.      */
/* factors[k] is I_k x R row-major FP64. out is I_n x R, overwritten.      */
/* ---------------------------------------------------------------------- */
int orc_mttkrp(const uint32_t *coords, const double *vals, const uint64_t *dims, int64_t nnz,
               int N, int mode, const double *const *factors, int R, double *out)
{
    if (mode < 0 || mode >= N || R < 1) return ORC_ERR_ARG;
    uint64_t In = dims[mode];
    double *comp = (double *)calloc(In * (uint64_t)R ? In * (uint64_t)R : 1, sizeof(double));
    if (!comp) return ORC_ERR_OOM;
    memset(out, 0, In * (uint64_t)R * sizeof(double));
    for (int64_t e = 0; e < nnz; e++) {
        uint32_t row = coords[(int64_t)mode * nnz + e];
        for (int r = 0; r < R; r++) {
            double t = vals[e];
            for (int k = 0; k < N; k++) {
                if (k == mode) continue;
                uint32_t i_k = coords[(int64_t)k * nnz + e];
                t *= factors[k][(uint64_t)i_k * R + r];
            }
            double *s = &out[(uint64_t)row * R + r];
            double *c = &comp[(uint64_t)row * R + r];
            double u = *s + t;
            if (fabs(*s) >= fabs(t))
                *c += (*s - u) + t;
            else
                *c += (t - u) + *s;
            *s = u;
        }
    }
    for (uint64_t j = 0; j < In * (uint64_t)R; j++) out[j] += comp[j];
    free(comp);
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Dense CP-ALS remainder (standard ALS, Kolda & Bader, cited in Sec. 2.2) */
/* ---------------------------------------------------------------------- */

/* G = A^T A for A (I x R), plain triple loop: G[r][s] = sum_i A[i][r] A[i][s],
 * every entry summed over i in increasing order from 0. The rows are the
 * outer loop so that A is read once, row by row. */
void orc_gram(const double *A, uint64_t I, int R, double *G)
{
    for (int j = 0; j < R * R; j++) G[j] = 0.0;
    for (uint64_t i = 0; i < I; i++) {
        const double *a = A + i * R;
        for (int r = 0; r < R; r++)
            for (int s = 0; s < R; s++) G[r * R + s] += a[r] * a[s];
    }
}

/* Textbook Cholesky V = L L^T (lower L, row-major R x R). Returns 0 on
 * success, ORC_ERR_NOT_PD if a pivot is not positive. */
int orc_cholesky(const double *V, int R, double *L)
{
    for (int j = 0; j < R * R; j++) L[j] = 0.0;
    for (int j = 0; j < R; j++) {
        double d = V[j * R + j];
        for (int k = 0; k < j; k++) d -= L[j * R + k] * L[j * R + k];
        if (!(d > 0.0)) return ORC_ERR_NOT_PD;
        double ljj = sqrt(d);
        L[j * R + j] = ljj;
        for (int i = j + 1; i < R; i++) {
            double s = V[i * R + j];
            for (int k = 0; k < j; k++) s -= L[i * R + k] * L[j * R + k];
            L[i * R + j] = s / ljj;
        }
    }
    return ORC_OK;
}

/* A = M V^{-1} row by row: V is symmetric, so row a of A solves V a^T = m^T;
 * forward substitution with L, then back substitution with L^T. */
void orc_solve_rows(const double *M, uint64_t I, int R, const double *L, double *A)
{
    double y[64];
    for (uint64_t i = 0; i < I; i++) {
        const double *m = M + i * R;
        double *a = A + i * R;
        for (int r = 0; r < R; r++) {
            double s = m[r];
            for (int k = 0; k < r; k++) s -= L[r * R + k] * y[k];
            y[r] = s / L[r * R + r];
        }
        for (int r = R - 1; r >= 0; r--) {
            double s = y[r];
            for (int k = r + 1; k < R; k++) s -= L[k * R + r] * a[k];
            a[r] = s / L[r * R + r];
        }
    }
}

/* Cholesky of V with one ridge retry: V + 1e-12 * tr(V)/R * I. */
int orc_factor_normal(const double *V, int R, double *L, int *ridged)
{
    *ridged = 0;
    if (orc_cholesky(V, R, L) == ORC_OK) return ORC_OK;
    double *W = (double *)malloc(sizeof(double) * R * R);
    if (!W) return ORC_ERR_OOM;
    double tr = 0.0;
    for (int r = 0; r < R; r++) tr += V[r * R + r];
    memcpy(W, V, sizeof(double) * R * R);
    for (int r = 0; r < R; r++) W[r * R + r] += 1e-12 * tr / R;
    *ridged = 1;
    int rc = orc_cholesky(W, R, L);
    free(W);
    return rc;
}

/* Full CP-ALS (Gauss-Seidel over modes 0..N-1):
 *   normX2 = sum v^2; G_k = A_k^T A_k for the initial factors.
 *   per iteration, per mode n:
 *     M   = MTTKRP_n(X, {A_k})
 *     V   = Hadamard product of G_k, k != n
 *     A_n = M V^{-1}            (Cholesky of V, FP64)
 *     lambda_r = ||A_n(:,r)||_2; column r scaled by 1/lambda_r if lambda_r > 0
 *     G_n = A_n^T A_n
 *   after the last mode:
 *     ||X - Xhat||^2 = normX2 + lambda^T (Hadamard_k G_k) lambda
 *                      - 2 sum_r lambda_r <M(:,r), A_{N-1}(:,r)>
 *     fit = 1 - sqrt(max(0, that)) / sqrt(normX2)
 *   stop when it > 1 and |fit - fit_prev| < tol, or after iters.
 * factors: N pointers, I_k x R row-major, in = initial, out = normalised.
 * Returns 0, or ORC_ERR_NOT_PD if Cholesky failed after the ridge retry. */
int orc_cpals(const uint32_t *coords, const double *vals, const uint64_t *dims, int64_t nnz,
              int N, int R, int iters, double tol, double *const *factors, double *lambda,
              double *fit_trace, int *iters_done, int *ridge_count)
{
    if (N < 2 || N > 64 || R < 1 || R > 64 || iters < 0) return ORC_ERR_ARG;
    uint64_t maxI = 0;
    for (int n = 0; n < N; n++)
        if (dims[n] > maxI) maxI = dims[n];
    double *G = (double *)malloc(sizeof(double) * (size_t)N * R * R);
    double *V = (double *)malloc(sizeof(double) * R * R);
    double *L = (double *)malloc(sizeof(double) * R * R);
    double *M = (double *)malloc(sizeof(double) * (maxI ? maxI : 1) * R);
    if (!G || !V || !L || !M) {
        free(G); free(V); free(L); free(M);
        return ORC_ERR_OOM;
    }
    double s = 0.0, c = 0.0; /* Neumaier sum of v^2 */
    for (int64_t e = 0; e < nnz; e++) {
        double t = vals[e] * vals[e], u = s + t;
        if (fabs(s) >= fabs(t)) c += (s - u) + t; else c += (t - u) + s;
        s = u;
    }
    double normX2 = s + c;
    for (int n = 0; n < N; n++) orc_gram(factors[n], dims[n], R, G + (size_t)n * R * R);
    for (int r = 0; r < R; r++) lambda[r] = 1.0;
    int rc = ORC_OK, done = 0, ridges = 0;
    double prev = 0.0;
    for (int it = 1; it <= iters; it++) {
        for (int n = 0; n < N; n++) {
            orc_mttkrp(coords, vals, dims, nnz, N, n, (const double *const *)factors, R, M);
            for (int j = 0; j < R * R; j++) V[j] = 1.0;
            for (int k = 0; k < N; k++) {
                if (k == n) continue;
                for (int j = 0; j < R * R; j++) V[j] *= G[(size_t)k * R * R + j];
            }
            int ridged = 0;
            rc = orc_factor_normal(V, R, L, &ridged);
            ridges += ridged;
            if (rc) goto out;
            orc_solve_rows(M, dims[n], R, L, factors[n]);
            /* column 2-norms (each summed over i in increasing order), then
             * every column with a nonzero norm divided by it */
            for (int r = 0; r < R; r++) lambda[r] = 0.0;
            for (uint64_t i = 0; i < dims[n]; i++)
                for (int r = 0; r < R; r++) lambda[r] += factors[n][i * R + r] * factors[n][i * R + r];
            for (int r = 0; r < R; r++) lambda[r] = sqrt(lambda[r]);
            for (uint64_t i = 0; i < dims[n]; i++)
                for (int r = 0; r < R; r++)
                    if (lambda[r] > 0.0) factors[n][i * R + r] /= lambda[r];
            orc_gram(factors[n], dims[n], R, G + (size_t)n * R * R);
        }
        /* fit, with M = MTTKRP of the last mode and A_{N-1} normalised */
        int last = N - 1;
        double xhat2 = 0.0;
        for (int r = 0; r < R; r++)
            for (int q = 0; q < R; q++) {
                double h = 1.0;
                for (int k = 0; k < N; k++) h *= G[(size_t)k * R * R + r * R + q];
                xhat2 += lambda[r] * h * lambda[q];
            }
        double inner = 0.0;
        for (int r = 0; r < R; r++) {
            double d = 0.0;
            for (uint64_t i = 0; i < dims[last]; i++) d += M[i * R + r] * factors[last][i * R + r];
            inner += lambda[r] * d;
        }
        double res2 = normX2 + xhat2 - 2.0 * inner;
        double fit = 1.0 - sqrt(res2 > 0.0 ? res2 : 0.0) / sqrt(normX2);
        if (fit_trace) fit_trace[it - 1] = fit;
        done = it;
        if (it > 1 && fabs(fit - prev) < tol) break;
        prev = fit;
    }
out:
    if (iters_done) *iters_done = done;
    if (ridge_count) *ridge_count = ridges;
    free(G); free(V); free(L); free(M);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* IEEE round-to-nearest-even FP32 -> BF16 (kept as the FP32 value of the  */
/* rounded BF16), done on the bit pattern. NaN is not expected.            */
/* ---------------------------------------------------------------------- */
void orc_round_bf16(const float *in, int64_t n, float *out)
{
    for (int64_t j = 0; j < n; j++) {
        uint32_t u;
        memcpy(&u, &in[j], 4);
        uint32_t lsb = (u >> 16) & 1u;
        u += 0x7fffu + lsb;
        u &= 0xffff0000u;
        memcpy(&out[j], &u, 4);
    }
}
