/*
 * synthc.c -- multithreaded helper of the seeded input generators.
 *
 * Same definitions as the numpy code in synth/__init__.py (which is the
 * reference it is tested against): SplitMix64 counter-mode draws, uniform
 * labels floor(u * I), Zipf labels by lower-bound search in the FP64
 * cumulative table, optional label permutation, and "first occurrence in
 * counter order" deduplication of coordinate tuples.
 *
 * Holds no arithmetic of the tensor method itself.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const uint64_t GAMMA = 0x9E3779B97F4A7C15ull;

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t draw(uint64_t base, uint64_t idx) { return mix64(base + (idx + 1) * GAMMA); }

uint64_t synth_base(uint64_t seed, uint64_t tag) { return mix64(seed * GAMMA + tag); }

/* labels for counter indices [lo, lo + count): kind 0 = uniform on [0, I),
 * kind 1 = Zipf via cdf (len I); perm (nullable) relabels. */
void synth_labels(uint64_t base, int64_t lo, int64_t count, int kind, uint64_t I, const double *cdf,
                  const uint32_t *perm, uint32_t *out, int nthreads)
{
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t j = 0; j < count; j++) {
        uint64_t x = draw(base, (uint64_t)(lo + j));
        uint64_t k;
        if (kind == 0) {
            double u = (double)(x >> 11) * (1.0 / 9007199254740992.0);
            double f = u * (double)I;
            k = (uint64_t)(int64_t)f;
            if (k > I - 1) k = I - 1;
        } else {
            double u = ((double)(x >> 11) + 1.0) * (1.0 / 9007199254740992.0);
            double t = u * cdf[I - 1];
            uint64_t a = 0, b = I; /* first index with cdf[k] >= t */
            while (a < b) {
                uint64_t m = a + (b - a) / 2;
                if (cdf[m] < t) a = m + 1; else b = m;
            }
            k = a < I ? a : I - 1;
        }
        out[j] = perm ? perm[k] : (uint32_t)k;
    }
}

/* ---------------------------------------------------------------------- */
typedef struct {
    int N, T;
    int split; /* modes [0, split) form the high key, [split, N) the low key */
    uint64_t dims[8];
    uint64_t cap_per; /* slots per thread region, power of two */
    uint64_t *hi, *lo; /* hi == UINT64_MAX marks an empty slot */
} dedup_t;

void *synth_dedup_new(int N, const uint64_t *dims, int split, uint64_t expect, int nthreads)
{
    dedup_t *d = (dedup_t *)calloc(1, sizeof(dedup_t));
    if (!d) return NULL;
    d->N = N;
    d->T = nthreads < 1 ? 1 : nthreads;
    d->split = split;
    for (int n = 0; n < N; n++) d->dims[n] = dims[n];
    uint64_t per = 1024;
    while (per * d->T < 2 * expect + 1024) per <<= 1;
    d->cap_per = per;
    size_t tot = (size_t)per * d->T;
    d->hi = (uint64_t *)malloc(tot * 8);
    d->lo = (uint64_t *)malloc(tot * 8);
    if (!d->hi || !d->lo) {
        free(d->hi); free(d->lo); free(d);
        return NULL;
    }
    memset(d->hi, 0xff, tot * 8);
    return d;
}

void synth_dedup_free(void *p)
{
    dedup_t *d = (dedup_t *)p;
    if (!d) return;
    free(d->hi); free(d->lo); free(d);
}

/* Inserts the M tuples (SoA, coords[n*M + e]) in order; keep[e] = 1 for a
 * first occurrence. Returns the number kept. */
int64_t synth_dedup_insert(void *p, const uint32_t *coords, int64_t M, uint8_t *keep)
{
    dedup_t *d = (dedup_t *)p;
    uint64_t *khi = (uint64_t *)malloc((size_t)M * 8), *klo = (uint64_t *)malloc((size_t)M * 8);
    uint64_t *hh = (uint64_t *)malloc((size_t)M * 8);
    if (!khi || !klo || !hh) {
        free(khi); free(klo); free(hh);
        return -1;
    }
    const int N = d->N, split = d->split, T = d->T;
#pragma omp parallel for schedule(static) num_threads(T)
    for (int64_t e = 0; e < M; e++) {
        uint64_t a = 0, b = 0;
        for (int n = 0; n < split; n++) a = a * d->dims[n] + coords[(int64_t)n * M + e];
        for (int n = split; n < N; n++) b = b * d->dims[n] + coords[(int64_t)n * M + e];
        khi[e] = a;
        klo[e] = b;
        hh[e] = mix64(a * GAMMA ^ mix64(b + 0x632BE59BD9B4E019ull));
    }
    int64_t kept = 0;
#pragma omp parallel num_threads(T) reduction(+ : kept)
    {
        int tid = 0, nth = 1;
#ifdef _OPENMP
        tid = omp_get_thread_num();
        nth = omp_get_num_threads();
#endif
        /* region t holds the keys with hash % T == t; each region is filled
         * by one thread, in counter order, whatever the team size */
        for (int t = tid; t < T; t += nth) {
            uint64_t *H = d->hi + (size_t)t * d->cap_per, *L = d->lo + (size_t)t * d->cap_per;
            const uint64_t mask = d->cap_per - 1;
            for (int64_t e = 0; e < M; e++) {
                uint64_t h = hh[e];
                if ((int)(h % (uint64_t)T) != t) continue;
                uint64_t s = (h / (uint64_t)T) & mask;
                for (uint64_t probe = 0;; probe++) {
                    if (probe > mask) { /* region full: caller falls back */
                        keep[e] = 2;
                        break;
                    }
                    if (H[s] == UINT64_MAX) {
                        H[s] = khi[e];
                        L[s] = klo[e];
                        keep[e] = 1;
                        kept++;
                        break;
                    }
                    if (H[s] == khi[e] && L[s] == klo[e]) {
                        keep[e] = 0;
                        break;
                    }
                    s = (s + 1) & mask;
                }
            }
        }
    }
    free(khi); free(klo); free(hh);
    return kept;
}
