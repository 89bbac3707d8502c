/*
 * relate.h -- C ABI of the GB300-native sparse MTTKRP / CP-ALS library.
 *
 * The library implements the hot path of "ReLATE: Accelerating Tensor
 * Decomposition via Safe and Efficient Learning of Sparse Encodings"
 * (arXiv 2509.00280): a linearized sparse-tensor encoding (Sec. 3.3), the
 * mode-n MTTKRP over it (Sec. 2.2, Fig. 2), and CP-ALS around it (Sec. 2.2,
 * the decomposition the paper accelerates; the ALS itself is the standard
 * Kolda-Bader algorithm the paper cites).
 *
 * Conventions
 *  - Modes are 0-based: the paper's mode n = 1..N is mode n-1 here.
 *  - Coordinates are uint32, structure-of-arrays: coords[m * nnz + e] is the
 *    mode-m index of nonzero e.
 *  - A factor matrix A_k (the paper's C^(k), F = R columns) is I_k x R,
 *    row-major with row stride R elements, in the handle's factor dtype.
 *  - All pointers named "device" must be CUDA device memory of the current
 *    device; "host" pointers are ordinary host memory.
 *  - Streams are cudaStream_t passed as void*; NULL = the legacy default stream.
 *  - Every call returns RELATE_OK (0) or a negative relate_status_t. The
 *    message of the last failure is available from relate_last_error().
 *  - Calls on one handle must not run concurrently from several host threads.
 */
#ifndef RELATE_H
#define RELATE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RELATE_MAX_MODES 8
#define RELATE_MAX_RANK 64
#define RELATE_MAX_KEY_BITS 128

typedef enum {
    RELATE_OK = 0,
    RELATE_ERR_INVALID_ARG = -1,        /* bad nmodes, dims, R, mode, pointer or dtype */
    RELATE_ERR_BAD_BIT_ORDER = -2,      /* bit order breaks the masking rule (Alg. 1) */
    RELATE_ERR_KEY_TOO_WIDE = -3,       /* l(p) > 128 */
    RELATE_ERR_COORD_OUT_OF_RANGE = -4, /* some i_n >= I_n (found on the device) */
    RELATE_ERR_OOM = -5,                /* device allocation failed */
    RELATE_ERR_NOT_PD = -6,             /* normal-equations matrix not positive definite
                                           even after the ridge retry */
    RELATE_ERR_TIMEOUT = -7,            /* a bounded device wait ran out */
    RELATE_ERR_CUDA = -8,               /* CUDA runtime error; see relate_last_error() */
    RELATE_ERR_UNSUPPORTED = -9         /* valid request the library does not handle */
} relate_status_t;

typedef enum { RELATE_F64 = 0, RELATE_F32 = 1, RELATE_BF16 = 2 } relate_dtype_t;

/* How one mode's MTTKRP resolves writes of many nonzeros to one output row
 * (Sec. 4.1.3: reduction-based vs atomic synchronisation, chosen from the
 * tensor's fiber statistics, Sec. 4.2.1).
 *  ATOMIC     - tiles keep the encoded order; runs of equal i_n are merged in
 *               registers and added to the output with global vector atomics,
 *               except the mode's most populated rows (up to 256), which
 *               accumulate in shared memory and are flushed once per block.
 *  SEGMENTED  - every 2048-nonzero tile is processed in an order sorted by i_n
 *               (a counting sort with bins = rows of the partition's
 *               [lo_n, hi_n] range, or a hash of the row when that range is
 *               wider than 2048; computed once per handle and mode on the
 *               mode's first MTTKRP and kept, 2 bytes per nonzero), so each
 *               run of equal rows is merged in registers and written once per
 *               tile; in a mode whose hottest row has >= 2^15 nonzeros, runs
 *               of its hottest rows (up to 31) go to per-block copies in
 *               handle-owned scratch, added into the output once per block;
 *               a mode with I_n x R x acc bytes <= 16 KB keeps all its rows
 *               in the per-block copy.
 *  PRIVATIZED - sorted tiles as SEGMENTED, and the whole output (I_n x R) is
 *               privatised in shared memory per thread block and flushed once
 *               per block (only when it fits; otherwise SEGMENTED runs).
 *  AUTO       - chosen per mode from the encode-time statistics:
 *               PRIVATIZED if I_n x R x acc bytes <= 32 KB (but SEGMENTED when
 *               I_n x R x acc bytes <= 16 KB, N <= 5 and the rows are whole
 *               16-byte vectors: every row then sits in the per-block copy in
 *               scratch), else SEGMENTED if nnz / distinct(i_n) >= 8 or the
 *               mean run of equal i_n >= 8, else ATOMIC. */
typedef enum {
    RELATE_CONFLICT_AUTO = 0,
    RELATE_CONFLICT_ATOMIC = 1,
    RELATE_CONFLICT_SEGMENTED = 2,
    RELATE_CONFLICT_PRIVATIZED = 3
} relate_conflict_t;

typedef struct relate_handle_s *relate_handle_t; /* opaque; owns all encoding memory */

typedef struct {
    /* Bit order of the linear position p (Sec. 3.3.1-3.3.2): entry t names
     * the mode whose next unused low bit becomes bit b^t of p. Host memory,
     * bit_order_len = l(p) entries, each mode n exactly l(n) times (Alg. 1
     * masking rule). NULL = the ALTO default order (Sec. 3.3, Fig. 4):
     * round robin from b^0 over the modes sorted by (l(n), mode id),
     * skipping exhausted modes. */
    const int8_t *bit_order;
    int bit_order_len;
    /* Nonzeros per equal-work partition of the sorted stream; 0 = 4096. */
    int64_t partition_size;
    /* Per-mode conflict strategy; AUTO = chosen from the statistics. */
    relate_conflict_t conflict[RELATE_MAX_MODES];
    /* dtype of the vals array given to relate_encode: RELATE_F64 or F32.
     * The handle keeps the values in this dtype. */
    relate_dtype_t val_dtype;
    /* Storage dtype of factor matrices given to relate_mttkrp/relate_cpals
     * (F64, F32 or BF16) and accumulation dtype of the MTTKRP output
     * (F64 for F64 factors; F32 for F32 and BF16 factors). */
    relate_dtype_t factor_dtype;
    relate_dtype_t acc_dtype;
    /* 1: coords and vals are device pointers; 0: host pointers (the library
     * copies them to the device inside relate_encode). */
    int coords_on_device;
    /* cudaStream_t used by relate_encode and relate_cpals. */
    void *stream;
    /* Shared-memory budget (bytes) per thread block for privatised
     * accumulators; 0 = the device maximum minus what the kernel needs. */
    int smem_budget;
    /* Nonzero sharding over shard_count processes (e.g. one per GPU):
     * shard_count > 1 keeps only the shard_rank-th contiguous, equal-nnz slice
     * of the sorted stream (relate_shard_range), the equal-work partitioning
     * of linearized formats (Sec. 4.2) across devices. Every process passes the
     * whole tensor; its handle then holds that slice, with its own partitions
     * and statistics. 0 or 1 = the whole tensor. */
    int shard_rank;
    int shard_count;
} relate_params_t;

/* Fills *p with the defaults (ALTO order, S = 4096, AUTO conflicts, F32
 * values, F32 factors, F32 accumulation, host inputs, default stream). */
void relate_params_default(relate_params_t *p);

/* Builds the linearized encoding on the device (Sec. 3.3):
 *   1. l(n) = ceil(log2 I_n) (0 bits for I_n = 1), l(p) = sum l(n);
 *   2. p = the coordinates' bits interleaved in bit_order (device kernel);
 *   3. a stable radix sort of (p, original index) on the device;
 *   4. the sorted stream is stored as one word of l(p) bits per nonzero --
 *      the coordinates as concatenated bit fields, a fixed bit permutation of
 *      p, so decoding is one shift and mask per mode -- plus the values;
 *   5. equal-work partitions of partition_size nonzeros with per-partition
 *      [lo_n, hi_n] bounds, and per-mode fiber statistics.
 * coords: N x nnz uint32 SoA (host or device per params). vals: nnz values in
 * params->val_dtype. dims: host, nmodes entries, each in [1, 2^32].
 * nmodes in [2, 8]; nnz in [0, 2^32 - 1]. Inputs are not retained.
 * Synchronises params->stream once (statistics to the host).
 * Errors: INVALID_ARG, BAD_BIT_ORDER, KEY_TOO_WIDE, COORD_OUT_OF_RANGE, OOM,
 * CUDA. On error *out is NULL and nothing is leaked. */
int relate_encode(const uint32_t *coords, const void *vals, const uint64_t *dims, int nmodes,
                  int64_t nnz, const relate_params_t *params, relate_handle_t *out);

/* Mode-n MTTKRP (Sec. 2.2, Fig. 2): for every nonzero (i_0..i_{N-1}, v),
 *   out(i_n, :) += v * Hadamard_{k != n} A_k(i_k, :).
 * factors: host array of nmodes DEVICE pointers, factors[k] is I_k x R in
 * the handle's factor dtype; factors[mode] is not read (may be NULL).
 * out: DEVICE, I_mode x R in the handle's acc dtype, overwritten (zeroed
 * by this call). R in [1, 64]. Asynchronous on `stream`; never synchronises.
 * Factor rows are read with 16-byte vector loads when every factor pointer
 * is 16-byte aligned and R * sizeof(factor) is a multiple of 16; otherwise
 * a scalar path runs. The first call for a SEGMENTED mode also builds the
 * mode's tile order (one stream-ordered allocation and one kernel on
 * `stream`; skipped while `stream` is being captured, the kernel then sorts
 * each tile itself). An FP64 mode with a Khatri-Rao pair (relate_set_mode_kr)
 * first builds the pair's table in device memory owned by the handle (grown
 * by a stream-ordered allocation outside a capture; inside one, or when the
 * allocation fails, the mode runs unfused). Calls on one handle must be
 * ordered (one stream, or events): the SEGMENTED strategy keeps per-block
 * copies of a skewed mode's hottest rows, and the pairs their table, in
 * memory owned by the handle. Errors: INVALID_ARG, OOM, CUDA (launch
 * failure). */
int relate_mttkrp(relate_handle_t h, int mode, void *const *factors, int R, void *out,
                  void *stream);

/* One MTTKRP of a batch: mode `mode` of the tensor encoded in `h`, with the
 * handle's N factors (host array of DEVICE pointers, factors[mode] not read),
 * rank R and output `out` (DEVICE, I_mode x R in the handle's acc dtype,
 * overwritten). */
typedef struct {
    relate_handle_t h;
    int mode;
    void *const *factors;
    int R;
    void *out;
} relate_mttkrp_item_t;

/* Several MTTKRPs (Sec. 2.2, Fig. 2) in the fewest kernel launches: items
 * whose handles share N (2..5), the stored word width and the factor dtype,
 * and that take the vector path (16-byte aligned factors and output, R x
 * element size a multiple of 16 bytes, partition size a multiple of 4), run
 * as ONE persistent launch per group of up to 24 items: the items' tiles are
 * numbered one after the other and a resident grid walks them, each tile
 * processed as a SEGMENTED tile (rows merged in registers, vector atomics).
 * Other items run one launch each. Each item's tile order is built on first
 * use (before any stream capture, as for relate_mttkrp). Results equal the
 * items' relate_mttkrp results up to the order of floating-point additions.
 * Asynchronous on `stream` (capturable once the tile orders exist). Items
 * must not share an output. The paper has no counterpart: this is the
 * batching of a service's small requests. Errors: INVALID_ARG, OOM, CUDA. */
int relate_mttkrp_batch(const relate_mttkrp_item_t *items, int nitems, void *stream);

typedef struct {
    double fit;          /* final fit 1 - ||X - Xhat|| / ||X|| */
    int iters;           /* iterations run */
    int status;          /* RELATE_OK or the failure status */
    int ridge_retries;   /* Cholesky ridge retries taken */
    double *fit_trace;   /* host, nullable: receives the fit of each iteration
                            (must hold `iters` doubles as passed in) */
} relate_cpals_info_t;

/* CP-ALS (standard ALS, Gauss-Seidel over modes 0..N-1): per mode n,
 *   M = MTTKRP_n; V = Hadamard_{k != n} A_k^T A_k (FP64); Cholesky of V in
 *   FP64 (one ridge retry with 1e-12 tr(V)/R on the diagonal); A_n = M V^{-1};
 *   lambda_r = ||A_n(:, r)||_2; columns scaled by 1/lambda_r (if > 0).
 * After the last mode the fit is
 *   1 - sqrt(max(0, ||X||^2 + lambda^T (Hadamard_k G_k) lambda
 *                 - 2 sum_r lambda_r <M(:,r), A_{N-1}(:,r)>)) / ||X||
 * and the loop stops when it > 1 and |fit - fit_prev| < tol, or after iters.
 * factors: host array of nmodes DEVICE pointers (handle's factor dtype),
 * in = initial factors, out = normalised factors. lambda: R doubles, out,
 * HOST or DEVICE memory (the copy's direction follows from the unified
 * address space); written when the call returns. info: nullable. Runs on the handle's stream; synchronises once per
 * iteration (the fit), or once per call in graph mode with tol <= 0
 * (relate_set_cpals_graph). TIMEOUT: a bounded device wait of the MTTKRP or
 * of the tensor-core Gram (BF16 factors) ran out. Errors: INVALID_ARG,
 * NOT_PD, OOM, TIMEOUT, CUDA. */
int relate_cpals(relate_handle_t h, int R, int iters, double tol, void *const *factors,
                 double *lambda, relate_cpals_info_t *info);

/* Encoding statistics. l(n), l(p) and the bit order are those of Sec. 3.3
 * (bit budget, Sec. 3.3.1-3.3.2 interleaving); runs / distinct / maxcount are
 * the fiber statistics that pick the synchronisation per mode (the "minimum
 * fiber reuse" rule of Sec. 4.1.3): fiber reuse = nnz / distinct. */
/* CP-ALS of n problems in lockstep (the relate_cpals algorithm for each):
 * per iteration and mode s, ONE relate_mttkrp_batch over mode s of every
 * problem with more than s modes, then each problem's dense update; one
 * iteration of all active problems is captured as a CUDA graph and replayed,
 * and re-captured when a problem stops. The host synchronises once per
 * iteration and stops a problem on its own rule (it > 1 and |fit - fit_prev|
 * < tol, or NOT_PD, or TIMEOUT, or `iters`); prev_fit (host, n doubles,
 * nullable; NaN = none) gives the fit before this call, so that a problem
 * resumed in a later call may stop at its first iteration. hs: n distinct
 * handles; R: host, n ranks; factors: host array of n host arrays of the
 * handle's DEVICE factor pointers (in: initial, out: normalised); lambdas:
 * host array of n pointers to R doubles (host or device memory); infos:
 * nullable, n entries (fit_trace, if set, must hold `iters` doubles).
 * stream: a non-default stream; every handle's work runs on it during the
 * call. Results equal each problem's relate_cpals results up to the order of
 * floating-point additions. The paper has no counterpart: this is the
 * batching of a service's small requests. Errors: INVALID_ARG, OOM, CUDA,
 * and NOT_PD / TIMEOUT of the first problem that stopped with one (infos
 * tells which). */
int relate_cpals_batch(relate_handle_t const *hs, int n, const int *R, int iters, double tol,
                       void *const *const *factors, double *const *lambdas, const double *prev_fit,
                       relate_cpals_info_t *infos, void *stream);

typedef struct {
    int nmodes;
    int lp;                 /* l(p) */
    int key_bytes;          /* 4, 8 or 16 bytes per stored word */
    int64_t nnz;
    int64_t partition_size;
    int64_t partitions;
    uint64_t dims[RELATE_MAX_MODES];
    int lbits[RELATE_MAX_MODES];
    int field_offset[RELATE_MAX_MODES]; /* bit offset of mode n's field in a word */
    uint64_t runs[RELATE_MAX_MODES];     /* maximal runs of equal i_n within partitions */
    uint64_t distinct[RELATE_MAX_MODES]; /* distinct values of i_n */
    uint64_t maxcount[RELATE_MAX_MODES]; /* largest fiber-slice population */
    int8_t bit_order[RELATE_MAX_KEY_BITS];
    int64_t nnz_total;      /* nonzeros of the whole tensor (nnz = this shard's) */
    int64_t shard_lo;       /* position of this shard in the sorted stream */
} relate_stats_t;

/* Fills the HOST struct *s from the handle (no device work, no
 * synchronisation). Errors: INVALID_ARG (NULL h or s). */
int relate_get_stats(relate_handle_t h, relate_stats_t *s);

/* Conflict strategy relate_mttkrp uses for `mode` at rank R (the AUTO rule
 * or the explicit choice in params). */
int relate_get_conflict(relate_handle_t h, int mode, int R, relate_conflict_t *out);

/* Overrides the per-mode strategy (AUTO restores the rule). */
int relate_set_conflict(relate_handle_t h, int mode, relate_conflict_t c);

/* Fiber-factoring plan of one mode's SEGMENTED MTTKRP (3 to 5 modes). The
 * per-nonzero MTTKRP of Sec. 2.2 (Fig. 2) is regrouped by distributivity:
 * with the other modes in `level` order p1, ..., p(N-1), each 2048-nonzero
 * tile is sorted by (i_n, i_p1, ..., i_p(depth)) once per handle and mode,
 * and the nonzeros sharing (i_n, i_p1..i_pl) (a level-l fiber, l <= depth)
 * are summed before one multiply by A_pl(i_pl, :): a factor row is gathered
 * and multiplied once per fiber instead of once per nonzero. depth 0 = the
 * flat loop; -1 = AUTO (N - 2 for FP64 factors, whose MTTKRP is bound by the
 * FP64 pipe; 0 for FP32 / BF16 factors, bound by gather latency).
 * level: host, N - 1 entries naming every other
 * mode once; NULL = AUTO (the other modes by decreasing I_k: the largest
 * factors, whose rows miss in L2, are gathered once per outer fiber). col_passes:
 * the records of a tile are walked once per chunk of R / col_passes columns
 * (0 = AUTO = 1; a value that does not split R into whole 16-byte vectors
 * runs as 1). Results differ from the flat loop by rounding only (the same
 * terms, another association). Changing depth or level re-sorts the mode's
 * tiles on its next MTTKRP. Host call. Errors: INVALID_ARG. The paper's
 * counterpart is the tuned encoding (Sec. 3.3); this plan is a GPU-side
 * knob of the same search. */
int relate_set_mode_plan(relate_handle_t h, int mode, int depth, const int8_t *level, int col_passes);

/* The plan relate_mttkrp uses for `mode` at rank R (AUTO resolved; depth 0
 * when the mode is not SEGMENTED or N is outside 3..5). level: host, N - 1
 * entries (nullable); depth, col_passes nullable. Errors: INVALID_ARG. */
int relate_get_mode_plan(relate_handle_t h, int mode, int R, int *depth, int8_t *level, int *col_passes);

/* Khatri-Rao pair of one mode's fiber-factored MTTKRP. The MTTKRP of Sec. 2.2
 * multiplies the unfolded tensor by the Khatri-Rao product of the other
 * factors; with FP64 factors, a plan of depth >= 2 and one unfactored slot,
 * the rows of A_a (.) A_b for a = level[depth - 1] and b = level[depth] (the
 * last factored mode and the innermost one) are formed first, in a table of
 * I_a * I_b rows of R values owned by the handle (device memory, grown on
 * demand, at most 16 GiB and 2^32 rows), and every nonzero then gathers one
 * table row and spends one FMA per element on those two modes: the level-a
 * fiber closes (one multiply each) disappear. relate_mttkrp builds the table
 * on every call (one more kernel, included in its time); relate_cpals builds
 * it once per iteration for the modes that share it. kr: -1 = AUTO (on when
 * I_a * I_b <= nnz / 4), 0 = off, 1 = on where the plan allows it (else the
 * mode runs unfused). Results differ from the unfused kernel by rounding only
 * (A_a (.) A_b is rounded once to FP64). Host call. Errors: INVALID_ARG. No
 * counterpart in the paper, whose kernels are on CPUs. */
int relate_set_mode_kr(relate_handle_t h, int mode, int kr);

/* 1 when `mode`'s MTTKRP at rank R fuses a Khatri-Rao pair (the plan and
 * the AUTO rule resolved), else 0; *rows: the table's rows (nullable).
 * Errors: INVALID_ARG. */
int relate_get_mode_kr(relate_handle_t h, int mode, int R, int *kr, uint64_t *rows);

/* Changes the factor / accumulation dtypes used by later calls
 * (F64/F64, F32/F32 or BF16/F32): the precision forms of the factors and of
 * the MTTKRP accumulation; the encoding itself does not depend on them
 * (storage of a linearized format depends only on the tensor, Sec. 4.2).
 * Errors: INVALID_ARG (NULL h or another pair). */
int relate_set_precision(relate_handle_t h, relate_dtype_t factor_dtype, relate_dtype_t acc_dtype);

/* Changes the stream used by relate_cpals. */
int relate_set_stream(relate_handle_t h, void *stream);

typedef struct {
    uint64_t encode_peak;      /* relate_encode's peak: resident + temporaries */
    uint64_t resident;         /* held by the handle after relate_encode */
    uint64_t cpals_workspace;  /* added to the handle by relate_cpals at rank R */
    uint64_t factors;          /* caller-owned factors: sum_n I_n * R * dtype */
} relate_footprint_t;

/* Device bytes requested from the library's stream-ordered pool by relate_encode
 * and relate_cpals for a tensor of this shape, before the allocator's own
 * rounding (a serving layer admits requests by this); `resident` counts the
 * per-mode tile orders (2 bytes per nonzero and mode) that the first MTTKRP
 * of a SEGMENTED mode adds. A request's peak is
 * max(encode_peak, resident + cpals_workspace) + factors. Host only: makes no
 * CUDA call, needs no GPU. The paper has no counterpart. Errors: INVALID_ARG,
 * KEY_TOO_WIDE. */
int relate_footprint(const uint64_t *dims, int nmodes, int64_t nnz, const relate_params_t *params, int R,
                     relate_footprint_t *out);

/* Returns to the driver the device memory that the library's allocation pool
 * of the current device keeps cached after handles were freed (the pool keeps
 * freed blocks mapped so that the next encode or CP-ALS reuses them). Memory
 * of live handles is untouched. Host call; no synchronisation. The paper has
 * no counterpart. Errors: CUDA. */
int relate_release_cached_memory(void);

/* enable != 0: relate_cpals captures one ALS iteration (every mode's MTTKRP,
 * normal equations, solve, Gram and normalisation, the fit, and the copy of
 * the fit and status words to pinned host memory) as a CUDA graph once per
 * call and replays it each iteration, instead of issuing the ~6N launches of
 * an iteration one by one. Results are those of the plain path (same kernels
 * in the same order). Needs a non-default stream (relate_set_stream); on the
 * legacy default stream the plain path runs. With tol <= 0 (a fixed number
 * of iterations) the iterations are replayed back to back and relate_cpals
 * synchronises once, at the end (each replay records its fit on the device);
 * if an iteration's normal equations are not positive definite, the later
 * iterations still run (on zeroed normal equations) and info reports the
 * failing iteration and its fit. Default: disabled. The paper has no
 * counterpart (launch overhead only). Errors: INVALID_ARG. */
int relate_set_cpals_graph(relate_handle_t h, int enable);

/* The shard of a sorted stream of nnz nonzeros that rank `rank` of `count`
 * holds: [lo, hi) = [floor(nnz * rank / count), floor(nnz * (rank + 1) /
 * count)), contiguous and of equal size within one nonzero (Sec. 4.2:
 * equal-work partitions of the linearized stream). Host only; out-of-range
 * ranks are clamped. */
void relate_shard_range(int64_t nnz, int rank, int count, int64_t *lo, int64_t *hi);

/* Sums `count` elements of `dtype` (F64 or F32) at the DEVICE address `buf`
 * over every shard, in place (an all-reduce), ordered on `stream` (enqueue
 * it on the stream, e.g. ncclAllReduce, or synchronise before reading).
 * Returns 0 on success. */
typedef int (*relate_reduce_fn)(void *buf, int64_t count, relate_dtype_t dtype, void *stream, void *user);

/* Makes relate_cpals a sharded CP-ALS: after each mode's MTTKRP it calls
 * fn(M, I_n * R, acc dtype, stream, user) to sum the shards' partial MTTKRPs
 * (Sec. 2.2: M is a sum over nonzeros), and at its start fn(norm, 1, F64,
 * ...) for ||X||^2; every other step (Grams, normal equations, solve,
 * normalisation, fit) then runs identically on every shard from the same
 * replicated factors. Graph replay is off while a hook is set. fn NULL
 * removes the hook. The hook runs on the calling thread between launches,
 * never inside a stream callback. Errors: INVALID_ARG. relate_cpals reports
 * a nonzero hook return as RELATE_ERR_CUDA. The paper has no counterpart (its
 * MTTKRP is one shared-memory process). */
int relate_set_reduce_hook(relate_handle_t h, relate_reduce_fn fn, void *user);

/* Decodes the linearized tensor {<v_i, p_i>} ordered by p (Sec. 3.3; the
 * inverse of the bit-level encoding of Sec. 3.3.1-3.3.2) to DEVICE buffers,
 * in encoded (sorted) order: coords_out N x nnz uint32 SoA (nullable),
 * vals_out nnz values in the val dtype (nullable), perm_out nnz uint32
 * original indices (nullable), keys_out nnz x 2 uint64 (lo, hi) positions p
 * (nullable). Buffers are caller-owned. Async on stream. Errors: INVALID_ARG
 * (NULL h), CUDA. */
int relate_decode(relate_handle_t h, uint32_t *coords_out, void *vals_out, uint32_t *perm_out,
                  uint64_t *keys_out, void *stream);

/* Copies the bounds of the equal-work partitions of the sorted stream
 * (Sec. 4.2: workload balance of linearized formats; partition q covers
 * nonzeros [qS, min((q+1)S, nnz))) to caller-owned DEVICE buffers lo/hi,
 * partitions x N uint32 each (row q, column n = min / max of i_n over the
 * partition). Async on stream. Errors: INVALID_ARG (NULL argument), CUDA. */
int relate_get_partitions(relate_handle_t h, uint32_t *lo, uint32_t *hi, void *stream);

/* G = A^T A (the Gram step of CP-ALS, the standard ALS cited in Sec. 2.2)
 * for a DEVICE matrix A (I x R, row-major, dtype F64/F32/BF16), written to
 * DEVICE G (R x R FP64). All paths use the tensor cores except BF16 inputs
 * with R % 8 != 0 or an A not 16-byte aligned:
 * - FP64 A (any 8-byte alignment): every entry as exact signed 7-bit integer
 *   slices on its column's scale, all slice products formed as BF16 MMAs
 *   whose FP32 sums stay exact integers, combined in 64-bit integers and
 *   FP64. The only error is the truncation of each entry below 2^-55 of its
 *   column's largest magnitude: |G_rs - exact| <= 2^-53 sqrt(I) |A_r| |A_s|,
 *   |A_r| the column norms. A column holding Inf or NaN gives NaN entries;
 *   subnormal entries count as 0.
 * - FP32 A (any 4-byte alignment): every entry as three BF16 terms, the
 *   products that matter at FP32 precision as BF16 MMAs, FP32 accumulation
 *   over at most 2048 rows, FP64 beyond.
 * - BF16 A with R % 8 == 0 and 16-byte aligned: BF16 MMAs, FP32 accumulation
 *   within blocks of rows, FP64 across blocks; otherwise FP32 accumulation
 *   on the FP32 pipe within blocks of rows.
 * The tensor-core paths synchronise `stream` once to read the kernel's
 * bounded-wait status; otherwise asynchronous on stream. Errors:
 * INVALID_ARG, OOM, TIMEOUT (a tensor-core wait ran out; G is then NaN),
 * CUDA. */
int relate_gram(const void *A, int64_t I, int R, relate_dtype_t dtype, double *G, void *stream);

/* In place M <- M W: the row update A_n = M V^{-1} of CP-ALS (the standard
 * ALS cited in Sec. 2.2) with W = V^{-1}, for a DEVICE matrix M (I x R,
 * row-major, dtype F64 or F32, 1 <= R <= 64) and a DEVICE W (R x R
 * row-major FP64). FP64 runs on the tensor cores: each row of M on its own
 * scale and each column of W on its own, as exact signed 7-bit integer
 * slices, all 64 slice products as BF16 MMAs with exact integer FP32 sums,
 * the dot products formed exactly in 128-bit integers and rounded once to
 * FP64; the only errors are the truncations of the entries (below 2^-55 of
 * their row's / column's largest magnitude): |error| <= 2^-53 R
 * max_r |M_ir| max_r |W_rs| plus the rounding. FP32 M is multiplied by W
 * rounded to FP32 on the FP32 pipe. Synchronises `stream` once. Errors:
 * INVALID_ARG, OOM, TIMEOUT (a tensor-core wait ran out; rows may be left
 * unchanged), CUDA. */
int relate_solve_rows(void *M, int64_t I, int R, relate_dtype_t dtype, const double *W, void *stream);

/* The same Gram step as relate_gram, for callers that cannot allocate device
 * memory when they call it: applications that hand all device memory to
 * their own pool up front, where one more allocation would fail or fragment
 * it, and loops that cannot afford an allocator call that may synchronise the
 * device. The per-block partial sums live in a fixed 5.06 MB array compiled
 * into the library instead of a per-call allocation; every GPU that loads
 * the library holds it until the process exits. The paper has no
 * counterpart; this is a deployment variant of the Gram step of CP-ALS.
 * A, G, R, dtype, stream: as for relate_gram (A DEVICE I x R row-major, G
 * DEVICE R x R FP64). R outside [1, 64] is rejected (RELATE_ERR_INVALID_ARG)
 * because the array holds the partials of at most 64 columns.
 * The first call on a device (and the first in a new CUDA context of it)
 * looks up the array's device address with that device current; make that
 * first call before capturing any stream work. Calls on one device share the
 * array, so calls whose kernels may overlap on the GPU (unordered streams)
 * race and must be serialised by the caller. Each call writes every partial
 * it reads and clears the one status word it needs at zero. Like every CUDA
 * call, it must not be made from a stream callback or a cudaLaunchHostFunc
 * function. Allocates nothing; asynchronous on stream, except that the
 * tensor-core path (BF16, R % 8 == 0, 16-byte aligned A) synchronises it once
 * to read the kernel's bounded-wait status. Errors: INVALID_ARG, TIMEOUT (a
 * tensor-core wait ran out; G is then NaN), UNSUPPORTED (device ordinal >=
 * 64), CUDA. */
int relate_gram_noalloc(const void *A, int64_t I, int R, relate_dtype_t dtype, double *G, void *stream);

/* Synchronises `stream` and reports whether any kernel of this handle gave
 * up a bounded device wait since the last call (RELATE_ERR_TIMEOUT; the flag
 * is then cleared). The MTTKRP kernel waits on its own tile copies with a
 * limit of 4e9 SM clock cycles (about 2 s) instead of spinning forever, then
 * sets the flag and returns. Returns RELATE_OK otherwise.
 * Test hook (environment variable, read at each call): RELATE_FAULT=alloc
 * makes every library allocation fail (RELATE_ERR_OOM); RELATE_FAULT=timeout
 * makes every MTTKRP launch skip its first tile copy with a ~50 ms wait limit,
 * so that its bounded wait runs out and this call reports the timeout;
 * RELATE_FAULT=gram_timeout makes every tensor-core Gram issue no MMA, with
 * the same short limit on its waits. After a real (not injected) timeout the
 * copies or tensor-core operations the kernel gave up on may still complete
 * later: do not reuse the handle or its buffers; tear down the CUDA context. */
int relate_sync_status(relate_handle_t h, void *stream);

/* Frees the handle and all its device memory, the encoding built by
 * relate_encode (Sec. 3.3) and the CP-ALS workspace (synchronises its stream
 * and its second stream, not the device). The memory returns to the
 * library's pool (see relate_release_cached_memory). Work that uses the
 * handle on other streams must be complete. NULL is ignored. */
void relate_free(relate_handle_t h);

/* Static description of a status code (the codes above; the paper defines
 * none). Never NULL; the string must not be freed. */
const char *relate_status_string(int status);

/* Message of the last error on this host thread ("" if none). */
const char *relate_last_error(void);

/* Library version string. */
const char *relate_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RELATE_H */
