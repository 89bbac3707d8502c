// internal.cuh -- declarations shared by the library's translation units.
// Nothing here is part of the public ABI (include/relate.h is).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "relate.h"

#define RELATE_VERSION_STRING "relate-gb300 0.1.0 (sm_103a)"

namespace relate {

constexpr int kMaxModes = RELATE_MAX_MODES;
constexpr int kMaxRuns = RELATE_MAX_KEY_BITS;
constexpr int kThreads = 256;  // threads per block of the streaming kernels

// The most dynamic shared memory `kern` can launch with on the current
// device: the opt-in limit per block minus the kernel's static shared memory
// (cached per kernel and device); 0 on error.
int max_dynamic_smem(const void *kern);

// Lets `kern` launch with up to max_dynamic_smem(kern). The limit is a
// per-function attribute shared by all host threads, so it is always set to
// that one value, never to a launch's own size: another thread's launch, or a
// node of a graph it is still capturing, is never left above a limit lowered
// in between.
template <typename K>
cudaError_t allow_max_dynamic_smem(K kern) {
    const int lim = max_dynamic_smem(reinterpret_cast<const void *>(kern));
    if (lim <= 0) return cudaErrorInvalidDeviceFunction;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

// A maximal run of bits that one mode contributes to the position p:
// bits [src, src+len) of i_mode land in bits [dst, dst+len) of p
// (Sec. 3.3.1-3.3.2: mode a_t gives its next low bit to b^t, so each mode's
// bits keep their order and consecutive b^t of one mode form a run).
struct BitRuns {
    int nruns;
    int mode_begin[kMaxModes + 1];  // runs grouped by mode: [mode_begin[m], mode_begin[m+1])
    uint8_t src[kMaxRuns];
    uint8_t dst[kMaxRuns];
    uint8_t len[kMaxRuns];
    int field_off[kMaxModes];        // bit offset of mode m's field in the stored word
};

// Field decoding for the stored word (coordinates as concatenated fields).
struct Fields {
    int shift[kMaxModes];
    uint32_t mask[kMaxModes];
};

// 128-bit stored word / key, little-endian 32-bit limbs, 16-byte aligned.
struct __align__(16) W128 {
    uint64_t lo, hi;
};

template <int KW> struct WordT;
template <> struct WordT<1> { using T = uint32_t; };
template <> struct WordT<2> { using T = unsigned long long; };
template <> struct WordT<4> { using T = W128; };

// ---------------------------------------------------------------- encode
// Temporary device memory the radix sort needs for n keys of KW limbs.
size_t radix_sort_temp_bytes(int64_t n);

// Stable LSD radix sort of (key, payload) over bits [0, lp) (K2). The
// result ends in (keys, vals) or (keys_alt, vals_alt); *in_alt tells which.
cudaError_t radix_sort_pairs(int KW, void *keys, uint32_t *vals, void *keys_alt, uint32_t *vals_alt,
                             int64_t n, int lp, void *temp, size_t temp_bytes, cudaStream_t st,
                             bool *in_alt);

// Table-driven bit permutation: table t (256 entries of the position /
// word type) maps the 8 bits of input byte `byte[t]` of input `src[t]` to
// their output bits. For the key build the inputs are the N coordinates,
// for the word packing the single input p.
struct ByteLuts {
    int ntab;
    int src_begin[kMaxModes + 1];  // tables of input m: [src_begin[m], src_begin[m+1])
    uint8_t byte[32];
};
// Builds the tables on the host (entries of 8 bytes for KW <= 2, 16 for KW = 4).
void build_key_luts(int N, const int *lbits, const int8_t *order, int lp, int KW, ByteLuts &d,
                    void *host_tables);
void build_word_luts(int N, const int *field_off, const int8_t *order, int lp, int KW, ByteLuts &d,
                     void *host_tables);
constexpr size_t kLutMaxBytes = 32 * 256 * 16;

cudaError_t launch_build_keys_lut(int KW, const uint32_t *coords, const uint64_t *dims_dev, int64_t n, int N,
                                  const ByteLuts &d, const void *tables, void *keys, uint32_t *idx, uint32_t *err,
                                  cudaStream_t st);
cudaError_t launch_make_words_lut(int KW, const void *keys, int64_t n, const ByteLuts &d, const void *tables,
                                  void *words, cudaStream_t st);

// stored word -> p (for export / tests).
cudaError_t launch_words_to_keys(int KW, const void *words, int64_t n, const BitRuns &runs,
                                 uint64_t *keys_out2, cudaStream_t st);

// stored word -> coordinates SoA.
cudaError_t launch_decode_words(int KW, const void *words, int64_t n, int N, const Fields &f,
                                uint32_t *coords_out, cudaStream_t st);

// vals_out[j] = vals_in[perm[j]] (elem_bytes 4 or 8).
cudaError_t launch_gather(const void *vals_in, const uint32_t *perm, int64_t n, int elem_bytes,
                          void *vals_out, cudaStream_t st);

struct CountPtrs {
    uint32_t *p[kMaxModes];
    uint64_t len[kMaxModes];  // entries of p[m] (= I_m); larger fields are not counted
};

// Per-partition [lo, hi] per mode, per-mode run counts and histograms (K3).
// runs: N uint64 (accumulated), counts: per mode dims[m] uint32 (zeroed by caller).
cudaError_t launch_partition_stats(int KW, const void *words, int64_t n, int N, const Fields &f,
                                   int64_t S, uint32_t *plo, uint32_t *phi,
                                   unsigned long long *runs, const CountPtrs &counts,
                                   cudaStream_t st);

// distinct / maxcount of a histogram (accumulated into out[0], out[1]).
cudaError_t launch_hist_summary(const uint32_t *counts, uint64_t len, unsigned long long *out2,
                                cudaStream_t st);

// sum of v^2 in FP64 (deterministic two-level reduction); partial: >= 1024 doubles
cudaError_t launch_sum_squares(const void *vals, int64_t n, int elem_bytes, double *partial,
                               double *out, cudaStream_t st);

// ---------------------------------------------------------------- mttkrp
struct MttkrpArgs {
    const void *words;
    const void *vals;
    int64_t nnz;
    int64_t S;
    int64_t P;
    int N;
    int mode;
    Fields fields;
    const void *factors[kMaxModes];
    int R;
    void *out;
    uint64_t In;
    int strategy;            // relate_conflict_t (resolved, not AUTO)
    const uint32_t *plo;
    const uint32_t *phi;
    const uint32_t *hot_rows;  // kHotMax rows of the mode, most populated first (0xffffffff = unused)
    int hot_n;                 // hot rows cached in shared memory by this launch
    uint64_t maxcount;         // nonzeros of the mode's most populated row
    void *hot_scratch;         // SEGMENTED: per-block copies of the hot rows (kHotScratchBytes)
    int full_copy;             // SEGMENTED: every row of the mode in the per-block copy (hot_n = I_n, slot = row)
    const uint16_t *tperm;     // SEGMENTED: precomputed tile order of the mode (null: sort in the kernel)
    long long wait_cycles;     // limit of a bounded wait, SM clock cycles (0: kWaitCycles)
    int fault_skip_copy;       // test hook: never issue the first tile copy (its wait times out)
    int vals_f64;              // values stored as FP64 (else FP32)
    int *err;                  // device flag: bit 0 = a bounded wait timed out
    // Fiber factoring of a SEGMENTED mode (0 = off): the record slots 1..N-1
    // hold the other modes in `level` order, the tile order sorts each tile by
    // (i_n, slot 1, ..., slot depth), and the kernel sums each fiber of equal
    // (i_n, slot 1..l) before one multiply by slot l's factor row.
    int depth;
    int8_t level[kMaxModes];   // level[s - 1] = the mode in record slot s (s = 1..N-1)
    int col_passes;            // R split into this many column chunks, one walk of the records each
    // Khatri-Rao pair of a fiber-factored mode with depth >= 2 and one
    // unfactored slot (null = off): the rows of A_a (.) A_b for a = the
    // deepest factored level's mode and b = the innermost mode, row
    // i_a * kr_mul + i_b (kr_mul = I_b). launch_mttkrp then runs the kernel
    // with those two slots as one, a level fewer: each nonzero gathers one
    // product row and the level's fiber closes cost no multiply.
    const void *kr_table;
    uint32_t kr_mul;
    // record slot j of a decoded nonzero: slot 0 = the output mode, slots
    // 1..N-1 = the other modes in increasing order (filled by the launcher)
    int rshift[kMaxModes];
    uint32_t rmask[kMaxModes];
    const void *rfac[kMaxModes];
};

// Limit of a bounded device wait: 4e9 SM cycles, about 2 s at 2 GHz.
constexpr long long kWaitCycles = 4000000000LL;

// Upper bound of hot (most populated) rows per mode kept in shared memory.
constexpr int kHotMax = 256;
// Global scratch of a handle for the SEGMENTED kernel's per-block copies of
// the hot rows: 16 KB per block for up to 1024 blocks.
constexpr size_t kHotBlockBytes = 16384;
constexpr size_t kHotScratchBytes = 1024 * kHotBlockBytes;
// Hot slots a 16-bit tile-order entry can tag (1 + slot in its top 5 bits).
constexpr int kHotTagMax = 31;
// A SEGMENTED mode keeps per-block copies of its hottest rows once its most
// populated row has this many nonzeros (about one global FP32 addition per
// tile holding the row): the random walk of 2^15 roundings, 2^-24 x
// sqrt(2^15) relative, stays well below 1e-5.
constexpr uint64_t kSegHotMinCount = 1u << 15;

// Hot rows of one mode from its histogram: the kHotMax most populated rows
// (ties by row id), most populated first; 0xffffffff pads modes with fewer
// populated rows. temp must hold hot_table_temp_bytes(I).
size_t hot_table_temp_bytes(uint64_t I);
cudaError_t launch_hot_table(const uint32_t *counts, uint64_t I, uint32_t *hot_rows, void *temp, cudaStream_t st);

// Launches K5/K6/K7 for the given dtypes. factor_dtype / val_dtype are
// relate_dtype_t. smem_budget: bytes available for shared accumulators.
// Builds the tile order of a.mode into tperm (nnz 16-bit entries: position in
// the tile sorted by output row | (1 + hot slot) << 11), for the SEGMENTED
// MTTKRP kernel.
cudaError_t launch_tile_order(const MttkrpArgs &a, int KW, int num_sms, uint16_t *tperm, cudaStream_t st);
cudaError_t launch_mttkrp(const MttkrpArgs &a, int KW, int factor_dtype, int val_dtype,
                          int smem_budget, int num_sms, cudaStream_t st);

// The batched MTTKRP (one persistent launch over the tiles of up to 24
// problems sharing N, the key width and the factor dtype, mttkrp_batch.cuh):
// an item needs its tile order, the vector path (16-byte factor rows and
// output) and 16-byte aligned tile starts.
constexpr int kBatchItems = 24;
bool batch_eligible(const MttkrpArgs &a, int factor_dtype);
cudaError_t launch_mttkrp_batch(const MttkrpArgs *items, int n, int KW, int factor_dtype, int num_sms,
                                cudaStream_t st);

// Bytes of shared memory one row of the output accumulator takes.
int mttkrp_acc_bytes(int factor_dtype);
// out(ia * Ib + ib, :) = A(ia, :) * B(ib, :) elementwise, the rows of the
// Khatri-Rao product A (.) B (FP64 or FP32, row-major with R columns, R even;
// 16-byte aligned pointers; Ia * Ib < 2^32).
cudaError_t launch_kr_rows(const void *A, const void *B, uint64_t Ia, uint64_t Ib, int R, int dtype, void *out,
                           cudaStream_t st);

// ---------------------------------------------------------------- dense
// Scratch the dense kernels need (doubles): partial sums for the Gram and
// the row passes.
size_t dense_scratch_doubles(int R);

// G = A^T A, FP64 out (R x R) via per-block partials in `scratch`. FP64,
// FP32 and aligned BF16 inputs with R % 8 == 0 (gram_uses_tc) run on the
// tensor cores, whose bounded waits report a
// timeout as *err |= 2 (err = null: the status word inside `scratch`,
// gram_err_word) and NaN partials; wait_cycles <= 0 = kWaitCycles;
// fault_skip (a test hook) issues no tensor-core work, so the waits run out.
cudaError_t launch_gram(const void *A, int64_t I, int R, int dtype, double *scratch, double *G, int *err,
                        cudaStream_t st, long long wait_cycles = 0, int fault_skip = 0, bool simt_f64 = false);
// FP64 dense steps small enough (I R (3R + 1) / 2 FMA <= 8e6, ~15 us on the
// FP64 pipe) that the FP64-pipe kernels beat the tensor-core ones' fixed
// costs (block setup, slicing of V^{-1}, several launches): CP-ALS passes
// simt_f64 = true for them.
bool dense_f64_small(int64_t I, int R);
bool gram_uses_tc(const void *A, int R, int dtype);
int *gram_err_word(double *scratch);

// Tensor-core Gram partials for BF16 A (R % 8 == 0, R <= 64): one FP64
// upper-triangle partial per block (gram_tc_blocks(I) blocks); err |= 2 and
// NaN partials if a bounded wait on the tensor cores gave up.
bool gram_tc_supported(int R);
int gram_tc_blocks(int64_t I);
cudaError_t launch_gram_tc(const __nv_bfloat16 *A, int64_t I, int R, double *partial, int *err,
                           long long wait_cycles, int fault_skip, cudaStream_t st);

// Tensor-core Gram partials for FP64 A (exact 7-bit slices), R <= 64, any
// 8-byte alignment: k_colexp writes the columns' largest exponent fields to
// colexp[0..64) (zeroed first), then one FP64 upper-triangle partial per
// block (gram_oz_blocks(I) blocks); err |= 2 and NaN partials if a bounded
// wait on the tensor cores gave up.
int gram_oz_blocks(int64_t I);
cudaError_t launch_gram_oz(const void *A, int64_t I, int R, int dtype, double *partial, int *colexp, int *err,
                           long long wait_cycles, int fault_skip, cudaStream_t st);
// The same for FP32 A as three BF16 terms per entry (FP32 accumulation per
// 2048 rows, FP64 beyond), any 4-byte alignment (gram_f32_blocks(I) blocks).
int gram_f32_blocks(int64_t I);
cudaError_t launch_gram_f32(const float *A, int64_t I, int R, double *partial, int *err, long long wait_cycles,
                            int fault_skip, cudaStream_t st);

// V = Hadamard_{k != n} G_k (kept in Vsave); FP64 Cholesky; V^{-1} in FP64
// (f64_apply) or FP32 (Vinv32, always written).
// status[0] |= 1 on ridge retry, status[1] = 1 if not PD after the retry.
cudaError_t launch_normal_eq(const double *G_all, int N, int n, int R, double *Vinv, float *Vinv32,
                             double *Vsave, int f64_apply, int *status, cudaStream_t st);

// In place, M (I x R, acc dtype) <- M V^{-1}. FP64 runs on the tensor cores
// (launch_solve_oz), whose bounded waits report a timeout as *err |= 2;
// FP32 on the FP32 pipe.
cudaError_t launch_solve_rows(void *M, int64_t I, int R, int acc_dtype, const double *Vinv,
                              const float *Vinv32, int *err, cudaStream_t st, long long wait_cycles = 0,
                              int fault_skip = 0, bool simt_f64 = false);
// y[i] = (float)x[i], i < n.
cudaError_t launch_to_float(const double *x, int n, float *y, cudaStream_t st);
// In place M <- M W, FP64, R <= 64, as exact 7-bit integer slices on the
// tensor cores; err |= 2 if a bounded wait gave up (wait_cycles <= 0:
// kWaitCycles); fault_skip (a test hook) issues no tensor-core work.
cudaError_t launch_solve_oz(double *M, int64_t I, int R, const double *W, int *err, long long wait_cycles,
                            int fault_skip, cudaStream_t st);

// lambda and the normalised Gram G_n from the raw Gram of M V^{-1} (in G_n),
// and the fit inner products from that Gram and V.
cudaError_t launch_finish_mode(const double *Vsave, int R, double *lambda, double *G_n, double *inner,
                               cudaStream_t st);

// BF16 path: lambda = column norms of Ahat (FP32), and the fit inner
// products from the Gram of the stored, normalised BF16 factor.
cudaError_t launch_colnorms(const float *M, int64_t I, int R, double *scratch, double *lambda, cudaStream_t st);
cudaError_t launch_inner_from_gram(const double *Vsave, const double *G_n, const double *lambda, int R,
                                   double *inner, cudaStream_t st);

// Row pass 2: A_n = Mhat / lambda, stored in the factor dtype.
cudaError_t launch_scale_store(const void *Mhat, int64_t I, int R, int acc_dtype,
                               const double *lambda, void *A, int factor_dtype, cudaStream_t st);

// fit after the last mode (device scalar out[0]).
// trace[counter[0]++] = *fit; counter[1] = first NOT_PD iteration (1-based).
cudaError_t launch_record_fit(const double *fit, const int *status, double *trace, int *counter, cudaStream_t st);
cudaError_t launch_fit(const double *G_all, int N, int R, const double *lambda, const double *inner,
                       const double *normX2, double *fit, cudaStream_t st);

}  // namespace relate
