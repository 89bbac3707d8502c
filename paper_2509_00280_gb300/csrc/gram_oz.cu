// gram_oz.cu -- G = A^T A for FP64 matrices on the tcgen05 tensor cores,
// by splitting every entry into exact 7-bit integer slices (the
// splitting scheme of Ozaki et al. for accurate products on low-precision
// multipliers).
//
// The Gram step of CP-ALS (the standard ALS cited in Sec. 2.2). Column r of
// A is put on one fixed-point scale from its largest exponent field E_r
// (k_colexp): a = q * 2^(E_r - 1077) with |q| < 2^55, q truncated toward
// zero. |q| is cut into S slices of 7 bits, u_0 (most significant) ..
// u_{S-1} (S = 8: q exactly), each carrying the sign of a, each exactly a
// BF16 value, so
//   q_r q_s = sum_{i, j < S} u_i u_j 2^(7 (14 - i - j)).
// Every pair (i, j) is a BF16 x BF16 MMA over the rows (K) accumulating in
// FP32 in tensor memory, pairs of one group g = i + j in one accumulator.
// A block of tensor memory holds at most 4 terms per group and row, each of
// magnitude <= 127^2, so over a 128-row period every partial sum is an integer
// below 2^23 and the tensor cores add exactly. After each period the groups
// are read back (tcgen05.ld), combined exactly in 64-bit integer words and
// added to the block's 64-bit integer words of each pair in shared memory
// (atomics, exact); the words are turned into FP64 and scaled by
// 2^(E_r + E_s) once at the end. The products are exact; the truncation of
// q (below 2^-55 of the column's largest magnitude per entry) bounds the
// error of G_rs by 2^-53 sqrt(I) ||A(:, r)|| ||A(:, s)||, within FP64
// summation's own typical error.
//
// Operands: two 64-row stages. Slice k of a 16-row chunk is a 2 KB block of
// the K-major layout (tcgen05.cuh) holding the 64 columns as M rows, the 8
// slices of a chunk in order, so that slices (a, a + 1) form one M = 128 A
// operand and slices b.. one N = 128 or 256 B operand. Entries with no data
// (columns >= R, rows past the end) are zero.
#include <cmath>

#include "internal.cuh"
#include "slices.cuh"
#include "tcgen05.cuh"

namespace relate {
namespace {

constexpr int OZ_THREADS = 256;
constexpr int OZ_STAGE_ROWS = 64;
constexpr int OZ_CHUNKS = OZ_STAGE_ROWS / 16;
constexpr int OZ_BLK = 2048;          // one slice of one 16-row chunk: 64 (M) x 16 (K) x 2 bytes
constexpr int OZ_BLOCKS = 152;
constexpr int OZ_ITEMS = OZ_STAGE_ROWS / 2 * 64 / OZ_THREADS;  // (column, row pair) items per thread per stage

// two stages of slices, a zero A operand (128 x 16 BF16), four 64-bit words per pair (r <= s)
template <int S> constexpr size_t oz_smem_bytes() { return 2 * (size_t)S * OZ_CHUNKS * OZ_BLK + 4096 + 4 * 2080 * 8; }

// Largest exponent field per column of a row-major I x R matrix (R <= 64),
// atomicMax into colexp[0..R) (zeroed by the launcher). A warp walks rows,
// lane l holding columns l and l + 32; 8 rows per step are in flight.
__global__ void __launch_bounds__(256) k_colexp(const double *__restrict__ A, int64_t I, int R, int *__restrict__ colexp) {
    __shared__ int smax[64];
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 64) smax[threadIdx.x] = 0;
    __syncthreads();
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int m0 = 0, m1 = 0;
    const bool c0 = lane < R, c1 = lane + 32 < R;
    for (int64_t i = w0; i < I; i += 8 * nw) {
        double x0[8], x1[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int64_t row = i + u * nw;
            x0[u] = (row < I && c0) ? A[row * R + lane] : 0.0;
            x1[u] = (row < I && c1) ? A[row * R + lane + 32] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; u++) {
            m0 = max(m0, sl::expo_of(x0[u]));
            m1 = max(m1, sl::expo_of(x1[u]));
        }
    }
    atomicMax(&smax[lane], m0);
    atomicMax(&smax[lane + 32], m1);
    __syncthreads();
    if (threadIdx.x < R && smax[threadIdx.x] > 0) atomicMax(colexp + threadIdx.x, smax[threadIdx.x]);
}

// Drain of the tensor-memory blocks [C0, C1) of one pass: block c holds
// group g = c + OFF (OFF = 0 in the lower 64 lanes, 1 in the upper 64).
// Each FP32 value is an exact integer; the groups are combined exactly in
// 64-bit words of four groups (word k = sum_{g = 4k..4k+3} acc_g
// 2^(7 (4k + 3 - g)), so q_r q_s = sum_k word_k 2^(7 (11 - 4k))) and added
// with 64-bit shared-memory atomics to the block's words of the pair (r, s),
// pair index p = r R - r (r - 1) / 2 + s - r, for r <= s < R (both halves of
// the lanes add to the same pairs). No FP64 arithmetic until the end.
template <int OFF, int C0, int C1>
__device__ __forceinline__ void oz_drain(uint32_t tbase, unsigned long long *words, int npairs, int r, int s0, int R) {
#pragma unroll
    for (int qc = 0; qc < 4; qc++) {  // 8 columns at a time, all blocks of the pass in flight
        uint32_t va[32], vb[32];
#pragma unroll
        for (int c = C0; c < C1; c++)
            tc::ld8_nowait(tbase + 64u * (uint32_t)(c - C0) + 8u * (uint32_t)qc, (c - C0 < 4 ? va : vb) + 8 * ((c - C0) & 3));
        tc::wait_ld32(va);
        tc::wait_ld32(vb);
        long long w[4][8];
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
            for (int j = 0; j < 8; j++) w[k][j] = 0;
#pragma unroll
        for (int c = C0; c < C1; c++) {
            const int g = c + OFF, k = g >> 2, sh = 7 * (4 * k + 3 - g);
            const uint32_t *v = (c - C0 < 4 ? va : vb) + 8 * ((c - C0) & 3);
#pragma unroll
            for (int j = 0; j < 8; j++) w[k][j] += (long long)__float2int_rn(__uint_as_float(v[j])) << sh;
        }
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int s = s0 + 8 * qc + j;
            if (s < r || s >= R) continue;
            const int p = r * R - r * (r - 1) / 2 + (s - r);
#pragma unroll
            for (int k = 0; k < 4; k++)
                if ((C0 + OFF) >> 2 <= k && k <= (C1 - 1 + OFF) >> 2)
                    atomicAdd(words + (size_t)k * npairs + p, (unsigned long long)w[k][j]);
        }
    }
}

// Per-block FP64 upper-triangle partials of A^T A (A: I x R row-major, R <=
// 64), given colexp. One MMA stacks slices a (D lanes 0..63) and a + 1 (lanes
// 64..127), a even, as the A operand and slices b.. (64 columns each) as the
// B operand: it forms the pairs (a, b + n) and (a + 1, b + n) into tensor-
// memory block a + b + n, whose lower lanes hold group a + b + n and upper
// lanes group a + b + n + 1. The 64 pairs take 10 MMAs per 16-row chunk over
// 14 blocks, 8 at a time in 512 columns, so a second pass re-reads the staged
// slices; each pass's blocks are zeroed first by MMAs of a zero operand. The
// products q_r q_s are exact and the only error is the truncation of q.
// Per 128-row period: stage two 64-row buffers, MMAs, drain, per pass.
// Waits on tensor-core commits give up after wait_cycles (then: err |= 2,
// NaN partials); fault_skip (a test hook) issues no MMA and no commit, so
// nothing is in flight when those waits run out.
template <typename T, int S>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_gram_oz(const T *__restrict__ A, int64_t I, int R, const int *__restrict__ colexp, double *__restrict__ partial,
              int *__restrict__ err, long long wait_cycles, int fault_skip) {
    static_assert(S == 8, "8 slices: q exactly");
    constexpr int NCB = 14;                          // tensor-memory blocks of one period (groups 0..14)
    constexpr int STAGE_BYTES = S * OZ_CHUNKS * OZ_BLK;
    constexpr uint32_t TMEM_COLS = 512;              // 8 blocks of 64 FP32 columns
    extern __shared__ __align__(1024) unsigned char smem_oz[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int gave_up;
    __shared__ int sE[64];
    unsigned char *zero_a = smem_oz + 2 * (size_t)STAGE_BYTES;  // a zero A operand
    unsigned long long *words = reinterpret_cast<unsigned long long *>(zero_a + 4096);  // [k][pair]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int npairs = R * (R + 1) / 2;

    const int64_t per = (I + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = min((int64_t)blockIdx.x * per, I);
    const int64_t r1 = min(r0 + per, I);
    const int nper = (int)((r1 - r0 + 2 * OZ_STAGE_ROWS - 1) / (2 * OZ_STAGE_ROWS));

    if (tid < 64) sE[tid] = tid < R ? colexp[tid] : 0;
    for (int i = tid; i < 4 * npairs; i += OZ_THREADS) words[i] = 0ull;
    if (warp == 0) tc::alloc(&tmem_base, TMEM_COLS);
    if (tid == 0) {
        tc::mbar_init1(&bar);
        gave_up = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc256 = tc::instr_desc_bf16(128, 256), idesc128 = tc::instr_desc_bf16(128, 128);
    for (int i = tid; i < 1024; i += OZ_THREADS) reinterpret_cast<uint32_t *>(zero_a)[i] = 0u;

    // drain roles: warp (lane quarter q, column half h) reads D lanes 32q..
    // (row r = 32 (q & 1) + lane of the lower (q < 2) or upper group set),
    // columns 32h..; the blocks with every row above every column are skipped
    const int q = warp & 3, hcol = warp >> 2;
    const bool upper = q >= 2;
    const bool drainer = ((q & 1) == 0 && (hcol == 0 || R > 32)) || ((q & 1) == 1 && hcol == 1 && R > 32);
    const int rloc = 32 * (q & 1) + lane;
    const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * hcol);

    // this thread's staging items: column m, row pairs kp of a stage
    const int m = ((tid >> 2) & 7) | (warp << 3);
    const bool mcol = m < R;
    const int Em = mcol ? sE[m] : 0;
    // byte offset of slice k of chunk c in a stage: slices i and i + H of a chunk are adjacent
    // byte offset of slice k of chunk c in a stage: the 8 slices of a chunk in order, 2 KB each
    auto blk = [](int k, int c) -> uint32_t { return (uint32_t)((c * S + k) * OZ_BLK); };

    uint32_t phase = 0;
    bool stop = false;  // a wait gave up (the same in every thread)
    for (int p = 0; p < nper && !stop; p++) {
        // ---- stage 128 rows: every entry's S slices, two rows per 32-bit store
#pragma unroll 1
        for (int b = 0; b < 2; b++) {
            unsigned char *buf = smem_oz + (size_t)b * STAGE_BYTES;
            const int64_t srow = r0 + (int64_t)p * 2 * OZ_STAGE_ROWS + (int64_t)b * OZ_STAGE_ROWS;
#pragma unroll
            for (int it0 = 0; it0 < OZ_ITEMS; it0 += OZ_ITEMS / 2) {  // two rounds of loads in flight
                T x[OZ_ITEMS / 2][2];
#pragma unroll
                for (int iu = 0; iu < OZ_ITEMS / 2; iu++) {
                    const int kp = (tid & 3) | ((it0 + iu) << 2);
                    const int64_t row = srow + 2 * kp;
                    x[iu][0] = (mcol && row < r1) ? A[row * R + m] : T(0);
                    x[iu][1] = (mcol && row + 1 < r1) ? A[(row + 1) * R + m] : T(0);
                }
#pragma unroll
                for (int iu = 0; iu < OZ_ITEMS / 2; iu++) {
                    const int kp = (tid & 3) | ((it0 + iu) << 2);
                    const int c = kp >> 3;
                    const uint32_t off =
                        (uint32_t)((m >> 3) * 256 + ((kp & 7) >> 2) * 128 + (m & 7) * 16 + (kp & 3) * 4);
                    uint32_t u0[8], u1[8];
                    sl::slices8((double)x[iu][0], Em, u0);
                    sl::slices8((double)x[iu][1], Em, u1);
#pragma unroll
                    for (int k = 0; k < S; k++)
                        *reinterpret_cast<uint32_t *>(buf + blk(k, c) + off) = u0[k] | (u1[k] << 16);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
        __syncthreads();
#pragma unroll 1
        for (int pass = 0; pass < 2; pass++) {
            if (tid == 0) {
                if (!fault_skip) {
                    tc::fence_after();
                    // this pass's blocks start at zero: MMAs of the zero A operand (pass 0: blocks
                    // 0..7, 512 columns; pass 1: blocks 8..13, 384 columns); every MMA below adds
                    const uint64_t dz = tc::smem_desc(tc::saddr(zero_a), 128, 256);
                    const uint64_t dany = tc::smem_desc(tc::saddr(smem_oz), 128, 256);
                    tc::mma(tmem, dz, dany, idesc256, 0u);
                    tc::mma(tmem + 256u, dz, dany, pass == 0 ? idesc256 : idesc128, 0u);
#pragma unroll 1
                    for (int b = 0; b < 2; b++)
#pragma unroll 1
                        for (int c = 0; c < OZ_CHUNKS; c++) {
                            // descriptors differ only in the start address field (address >> 4)
                            const uint64_t d0 = tc::smem_desc(tc::saddr(smem_oz + (size_t)b * STAGE_BYTES), 128, 256);
                            // A = slices (a, a + 1) stacked (D lanes 0..63 / 64..127), B = slices
                            // b.. (N = 64 per slice): pairs (a, b + n) and (a + 1, b + n) into block
                            // a + b + n, whose lower lanes hold group a + b + n, upper lanes the next
                            auto mma = [&](int a, int bs, int nsl) {
                                const int blk0 = a + bs - (pass == 0 ? 0 : 8);
                                tc::mma(tmem + 64u * (uint32_t)blk0, d0 + (uint64_t)(blk(a, c) >> 4),
                                        d0 + (uint64_t)(blk(bs, c) >> 4), nsl == 4 ? idesc256 : idesc128, 1u);
                            };
                            if (pass == 0) {  // blocks 0..7
                                mma(0, 0, 4);
                                mma(2, 0, 4);
                                mma(4, 0, 4);
                                mma(0, 4, 4);
                                mma(6, 0, 2);
                                mma(2, 4, 2);
                            } else {          // blocks 8..13
                                mma(4, 4, 4);
                                mma(6, 4, 4);
                                mma(6, 2, 2);
                                mma(2, 6, 2);
                            }
                        }
                    tc::commit(&bar);
                }
            }
            // ---- drain this pass: its MMAs are complete once the commit lands
            const bool ok = tc::mbar_wait_limit(&bar, phase, wait_cycles);
            phase ^= 1;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) gave_up = 1;
                stop = true;
                break;
            }
            tc::fence_after();
            if (drainer) {
                if (pass == 0) {
                    if (upper) oz_drain<1, 0, 8>(tbase, words, npairs, rloc, 32 * hcol, R);
                    else oz_drain<0, 0, 8>(tbase, words, npairs, rloc, 32 * hcol, R);
                } else if constexpr (NCB > 8) {
                    if (upper) oz_drain<1, 8, NCB>(tbase, words, npairs, rloc, 32 * hcol, R);
                    else oz_drain<0, 8, NCB>(tbase, words, npairs, rloc, 32 * hcol, R);
                }
            }
            tc::fence_before();
            __syncthreads();  // the next MMAs overwrite the accumulators
        }
    }
    __syncthreads();
    tc::fence_after();
    if (gave_up) {  // a tensor-core commit never arrived: poison this block's partials and report
        if (tid == 0) atomicOr(err, 2);
        for (int pp = tid; pp < npairs; pp += OZ_THREADS)
            partial[(int64_t)blockIdx.x * npairs + pp] = __longlong_as_double(0x7ff8000000000000ll);
    } else {
        // G_rs = 2^(E_r + E_s - 2154) q_r q_s, a = q 2^(E - 1077)
        for (int pp = tid; pp < npairs; pp += OZ_THREADS) {
            int r = 0, left = pp;
            while (left >= R - r) {
                left -= R - r;
                r++;
            }
            const int s2 = r + left;
            const int Er = sE[r], Es = sE[s2];
            double g;
            if (Er >= 0x7ff || Es >= 0x7ff) g = __longlong_as_double(0x7ff8000000000000ll);
            else if (Er == 0 || Es == 0) g = 0.0;
            else {
                // q_r q_s = sum_k word_k 2^(7 (11 - 4k)): the words exactly in FP64 (|word| < 2^63
                // rounds once each), summed from the smallest weight up
                double acc = 0.0;
#pragma unroll
                for (int k = 3; k >= 0; k--)
                    acc += ldexp((double)(long long)words[(size_t)k * npairs + pp], 7 * (11 - 4 * k));
                g = ldexp(acc, Er + Es - 2154);
            }
            partial[(int64_t)blockIdx.x * npairs + pp] = g;
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::dealloc(tmem, TMEM_COLS);
}

template <typename T, int S>
cudaError_t launch_oz(const T *A, int64_t I, int R, double *partial, int *colexp, int *err, long long wait_cycles,
                      int fault_skip, int g, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(colexp, 0, 64 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    int64_t gw = (I + 8 * 8 - 1) / (8 * 8);  // 8 warps per block, 8 rows in flight per warp
    const int g1 = (int)(gw > 152 * 4 ? 152 * 4 : gw < 1 ? 1 : gw);
    k_colexp<<<g1, 256, 0, st>>>(A, I, R, colexp);
    auto kern = k_gram_oz<T, S>;
    if ((e = allow_max_dynamic_smem(kern)) != cudaSuccess) return e;
    kern<<<g, OZ_THREADS, oz_smem_bytes<S>(), st>>>(A, I, R, colexp, partial, err,
                                                    wait_cycles > 0 ? wait_cycles : kWaitCycles, fault_skip);
    return cudaGetLastError();
}

}  // namespace

int gram_oz_blocks(int64_t I) {
    int64_t g = (I + OZ_STAGE_ROWS - 1) / OZ_STAGE_ROWS;
    if (g > OZ_BLOCKS) g = OZ_BLOCKS;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t launch_gram_oz(const void *A, int64_t I, int R, int dtype, double *partial, int *colexp, int *err,
                           long long wait_cycles, int fault_skip, cudaStream_t st) {
    if (R < 1 || R > 64) return cudaErrorInvalidValue;
    const int g = gram_oz_blocks(I);
    if (dtype != RELATE_F64) return cudaErrorInvalidValue;
    return launch_oz<double, 8>((const double *)A, I, R, partial, colexp, err, wait_cycles, fault_skip, g, st);
}

}  // namespace relate
