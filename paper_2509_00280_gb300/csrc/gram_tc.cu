// gram_tc.cu -- G = A^T A for BF16 factor matrices on the 5th-generation
// tensor cores (tcgen05.mma, FP32 accumulation in tensor memory).
//
// The Gram step of CP-ALS (the standard ALS cited in Sec. 2.2). As a GEMM it
// is C (R x R) = A^T (R x I) * A (I x R): M = N = R, K = I (the rows). A
// block takes a contiguous range of rows; per 16 rows it issues one
// tcgen05.mma of shape M=128, N=64, K=16 whose A operand is the transposed
// row chunk (rows r >= R are ignored on output) and whose B operand is the
// first 64 rows of the same tile. BF16 x BF16 products are exact in FP32;
// accumulation is FP32 in tensor memory within a block and FP64 across blocks.
//
// Shared-memory operand layout: K-major core matrices without swizzling
// (tcgen05.cuh); a 16-row chunk is 16 M-groups x 2 K-groups of cores.
#include "internal.cuh"
#include "tcgen05.cuh"

namespace relate {
namespace {

constexpr int TC_THREADS = 128;           // 4 warps: one row per thread per stage
constexpr int TC_CHUNK = 16;              // K per tcgen05.mma (16-bit inputs)
constexpr int TC_STAGE_ROWS = 128;        // rows staged per buffer
constexpr int TC_CHUNKS = TC_STAGE_ROWS / TC_CHUNK;
constexpr int TC_CHUNK_BYTES = 4096;      // 128 (M) x 16 (K) x 2 bytes
constexpr int TC_STAGE_BYTES = TC_CHUNKS * TC_CHUNK_BYTES;
constexpr int TC_M = 128, TC_N = 64;
constexpr int TC_TMEM_COLS = 64;          // FP32 accumulator columns (N)
constexpr int TC_BLOCKS = 152;

using namespace tc;

// Per-block upper-triangle partials (FP64) of A^T A, A BF16 I x R (R <= 64,
// R % 8 == 0 so a row is a whole number of 16-byte vectors). Every wait on a
// commit gives up after wait_cycles; fault_skip (a test hook) issues no MMA
// and no commit, so nothing is in flight when those waits run out.
__global__ void __launch_bounds__(TC_THREADS, 1) k_gram_tc(const __nv_bfloat16 *__restrict__ A, int64_t I, int R,
                                                           double *__restrict__ partial, int *__restrict__ err,
                                                           long long wait_cycles, int fault_skip) {
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int gave_up;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int npairs = R * (R + 1) / 2;

    const int64_t per = (I + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = min((int64_t)blockIdx.x * per, I);
    const int64_t r1 = min(r0 + per, I);
    const int nstages = (int)((r1 - r0 + TC_STAGE_ROWS - 1) / TC_STAGE_ROWS);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init1(&bar[0]);
        mbar_init1(&bar[1]);
        gave_up = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = instr_desc_bf16(TC_M, TC_N);
    uint32_t phase[2] = {0, 0};
    int issued[2] = {0, 0};
    const int nvec = R / 8;  // 16-byte vectors per row

    for (int s = 0; s < nstages; s++) {
        const int b = s & 1;
        unsigned char *buf = smem_tc + (size_t)b * TC_STAGE_BYTES;
        if (issued[b]) {  // the MMAs that read this buffer two stages ago are done
            const bool ok = mbar_wait_limit(&bar[b], phase[b], wait_cycles);
            phase[b] ^= 1;
            issued[b] = 0;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) gave_up = 1;
                break;
            }
        }
        // stage rows [row, row + 128): thread t writes row t transposed (k = t)
        const int64_t row = r0 + (int64_t)s * TC_STAGE_ROWS + tid;
        const int c = tid / TC_CHUNK, kk = tid % TC_CHUNK;
        unsigned char *chunk = buf + (size_t)c * TC_CHUNK_BYTES + (kk / 8) * 128 + (kk % 8) * 2;
        for (int v = 0; v < nvec; v++) {
            uint4 q = make_uint4(0, 0, 0, 0);
            if (row < r1) q = __ldg(reinterpret_cast<const uint4 *>(A + row * R) + v);
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int h = 0; h < 4; h++) {
                const int m = v * 8 + 2 * h;  // two bf16 per 32-bit word
                *reinterpret_cast<uint16_t *>(chunk + (m / 8) * 256 + (m % 8) * 16) = (uint16_t)(w[h] & 0xffffu);
                *reinterpret_cast<uint16_t *>(chunk + ((m + 1) / 8) * 256 + ((m + 1) % 8) * 16) =
                    (uint16_t)(w[h] >> 16);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
        __syncthreads();
        if (tid == 0 && !fault_skip) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int cc = 0; cc < TC_CHUNKS; cc++) {
                const uint32_t a_addr = saddr(buf + (size_t)cc * TC_CHUNK_BYTES);
                const uint64_t da = smem_desc(a_addr, 128, 256);
                mma(tmem, da, da, idesc, (s > 0 || cc > 0) ? 1u : 0u);
            }
            commit(&bar[b]);
        }
        issued[b] = 1;
    }
    // all MMAs of this block are complete once both buffers' last commits land
    bool all_ok = true;
    for (int b = 0; b < 2; b++)
        if (issued[b]) all_ok &= mbar_wait_limit(&bar[b], phase[b], wait_cycles);
    if (__syncthreads_or(!all_ok) && tid == 0) gave_up = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (gave_up) {  // a tensor-core commit never arrived: poison this block's partials and report
        if (tid == 0) atomicOr(err, 2);
        for (int p = tid; p < npairs; p += TC_THREADS) partial[(int64_t)blockIdx.x * npairs + p] = __longlong_as_double(0x7ff8000000000000ll);
    } else if (nstages > 0 && warp < 2) {
        // warp w holds D rows 32w..32w+31 (lane = row), columns 0..63
        uint32_t v[32];
        for (int half = 0; half < 2; half++) {
            ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * half), v);
            const int r = 32 * warp + lane;
            if (r < R) {
                for (int j = 0; j < 32; j++) {
                    const int s2 = 32 * half + j;
                    if (s2 >= r && s2 < R) {
                        // index of pair (r, s2) in the upper triangle, row-major
                        const int p = r * R - r * (r - 1) / 2 + (s2 - r);
                        partial[(int64_t)blockIdx.x * npairs + p] = (double)__uint_as_float(v[j]);
                    }
                }
            }
        }
    } else if (nstages == 0) {
        for (int p = tid; p < npairs; p += TC_THREADS) partial[(int64_t)blockIdx.x * npairs + p] = 0.0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
}

}  // namespace

bool gram_tc_supported(int R) { return R >= 8 && R <= 64 && R % 8 == 0; }

int gram_tc_blocks(int64_t I) {
    int64_t g = (I + TC_STAGE_ROWS - 1) / TC_STAGE_ROWS;
    if (g > TC_BLOCKS) g = TC_BLOCKS;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t launch_gram_tc(const __nv_bfloat16 *A, int64_t I, int R, double *partial, int *err, long long wait_cycles,
                           int fault_skip, cudaStream_t st) {
    const int g = gram_tc_blocks(I);
    const size_t smem = 2 * (size_t)TC_STAGE_BYTES;
    cudaError_t e = allow_max_dynamic_smem(k_gram_tc);
    if (e != cudaSuccess) return e;
    k_gram_tc<<<g, TC_THREADS, smem, st>>>(A, I, R, partial, err, wait_cycles > 0 ? wait_cycles : kWaitCycles,
                                           fault_skip);
    return cudaGetLastError();
}

}  // namespace relate
