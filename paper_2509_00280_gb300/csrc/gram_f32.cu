// gram_f32.cu -- G = A^T A for FP32 matrices on the tcgen05 tensor cores,
// each entry split into three BF16 terms.
//
// The Gram step of CP-ALS (the standard ALS cited in Sec. 2.2). Every FP32
// entry is x = h + m + l + d with h = bf16(x), m = bf16(x - h), l = bf16(x -
// h - m) (the differences are exact in FP32) and |d| <= 2^-27 |x|. The
// products kept are
//   (h_r + m_r) (h_s + m_s + l_s) + l_r h_s,
// which drop only l_r m_s, l_r l_s and the d terms: below 2^-23 |x_r| |x_s|
// per row, FP32's own rounding level. Two tensor-memory accumulators hold
// them: X (M = 128 operand [h ; m] stacked, times h, m and l: lanes 0..63 get
// h_r (h + m + l)_s, lanes 64..127 get m_r (h + m + l)_s) and Y ([l ; -]
// times h, lanes 0..63). BF16 x BF16 products are exact; the tensor cores
// accumulate in FP32 over periods of 128 rows, after which the accumulators
// are read back (tcgen05.ld) and added to compensated FP32 sums (a sum and
// its running error, Neumaier's variant of Kahan summation) in shared memory,
// so the FP32 rounding is that of 128-term sums and the rest is compensated.
//
// Operands: 64-row stages, two buffers; per 16-row chunk four 2 KB blocks
// h, m, l, (zero) of the K-major layout (tcgen05.cuh) with the 64 columns as
// M rows; entries with no data (columns >= R, rows past the end) are zero.
#include "internal.cuh"
#include "tcgen05.cuh"

namespace relate {
namespace {

constexpr int G3_THREADS = 256;
constexpr int G3_STAGE_ROWS = 64;
constexpr int G3_CHUNKS = G3_STAGE_ROWS / 16;
constexpr int G3_BLK = 2048;                    // 64 (M) x 16 (K) x 2 bytes
constexpr int G3_CHUNK_BYTES = 4 * G3_BLK;      // h, m, l, zero
constexpr int G3_STAGE_BYTES = G3_CHUNKS * G3_CHUNK_BYTES;
constexpr int G3_PERIOD = 2;                    // stages (128 rows) per tensor-memory accumulation period
constexpr int G3_BLOCKS = 152;
constexpr int G3_ITEMS = G3_STAGE_ROWS / 2 * 64 / G3_THREADS;
constexpr uint32_t G3_TMEM_COLS = 128;          // X and Y, 64 columns each
constexpr size_t G3_SMEM = 2 * (size_t)G3_STAGE_BYTES + 2 * 64 * 64 * sizeof(float2);

// s + c += v, compensated (Neumaier): c collects the rounding error of every addition.
__device__ __forceinline__ void comp_add(float2 &sc, float v) {
    const float t = sc.x + v;
    sc.y += fabsf(sc.x) >= fabsf(v) ? (sc.x - t) + v : (v - t) + sc.x;
    sc.x = t;
}

__device__ __forceinline__ void split3(float x, uint32_t &h, uint32_t &m, uint32_t &l) {
    const __nv_bfloat16 bh = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(bh);
    const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(bm);
    const __nv_bfloat16 bl = __float2bfloat16_rn(r2);
    h = __bfloat16_as_ushort(bh);
    m = __bfloat16_as_ushort(bm);
    l = __bfloat16_as_ushort(bl);
}

// Per-block FP64 upper-triangle partials of A^T A, A FP32 I x R row-major
// (R <= 64, any 4-byte alignment). Waits on commits give up after
// wait_cycles (then err |= 2 and NaN partials); fault_skip (a test hook)
// issues no MMA and no commit.
__global__ void __launch_bounds__(G3_THREADS, 1)
    k_gram_f32(const float *__restrict__ A, int64_t I, int R, double *__restrict__ partial, int *__restrict__ err,
               long long wait_cycles, int fault_skip) {
    extern __shared__ __align__(1024) unsigned char smem_g3[];
    float2 *acc_s = reinterpret_cast<float2 *>(smem_g3 + 2 * (size_t)G3_STAGE_BYTES);  // [lanes 0-63 | 64-127][s][r]
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int gave_up;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int npairs = R * (R + 1) / 2;

    const int64_t per = (I + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = min((int64_t)blockIdx.x * per, I);
    const int64_t r1 = min(r0 + per, I);
    const int nstages = (int)((r1 - r0 + G3_STAGE_ROWS - 1) / G3_STAGE_ROWS);

    for (int i = tid; i < 2 * 64 * 64; i += G3_THREADS) acc_s[i] = make_float2(0.0f, 0.0f);
    for (int b = 0; b < 2; b++)  // the zero blocks (rows 64..127 of the [l ; 0] operand)
        for (int c = 0; c < G3_CHUNKS; c++)
            for (int i = tid; i < G3_BLK / 4; i += G3_THREADS)
                reinterpret_cast<uint32_t *>(smem_g3 + (size_t)b * G3_STAGE_BYTES + (size_t)c * G3_CHUNK_BYTES +
                                             3 * G3_BLK)[i] = 0u;
    if (warp == 0) tc::alloc(&tmem_base, G3_TMEM_COLS);
    if (tid == 0) {
        tc::mbar_init1(&bar[0]);
        tc::mbar_init1(&bar[1]);
        gave_up = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = tc::instr_desc_bf16(128, R <= 32 ? 32 : 64);

    // drain roles: warp (lane quarter q, column half h); quarters 0-1 read X + Y
    // (lanes 0..63), quarters 2-3 read X (lanes 64..127); row r = 32 (q & 1) + lane
    const int q = warp & 3, hcol = warp >> 2;
    const bool upper = q >= 2;
    const bool drainer = ((q & 1) == 0 && (hcol == 0 || R > 32)) || ((q & 1) == 1 && hcol == 1 && R > 32);
    const int rloc = 32 * (q & 1) + lane;
    float2 *acc = acc_s + (upper ? 64 * 64 : 0) + 64 * (32 * hcol) + rloc;  // column s at acc[64 * (s - 32h)]

    const int m = ((tid >> 2) & 7) | (warp << 3);  // staging column
    const bool mcol = m < R;

    uint32_t phase[2] = {0, 0};
    int issued[2] = {0, 0};
    bool stop = false;
    for (int s = 0; s < nstages && !stop; s++) {
        const int b = s & 1;
        unsigned char *buf = smem_g3 + (size_t)b * G3_STAGE_BYTES;
        if (issued[b]) {  // the MMAs that read this buffer two stages ago are done
            const bool ok = tc::mbar_wait_limit(&bar[b], phase[b], wait_cycles);
            phase[b] ^= 1;
            issued[b] = 0;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) gave_up = 1;
                break;
            }
        }
        const int64_t srow = r0 + (int64_t)s * G3_STAGE_ROWS;
        float x[G3_ITEMS][2];
#pragma unroll
        for (int it = 0; it < G3_ITEMS; it++) {
            const int64_t row = srow + 2 * ((tid & 3) | (it << 2));
            x[it][0] = (mcol && row < r1) ? A[row * R + m] : 0.0f;
            x[it][1] = (mcol && row + 1 < r1) ? A[(row + 1) * R + m] : 0.0f;
        }
#pragma unroll
        for (int it = 0; it < G3_ITEMS; it++) {
            const int kp = (tid & 3) | (it << 2);
            const uint32_t off = (uint32_t)((kp >> 3) * G3_CHUNK_BYTES + (m >> 3) * 256 + ((kp & 7) >> 2) * 128 +
                                            (m & 7) * 16 + (kp & 3) * 4);
            uint32_t h0, m0, l0, h1, m1, l1;
            split3(x[it][0], h0, m0, l0);
            split3(x[it][1], h1, m1, l1);
            *reinterpret_cast<uint32_t *>(buf + off) = h0 | (h1 << 16);
            *reinterpret_cast<uint32_t *>(buf + off + G3_BLK) = m0 | (m1 << 16);
            *reinterpret_cast<uint32_t *>(buf + off + 2 * G3_BLK) = l0 | (l1 << 16);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
        __syncthreads();
        const bool first = (s % G3_PERIOD) == 0;
        if (tid == 0 && !fault_skip) {
            tc::fence_after();
            const uint32_t base = tc::saddr(buf);
#pragma unroll 1
            for (int c = 0; c < G3_CHUNKS; c++) {
                const uint32_t ch = base + (uint32_t)(c * G3_CHUNK_BYTES);
                const uint64_t dh = tc::smem_desc(ch, 128, 256), dm = tc::smem_desc(ch + G3_BLK, 128, 256),
                               dl = tc::smem_desc(ch + 2 * G3_BLK, 128, 256);
                const uint32_t fresh = (first && c == 0) ? 0u : 1u;
                tc::mma(tmem, dh, dh, idesc, fresh);  // [h ; m] x h
                tc::mma(tmem, dh, dm, idesc, 1u);     // [h ; m] x m
                tc::mma(tmem, dh, dl, idesc, 1u);     // [h ; m] x l
                tc::mma(tmem + 64u, dl, dh, idesc, fresh);  // [l ; 0] x h
            }
            tc::commit(&bar[b]);
        }
        issued[b] = 1;
        if ((s % G3_PERIOD) == G3_PERIOD - 1 || s == nstages - 1) {
            const bool ok = tc::mbar_wait_limit(&bar[b], phase[b], wait_cycles);
            phase[b] ^= 1;
            issued[b] = 0;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) gave_up = 1;
                stop = true;
                break;
            }
            tc::fence_after();
            if (drainer) {
                const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * hcol);
                uint32_t vx[32], vy[32];
#pragma unroll
                for (int qc = 0; qc < 4; qc++) tc::ld8_nowait(tb + 8u * (uint32_t)qc, vx + 8 * qc);
                tc::wait_ld32(vx);
                if (!upper) {
#pragma unroll
                    for (int qc = 0; qc < 4; qc++) tc::ld8_nowait(tb + 64u + 8u * (uint32_t)qc, vy + 8 * qc);
                    tc::wait_ld32(vy);
                }
#pragma unroll
                for (int j = 0; j < 32; j++) {
                    const float v = upper ? __uint_as_float(vx[j]) : __uint_as_float(vx[j]) + __uint_as_float(vy[j]);
                    comp_add(acc[64 * j], v);
                }
            }
            tc::fence_before();
            __syncthreads();  // the next period's first MMAs overwrite the accumulators
        }
    }
    // every MMA of this block is complete once the pending commits land
    bool all_ok = true;
    for (int b = 0; b < 2; b++)
        if (issued[b]) all_ok &= tc::mbar_wait_limit(&bar[b], phase[b], wait_cycles);
    if (__syncthreads_or(!all_ok) && tid == 0) gave_up = 1;
    __syncthreads();
    tc::fence_after();
    if (gave_up) {
        if (tid == 0) atomicOr(err, 2);
        for (int p = tid; p < npairs; p += G3_THREADS)
            partial[(int64_t)blockIdx.x * npairs + p] = __longlong_as_double(0x7ff8000000000000ll);
    } else {
        for (int p = tid; p < npairs; p += G3_THREADS) {
            int r = 0, left = p;
            while (left >= R - r) {
                left -= R - r;
                r++;
            }
            const int s2 = r + left;
            const float2 a = acc_s[64 * s2 + r], b = acc_s[64 * 64 + 64 * s2 + r];
            partial[(int64_t)blockIdx.x * npairs + p] = ((double)a.x + (double)a.y) + ((double)b.x + (double)b.y);
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::dealloc(tmem, G3_TMEM_COLS);
}

}  // namespace

int gram_f32_blocks(int64_t I) {
    int64_t g = (I + G3_STAGE_ROWS - 1) / G3_STAGE_ROWS;
    if (g > G3_BLOCKS) g = G3_BLOCKS;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t launch_gram_f32(const float *A, int64_t I, int R, double *partial, int *err, long long wait_cycles,
                            int fault_skip, cudaStream_t st) {
    if (R < 1 || R > 64) return cudaErrorInvalidValue;
    cudaError_t e = allow_max_dynamic_smem(k_gram_f32);
    if (e != cudaSuccess) return e;
    k_gram_f32<<<gram_f32_blocks(I), G3_THREADS, G3_SMEM, st>>>(A, I, R, partial, err,
                                                                 wait_cycles > 0 ? wait_cycles : kWaitCycles,
                                                                 fault_skip);
    return cudaGetLastError();
}

}  // namespace relate
