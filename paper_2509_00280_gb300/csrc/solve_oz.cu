// solve_oz.cu -- the FP64 row pass of the normal equations, A_n = M V^{-1},
// on the tcgen05 tensor cores by exact 7-bit integer slices (the splitting
// scheme of Ozaki et al.).
//
// The CP-ALS update of Sec. 2.2 (the standard ALS the paper cites): after
// the MTTKRP M (I x R) and the inverse W = V^{-1} (R x R, FP64 from the
// Cholesky factor), every row is m_i W. As a GEMM, D (128 rows x R) = M_tile
// (128 x R) * W, K = R. Row i of M is put on a fixed-point scale from its own
// largest exponent field e_i, column s of W from its own E_s:
//   m_ir = p_ir 2^(e_i - 1077),  w_rs = q_rs 2^(E_s - 1077),  |p|, |q| < 2^55,
// both truncated toward zero, and cut into 8 signed 7-bit slices (most
// significant first), each exactly a BF16 value. Every pair of slices (u, v)
// is one BF16 x BF16 MMA accumulating in FP32 in tensor memory, the pairs of
// one group g = u + v in one accumulator; a group has at most 8 pairs of K <=
// 64 products of magnitude <= 127^2, so its sum is an integer below 2^23 and
// the tensor cores add exactly. The drain reads the 15 groups back
// (tcgen05.ld), forms
//   sum_r p_ir q_rs = sum_g acc_g 2^(7 (14 - g))
// exactly in a 128-bit integer and rounds it once to FP64 (round to
// nearest, integer operations only) with the scale 2^(e_i + E_s - 2154).
// The only errors are the truncations of p and q: |error| <= 2^-54 sum_r
// (max_r |m_ir| |w_rs| + |m_ir| max_r |w_rs|) <= 2^-53 R max|m_i| max|w_s|,
// the order of FP64's own dot-product error bound (gamma_R sum_r |m_ir w_rs|),
// plus the final rounding.
//
// Layout: W's 8 slices (B operand) are staged once per block, per 32-column
// half of the output and 16-wide K chunk one 256-row block whose row 32 v + j
// is slice v of output column j, so that one MMA of M = 128, N = 256, K = 16
// forms the pairs (u, 0..7) of slice u of a row tile into the 8 consecutive
// group accumulators u..u+7 (32 tensor-memory columns each, 480 in all; the
// groups 8..14 are zeroed first by one MMA of a zero operand). Per 128-row
// tile the 8 slices of M (A operand, M = 128 x K) are staged (K-major core
// matrices, tcgen05.cuh); per half 1 + 8 K/16 MMAs, then 8 warps drain the
// groups. The tile is read completely before its rows are overwritten (in
// place).
#include "internal.cuh"
#include "slices.cuh"
#include "tcgen05.cuh"

namespace relate {
namespace {

using sl::expo_of;
using sl::slices8;

constexpr int SO_THREADS = 256;
constexpr int SO_ROWS = 128;
constexpr int SO_S = 8;                           // slices per entry
constexpr int SO_GROUPS = 2 * SO_S - 1;           // g = u + v in 0..14
constexpr int SO_MBLK = SO_ROWS * 16 * 2;         // one slice of one 16-wide K chunk of the tile: 4 KB
constexpr int SO_WBLK = 256 * 16 * 2;             // one K chunk of one 32-column half of W, all 8 slices: 8 KB
constexpr int SO_MBYTES = SO_S * 4 * SO_MBLK;     // 128 KB
constexpr int SO_WBYTES = 2 * 4 * SO_WBLK;        // 64 KB
constexpr int SO_ZBYTES = SO_ROWS * 16 * 2;        // a zero A operand (128 x 16): 4 KB
constexpr int SO_BLOCKS = 152;
constexpr uint32_t SO_TMEM_COLS = 512;

// Round a signed 128-bit integer times 2^scale to the nearest FP64 (ties to
// even), integer operations only while the result is a normal number.
__device__ __forceinline__ double i128_to_double(__int128 v, int scale) {
    if (v == 0) return 0.0;
    const bool neg = v < 0;
    unsigned __int128 a = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const uint64_t hi = (uint64_t)(a >> 64), lo = (uint64_t)a;
    const int nbits = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
    uint64_t mant;
    int sh = nbits - 53;
    if (sh > 0) {
        mant = (uint64_t)(a >> sh);
        const unsigned __int128 rem = a & ((((unsigned __int128)1) << sh) - 1);
        const unsigned __int128 half = ((unsigned __int128)1) << (sh - 1);
        if (rem > half || (rem == half && (mant & 1))) {
            mant++;
            if (mant == (1ull << 53)) {
                mant >>= 1;
                sh++;
            }
        }
    } else {
        mant = lo << (-sh);
    }
    const int ef = 1075 + sh + scale;  // value = mant * 2^(sh + scale), mant in [2^52, 2^53)
    if (ef >= 1 && ef <= 2046)
        return __longlong_as_double((long long)(((uint64_t)neg << 63) | ((uint64_t)ef << 52) |
                                                (mant & 0xfffffffffffffull)));
    const double d = ldexp((double)mant, sh + scale);  // subnormal or overflow: rare, FP64 path
    return neg ? -d : d;
}

// In place M <- M W for FP64 M (I x R row-major, R <= 64) and W (R x R
// row-major). Bounded waits: on a timeout err |= 2
// and the block stops (rows it had not finished keep M); fault_skip (a test
// hook) issues no MMA and no commit.
__global__ void __launch_bounds__(SO_THREADS, 1)
    k_solve_oz(double *__restrict__ M, int64_t I, int R, const double *__restrict__ W, int *__restrict__ err,
               long long wait_cycles, int fault_skip) {
    extern __shared__ __align__(1024) unsigned char smem_so[];
    unsigned char *sm = smem_so;               // M slices: [slice][chunk] 4 KB blocks
    unsigned char *sw = smem_so + SO_MBYTES;   // W slices: [half][chunk] 8 KB blocks of 256 N rows
    unsigned char *sz = sw + SO_WBYTES;        // zeros
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int gave_up;
    __shared__ int wexp[64];
    __shared__ int rexp[SO_ROWS];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int KC = (R + 15) / 16;              // 16-wide K chunks
    const int NH = (R + 31) / 32;              // 32-column output halves
    const int64_t ntiles = (I + SO_ROWS - 1) / SO_ROWS;

    // ---- W: column exponents, then its 8 slices as the B operand (row s = output column)
    if (tid < 64) wexp[tid] = 0;
    __syncthreads();
    for (int x = tid; x < R * R; x += SO_THREADS) atomicMax(&wexp[x % R], expo_of(W[x]));
    __syncthreads();
    // B operand of half h, chunk c: N row n = 32 v + j is slice v of output column 32 h + j, so one
    // N = 256 MMA forms the pairs (u, 0..7) of a slice u of M into 8 consecutive groups
    for (int x = tid; x < 64 * 64; x += SO_THREADS) {  // (s, k = r), zero outside R x R
        const int s = x >> 6, r = x & 63;
        uint32_t u[SO_S];
        const double w = (s < R && r < R) ? W[r * R + s] : 0.0;
        slices8(w, s < R ? wexp[s] : 0, u);
        unsigned char *blk = sw + (size_t)((s >> 5) * 4 + (r >> 4)) * SO_WBLK;
#pragma unroll
        for (int k = 0; k < SO_S; k++) {
            const int n = 32 * k + (s & 31);
            *reinterpret_cast<uint16_t *>(blk + (n >> 3) * 256 + ((r & 15) >> 3) * 128 + (n & 7) * 16 + (r & 7) * 2) =
                (uint16_t)u[k];
        }
    }
    for (int x = tid; x < SO_ZBYTES / 4; x += SO_THREADS) reinterpret_cast<uint32_t *>(sz)[x] = 0u;
    if (warp == 0) tc::alloc(&tmem_base, SO_TMEM_COLS);
    if (tid == 0) {
        tc::mbar_init1(&bar);
        gave_up = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = tc::instr_desc_bf16(128, 256);
    const uint32_t idesc_z = tc::instr_desc_bf16(128, 224);
    uint32_t phase = 0;
    bool stop = false;

    // staging role: row i = tid / 2 of the tile, columns [32 (tid & 1), +32)
    const int si = tid >> 1, sc0 = 32 * (tid & 1);
    // drain role: D lane quarter q (rows 32q..), 16 columns of the half
    const int q = warp & 3, dc0 = 16 * (warp >> 2);

    for (int64_t tile = blockIdx.x; tile < ntiles && !stop; tile += gridDim.x) {
        const int64_t t0 = tile * SO_ROWS;
        // ---- stage the tile's rows as 8 slices on the rows' own scales
        {
            const int64_t row = t0 + si;
            double x[32];
#pragma unroll
            for (int j = 0; j < 32; j++) x[j] = (row < I && sc0 + j < R) ? M[row * R + sc0 + j] : 0.0;
            int e = 0;
#pragma unroll
            for (int j = 0; j < 32; j++) e = max(e, expo_of(x[j]));
            e = max(e, __shfl_xor_sync(0xffffffffu, e, 1));
            if ((tid & 1) == 0) rexp[si] = e;
#pragma unroll
            for (int g8 = 0; g8 < 4; g8++) {  // 8 consecutive K entries = one 16-byte core-matrix row
                const int r0 = sc0 + 8 * g8;
                uint32_t u[8][SO_S];
#pragma unroll
                for (int j = 0; j < 8; j++) slices8(x[8 * g8 + j], e, u[j]);
                const uint32_t off = (uint32_t)((si >> 3) * 256 + ((r0 & 15) >> 3) * 128 + (si & 7) * 16);
#pragma unroll
                for (int k = 0; k < SO_S; k++) {
                    uint4 v;
                    v.x = u[0][k] | (u[1][k] << 16);
                    v.y = u[2][k] | (u[3][k] << 16);
                    v.z = u[4][k] | (u[5][k] << 16);
                    v.w = u[6][k] | (u[7][k] << 16);
                    *reinterpret_cast<uint4 *>(sm + (size_t)(k * 4 + (r0 >> 4)) * SO_MBLK + off) = v;
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
        __syncthreads();

        for (int h = 0; h < NH; h++) {
            if (tid == 0 && !fault_skip) {
                tc::fence_after();
                // descriptors differ only in the start address field (address >> 4, below 2^14 for
                // shared memory): offsets are added to base descriptors
                const uint64_t dm0 = tc::smem_desc(tc::saddr(sm), 128, 256);
                const uint64_t dw0 = tc::smem_desc(tc::saddr(sw) + (uint32_t)(h * 4 * SO_WBLK), 128, 256);
                // groups 8..14 (columns 256..479) start at zero: one MMA of a zero A operand
                tc::mma(tmem + 256u, tc::smem_desc(tc::saddr(sz), 128, 256), dw0, idesc_z, 0u);
#pragma unroll 1
                for (int c = 0; c < KC; c++)
#pragma unroll
                    for (int u = 0; u < SO_S; u++) {
                        // pairs (u, v = 0..7) into groups u..u+7 (columns 32 u .. 32 u + 255); the first
                        // MMA writes groups 0..7, every later one accumulates
                        const uint64_t da = dm0 + (uint64_t)(((u * 4 + c) * SO_MBLK) >> 4);
                        const uint64_t db = dw0 + (uint64_t)((c * SO_WBLK) >> 4);
                        tc::mma(tmem + 32u * (uint32_t)u, da, db, idesc, (c == 0 && u == 0) ? 0u : 1u);
                    }
                tc::commit(&bar);
            }
            const bool ok = tc::mbar_wait_limit(&bar, phase, wait_cycles);
            phase ^= 1;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) gave_up = 1;
                stop = true;
                break;
            }
            tc::fence_after();
            // ---- drain: row i = 32q + lane of the tile, columns 32h + dc0 + 0..15
            {
                const int i = 32 * q + lane;
                const int64_t row = t0 + i;
                const int e = rexp[i];
                const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)dc0;
#pragma unroll
                for (int cq = 0; cq < 2; cq++) {  // 8 columns at a time
                    long long w[4][8];  // groups 4k..4k+3 with weights 2^(7 (4k + 3 - g))
#pragma unroll
                    for (int half8 = 0; half8 < 2; half8++) {  // groups 0..7, then 8..14: two waits
                        uint32_t va[32], vb[32];
#pragma unroll
                        for (int gg = 0; gg < 8; gg++) {
                            const int g = 8 * half8 + gg;
                            if (g < SO_GROUPS)
                                tc::ld8_nowait(tb + 32u * (uint32_t)g + 8u * (uint32_t)cq, (gg < 4 ? va : vb) + 8 * (gg & 3));
                        }
                        tc::wait_ld32(va);
                        tc::wait_ld32(vb);
#pragma unroll
                        for (int kk = 0; kk < 2; kk++) {
                            const int k = 2 * half8 + kk;
                            const uint32_t *v = kk == 0 ? va : vb;
#pragma unroll
                            for (int j = 0; j < 8; j++)  // group 15 does not exist: its slot reads as 0
                                w[k][j] = sl::word4(__uint_as_float(v[j]), __uint_as_float(v[8 + j]),
                                                    __uint_as_float(v[16 + j]),
                                                    4 * k + 3 < SO_GROUPS ? __uint_as_float(v[24 + j]) : 0.0f);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        const int s = 32 * h + dc0 + 8 * cq + j;
                        if (row >= I || s >= R) continue;
                        // sum_g acc_g 2^(7 (14 - g)) = w0 2^77 + w1 2^49 + w2 2^21 + w3 2^-7; times 2^7 to stay integral
                        const __int128 tot = (__int128)w[0][j] * ((__int128)1 << 84) +
                                             (__int128)w[1][j] * ((__int128)1 << 56) +
                                             (__int128)w[2][j] * ((__int128)1 << 28) + (__int128)w[3][j];
                        const int Es = wexp[s];
                        double out;
                        if (e >= 0x7ff || Es >= 0x7ff) out = __longlong_as_double(0x7ff8000000000000ll);
                        else if (e == 0 || Es == 0) out = 0.0;
                        else out = i128_to_double(tot, e + Es - 2154 - 7);
                        M[row * R + s] = out;
                    }
                }
            }
            tc::fence_before();
            __syncthreads();  // the next MMAs overwrite the accumulators; the next tile restages
        }
    }
    __syncthreads();
    if (gave_up && tid == 0) atomicOr(err, 2);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::dealloc(tmem, SO_TMEM_COLS);
}

}  // namespace

cudaError_t launch_solve_oz(double *M, int64_t I, int R, const double *W, int *err, long long wait_cycles,
                            int fault_skip, cudaStream_t st) {
    if (R < 1 || R > 64) return cudaErrorInvalidValue;
    if (I == 0) return cudaSuccess;
    int64_t g = (I + SO_ROWS - 1) / SO_ROWS;
    if (g > SO_BLOCKS) g = SO_BLOCKS;
    cudaError_t e = allow_max_dynamic_smem(k_solve_oz);
    if (e != cudaSuccess) return e;
    k_solve_oz<<<(unsigned)g, SO_THREADS, SO_MBYTES + SO_WBYTES + SO_ZBYTES, st>>>(
        M, I, R, W, err, wait_cycles > 0 ? wait_cycles : kWaitCycles, fault_skip);
    return cudaGetLastError();
}

}  // namespace relate
