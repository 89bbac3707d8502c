// mttkrp_impl.cuh -- the mode-n MTTKRP kernel over the linearized encoding.
//
// Sec. 2.2 and Fig. 2 of the paper: every nonzero (i_0..i_{N-1}, v) reads
// rows i_k of the factors A_k (k != n), multiplies them element-wise, scales
// by v and adds the result into row i_n of the output; writes to one row
// from many nonzeros must be synchronised (Sec. 2.2; Sec. 4.1.3 picks
// reduction or atomics per mode from fiber reuse).
//
// GB300 mapping:
//  * A block walks equal-work partitions of the sorted stream (grid-stride,
//    so neighbouring blocks work on neighbouring partitions and share factor
//    rows in L2).
//  * Inside a block, a "group" of G lanes owns one nonzero at a time; each
//    lane holds 16 bytes of the R-wide row (VEC elements), so a factor-row
//    gather is G coalesced 16-byte loads (one 128-byte line for R = 32 FP32).
//  * Each group walks a contiguous slice of the partition. Consecutive
//    nonzeros with the same output row (runs of equal i_n in encoded order)
//    are summed in registers; a run is flushed once:
//      ATOMIC      -> global vector atomics (red.global.add.v4.f32 / f64),
//      SEGMENTED   -> shared-memory atomics into a window over the
//                     partition's [lo_n, hi_n] rows, flushed per partition,
//      PRIVATIZED  -> shared-memory atomics into a block-private copy of the
//                     whole output, flushed once per block.
#pragma once

#include "internal.cuh"

namespace relate {
namespace mk {

template <typename FT> struct Prec;
template <> struct Prec<double> {
    using C = double;
    static constexpr int VEC = 2;
};
template <> struct Prec<float> {
    using C = float;
    static constexpr int VEC = 4;
};
template <> struct Prec<__nv_bfloat16> {
    using C = float;
    static constexpr int VEC = 8;
};

template <int KW> __device__ __forceinline__ typename WordT<KW>::T load_word(const void *p, int64_t j);
template <> __device__ __forceinline__ uint32_t load_word<1>(const void *p, int64_t j) {
    return __ldg(reinterpret_cast<const unsigned int *>(p) + j);
}
template <> __device__ __forceinline__ unsigned long long load_word<2>(const void *p, int64_t j) {
    return __ldg(reinterpret_cast<const unsigned long long *>(p) + j);
}
template <> __device__ __forceinline__ W128 load_word<4>(const void *p, int64_t j) {
    uint4 u = __ldg(reinterpret_cast<const uint4 *>(p) + j);
    W128 w;
    w.lo = ((uint64_t)u.y << 32) | u.x;
    w.hi = ((uint64_t)u.w << 32) | u.z;
    return w;
}

__device__ __forceinline__ uint32_t fld(uint32_t w, int s, uint32_t m) { return (uint32_t)((uint64_t)w >> s) & m; }
__device__ __forceinline__ uint32_t fld(unsigned long long w, int s, uint32_t m) { return (uint32_t)(w >> s) & m; }
__device__ __forceinline__ uint32_t fld(W128 w, int s, uint32_t m) {
    uint64_t x;
    if (s >= 64)
        x = w.hi >> (s - 64);
    else if (s == 0)
        x = w.lo;
    else
        x = (w.lo >> s) | (w.hi << (64 - s));
    return (uint32_t)x & m;
}

// 16-byte (or scalar) load of vector j of a factor row, converted to C.
template <typename FT, int VEC> struct VecLoad;
template <> struct VecLoad<double, 2> {
    static __device__ __forceinline__ void run(const double *row, int j, double (&x)[2]) {
        double2 v = __ldg(reinterpret_cast<const double2 *>(row) + j);
        x[0] = v.x;
        x[1] = v.y;
    }
};
template <> struct VecLoad<float, 4> {
    static __device__ __forceinline__ void run(const float *row, int j, float (&x)[4]) {
        float4 v = __ldg(reinterpret_cast<const float4 *>(row) + j);
        x[0] = v.x;
        x[1] = v.y;
        x[2] = v.z;
        x[3] = v.w;
    }
};
template <> struct VecLoad<__nv_bfloat16, 8> {
    static __device__ __forceinline__ void run(const __nv_bfloat16 *row, int j, float (&x)[8]) {
        uint4 u = __ldg(reinterpret_cast<const uint4 *>(row) + j);
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int i = 0; i < 4; i++) {
            x[2 * i] = __uint_as_float(w[i] << 16);             // low bf16
            x[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);  // high bf16
        }
    }
};
template <typename FT> struct VecLoad<FT, 1> {
    using C = typename Prec<FT>::C;
    static __device__ __forceinline__ void run(const FT *row, int j, C (&x)[1]) {
        x[0] = (C)row[j];
    }
};

// global accumulation of one vector (VEC elements) at out + off
template <typename C, int VEC> struct GAdd;
template <> struct GAdd<float, 4> {
    static __device__ __forceinline__ void run(float *p, const float (&a)[4]) {
        atomicAdd(reinterpret_cast<float4 *>(p), make_float4(a[0], a[1], a[2], a[3]));
    }
};
template <> struct GAdd<float, 8> {
    static __device__ __forceinline__ void run(float *p, const float (&a)[8]) {
        atomicAdd(reinterpret_cast<float4 *>(p), make_float4(a[0], a[1], a[2], a[3]));
        atomicAdd(reinterpret_cast<float4 *>(p) + 1, make_float4(a[4], a[5], a[6], a[7]));
    }
};
template <> struct GAdd<double, 2> {
    static __device__ __forceinline__ void run(double *p, const double (&a)[2]) {
        atomicAdd(p, a[0]);
        atomicAdd(p + 1, a[1]);
    }
};
template <typename C> struct GAdd<C, 1> {
    static __device__ __forceinline__ void run(C *p, const C (&a)[1]) { atomicAdd(p, a[0]); }
};

template <int NT, int KW, typename FT, typename VT, int VEC, int VPL>
__global__ void __launch_bounds__(kThreads) k_mttkrp(const MttkrpArgs a, const int log2G) {
    using C = typename Prec<FT>::C;
    using Word = typename WordT<KW>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sacc = reinterpret_cast<C *>(smem_raw);

    const int N = NT ? NT : a.N;
    const int G = 1 << log2G;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int gid = threadIdx.x >> log2G;
    const int ngroups = kThreads >> log2G;
    const int R = a.R;
    const int nvec = (R + VEC - 1) / VEC;
    const int mode = a.mode;
    const int mshift = a.fields.shift[mode];
    const uint32_t mmask = a.fields.mask[mode];
    const VT *__restrict__ vals = reinterpret_cast<const VT *>(a.vals);
    C *__restrict__ out = reinterpret_cast<C *>(a.out);
    const int strat = a.strategy;

    int vj[VPL];
    bool act[VPL];
#pragma unroll
    for (int v = 0; v < VPL; v++) {
        vj[v] = gl + v * G;
        act[v] = vj[v] < nvec;
    }

    if (strat == RELATE_CONFLICT_PRIVATIZED) {
        const int64_t tot = (int64_t)a.In * R;
        for (int64_t i = threadIdx.x; i < tot; i += kThreads) sacc[i] = C(0);
        __syncthreads();
    }

    for (int64_t q = blockIdx.x; q < a.P; q += gridDim.x) {
        const int64_t b = q * a.S;
        const int64_t e = min(b + a.S, a.nnz);
        const int64_t chunk = (e - b + ngroups - 1) / ngroups;
        const int64_t jb = min(b + gid * chunk, e);
        const int64_t je = min(jb + chunk, e);

        bool win = false;
        uint32_t wlo = 0, wrows = 0;
        if (strat == RELATE_CONFLICT_SEGMENTED) {
            wlo = a.plo[q * N + mode];
            wrows = a.phi[q * N + mode] - wlo + 1;
            win = (int)wrows <= a.window_rows;
            if (win) {
                const int tot = (int)wrows * R;
                for (int i = threadIdx.x; i < tot; i += kThreads) sacc[i] = C(0);
                __syncthreads();
            }
        }
        C *acc_base;          // where runs are flushed
        int64_t row_bias;     // row offset subtracted before indexing acc_base
        bool shared_acc;
        if (strat == RELATE_CONFLICT_PRIVATIZED) {
            acc_base = sacc;
            row_bias = 0;
            shared_acc = true;
        } else if (win) {
            acc_base = sacc;
            row_bias = wlo;
            shared_acc = true;
        } else {
            acc_base = out;
            row_bias = 0;
            shared_acc = false;
        }

        uint32_t cur = 0xffffffffu;
        C acc[VPL][VEC];
#pragma unroll
        for (int v = 0; v < VPL; v++)
#pragma unroll
            for (int i = 0; i < VEC; i++) acc[v][i] = C(0);

        auto flush = [&](uint32_t row) {
            C *dst = acc_base + ((int64_t)row - row_bias) * R;
#pragma unroll
            for (int v = 0; v < VPL; v++) {
                if (!act[v]) continue;
                C *p = dst + vj[v] * VEC;
                if (shared_acc) {
#pragma unroll
                    for (int i = 0; i < VEC; i++)
                        if (vj[v] * VEC + i < R) atomicAdd(p + i, acc[v][i]);
                } else {
                    if (VEC == 1 || (vj[v] + 1) * VEC <= R) {
                        GAdd<C, VEC>::run(p, acc[v]);
                    } else {
#pragma unroll
                        for (int i = 0; i < VEC; i++)
                            if (vj[v] * VEC + i < R) atomicAdd(p + i, acc[v][i]);
                    }
                }
            }
        };

        for (int64_t j = jb; j < je; j++) {
            const Word w = load_word<KW>(a.words, j);
            const C val = (C)__ldg(vals + j);
            const uint32_t row = fld(w, mshift, mmask);
            if (row != cur) {
                if (cur != 0xffffffffu) flush(cur);
#pragma unroll
                for (int v = 0; v < VPL; v++)
#pragma unroll
                    for (int i = 0; i < VEC; i++) acc[v][i] = C(0);
                cur = row;
            }
            C t[VPL][VEC];
#pragma unroll
            for (int v = 0; v < VPL; v++)
#pragma unroll
                for (int i = 0; i < VEC; i++) t[v][i] = val;
#pragma unroll
            for (int k = 0; k < (NT ? NT : kMaxModes); k++) {
                if (k >= N || k == mode) continue;
                const uint32_t ik = fld(w, a.fields.shift[k], a.fields.mask[k]);
                const FT *rowp = reinterpret_cast<const FT *>(a.factors[k]) + (int64_t)ik * R;
#pragma unroll
                for (int v = 0; v < VPL; v++) {
                    if (!act[v]) continue;
                    C x[VEC];
                    VecLoad<FT, VEC>::run(rowp, vj[v], x);
#pragma unroll
                    for (int i = 0; i < VEC; i++) t[v][i] *= x[i];
                }
            }
#pragma unroll
            for (int v = 0; v < VPL; v++)
#pragma unroll
                for (int i = 0; i < VEC; i++) acc[v][i] += t[v][i];
        }
        if (cur != 0xffffffffu) flush(cur);

        if (win) {
            __syncthreads();
            const int tot = (int)wrows * R;
            C *gdst = out + (int64_t)wlo * R;
            for (int i = threadIdx.x; i < tot; i += kThreads) {
                C s = sacc[i];
                if (s != C(0)) atomicAdd(gdst + i, s);
            }
            __syncthreads();
        } else if (strat == RELATE_CONFLICT_SEGMENTED) {
            // keep the block's partitions in lock-step (a later partition may
            // take the window path and zero the shared buffer)
            __syncthreads();
        }
    }

    if (strat == RELATE_CONFLICT_PRIVATIZED) {
        __syncthreads();
        const int64_t tot = (int64_t)a.In * R;
        for (int64_t i = threadIdx.x; i < tot; i += kThreads) {
            C s = sacc[i];
            if (s != C(0)) atomicAdd(out + i, s);
        }
    }
}

// Chooses lanes per group for R and launches one instantiation.
template <int NT, int KW, typename FT, typename VT, int VEC, int VPL>
cudaError_t launch_one(const MttkrpArgs &a, size_t smem, int grid, cudaStream_t st) {
    const int nvec = (a.R + VEC - 1) / VEC;
    int G = 1, log2G = 0;
    while (G * VPL < nvec && G < 32) {
        G <<= 1;
        log2G++;
    }
    auto kern = k_mttkrp<NT, KW, FT, VT, VEC, VPL>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, kThreads, smem, st>>>(a, log2G);
    return cudaGetLastError();
}

// Dispatch over N (3, 4, generic), word width and value dtype for one FT.
template <typename FT>
cudaError_t dispatch_ft(const MttkrpArgs &a, int KW, int val_dtype, bool vec_ok, size_t smem, int grid,
                        cudaStream_t st) {
    constexpr int V = Prec<FT>::VEC;
#define RELATE_MK_VT(NT_, KW_, VT_)                                                    \
    (vec_ok ? launch_one<NT_, KW_, FT, VT_, V, 1>(a, smem, grid, st)                   \
            : launch_one<0, KW_, FT, VT_, 1, 2>(a, smem, grid, st))
#define RELATE_MK_KW(NT_, VT_)                                                         \
    (KW == 1 ? RELATE_MK_VT(NT_, 1, VT_) : KW == 2 ? RELATE_MK_VT(NT_, 2, VT_) : RELATE_MK_VT(NT_, 4, VT_))
    if (val_dtype == RELATE_F64) {
        if (a.N == 3) return RELATE_MK_KW(3, double);
        if (a.N == 4) return RELATE_MK_KW(4, double);
        return RELATE_MK_KW(0, double);
    }
    if (a.N == 3) return RELATE_MK_KW(3, float);
    if (a.N == 4) return RELATE_MK_KW(4, float);
    return RELATE_MK_KW(0, float);
#undef RELATE_MK_KW
#undef RELATE_MK_VT
}

}  // namespace mk

cudaError_t mttkrp_f64(const MttkrpArgs &a, int KW, int val_dtype, bool vec_ok, size_t smem, int grid, cudaStream_t st);
cudaError_t mttkrp_f32(const MttkrpArgs &a, int KW, int val_dtype, bool vec_ok, size_t smem, int grid, cudaStream_t st);
cudaError_t mttkrp_bf16(const MttkrpArgs &a, int KW, int val_dtype, bool vec_ok, size_t smem, int grid, cudaStream_t st);

}  // namespace relate
