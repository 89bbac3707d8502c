// gram_noalloc.cu -- relate_gram_noalloc: the Gram step (G = A^T A) without
// any device-memory allocation.
//
// relate_gram obtains its per-block partial sums from a stream-ordered
// allocation on every call. Some callers cannot allocate device memory at
// that point: code running inside a host callback enqueued on a stream (CUDA
// calls are not allowed there), services that hand all device memory to
// their own pool up front (an extra allocation would fail or fragment it),
// and latency-critical loops where an allocator call that may synchronise the
// device is not acceptable. For them this entry point keeps the partials in a
// fixed array compiled into the library, so the caller only passes the input
// matrix and the output Gram.
//
// The array lives in every GPU that loads the library until the process exits
// (5.06 MB of FP64). All calls on a device share it: two calls whose kernels
// overlap on the GPU (different streams, no ordering between them) overwrite
// each other's partials and give wrong results, so such calls must be ordered.
// Every partial a call reads is written by the same call first, so nothing is
// carried over from a previous call and nothing needs clearing.
#include <mutex>

#include "internal.cuh"

namespace relate {
int set_last_error(int status, const char *msg);  // capi.cu
}

namespace {

// Per-block Gram partials: up to 304 blocks x 2080 upper-triangle entries
// (R = 64), plus the row-pass partial area of the same scratch layout.
constexpr size_t kScratchDoubles = 304u * 2080u + 304u * 64u + 64u;
static __device__ __align__(256) double g_gram_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_gram_scratch on the current device. In host code the
// symbol's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
int scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return relate::set_last_error(RELATE_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return relate::set_last_error(RELATE_ERR_UNSUPPORTED, "relate_gram_noalloc: device ordinal >= 64");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_gram_scratch);
        if (e != cudaSuccess || !p)
            return relate::set_last_error(RELATE_ERR_CUDA, "relate_gram_noalloc: cudaGetSymbolAddress failed");
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return RELATE_OK;
}

}  // namespace

extern "C" int relate_gram_noalloc(const void *A, int64_t I, int R, relate_dtype_t dtype, double *G,
                                   void *stream) {
    relate::set_last_error(RELATE_OK, "");
    if ((!A && I > 0) || !G || I < 0 ||
        (dtype != RELATE_F64 && dtype != RELATE_F32 && dtype != RELATE_BF16))
        return relate::set_last_error(RELATE_ERR_INVALID_ARG, "relate_gram_noalloc: bad argument");
    if (R < 1 || R > RELATE_MAX_RANK)
        return relate::set_last_error(RELATE_ERR_INVALID_ARG,
                                      "relate_gram_noalloc: R must be in [1, 64] (the fixed scratch holds "
                                      "the partial sums of at most 64 columns)");
    if (relate::dense_scratch_doubles(R) > kScratchDoubles)
        return relate::set_last_error(RELATE_ERR_UNSUPPORTED,
                                      "relate_gram_noalloc: partial sums exceed the fixed scratch");
    double *scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc != RELATE_OK) return rc;
    const cudaError_t e = relate::launch_gram(A, I, R, dtype, scratch, G, (cudaStream_t)stream);
    if (e != cudaSuccess) return relate::set_last_error(RELATE_ERR_CUDA, cudaGetErrorString(e));
    return RELATE_OK;
}
