// gram_noalloc.cu -- relate_gram_noalloc: the Gram step (G = A^T A) without
// any device-memory allocation.
//
// relate_gram obtains its per-block partial sums from a stream-ordered
// allocation on every call. Some callers cannot allocate device memory at
// that point: services that hand all device memory to their own pool up
// front (an extra allocation would fail or fragment it), and latency-critical
// loops where an allocator call that may synchronise the device is not
// acceptable. For them this entry point keeps the partials in a fixed array
// compiled into the library, so the caller only passes the input matrix and
// the output Gram. It makes CUDA runtime calls and launches kernels, so, like
// every CUDA call, it must not be made from inside a stream callback or a
// host function enqueued with cudaLaunchHostFunc.
//
// The array lives in every GPU that loads the library until the process exits
// (5.06 MB of FP64). All calls on a device share it: two calls whose kernels
// overlap on the GPU (different streams, no ordering between them) overwrite
// each other's partials and give wrong results, so such calls must be ordered.
// Every partial a call reads is written by the same call first; the one word
// that must start at zero (the tensor-core kernel's bounded-wait status) is
// cleared by each call before its kernels run.
#include <mutex>

#include "internal.cuh"

namespace relate {
int set_last_error(int status, const char *msg);  // capi.cu
bool fault_injected(const char *what);            // capi.cu
}

namespace {

// Per-block Gram partials: up to 304 blocks x 2080 upper-triangle entries
// (R = 64), plus the row-pass partial area and the status word of the same
// scratch layout.
constexpr size_t kScratchDoubles = 304u * 2080u + 304u * 64u + 64u;
static __device__ __align__(256) double g_gram_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
// Device address of g_gram_scratch per device, and the id of the CUDA context
// it was looked up in: a context created later on the same device (after
// cudaDeviceReset, or a destroyed and re-created primary context) loads the
// module again at another address, so the lookup is repeated.
double *g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

using CtxGetCurrentFn = int (*)(void **);
using CtxGetIdFn = int (*)(void *, unsigned long long *);

// Id of the current driver context (0 if it cannot be read). The driver
// entry points are looked up through the runtime, so the library does not
// link libcuda itself.
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of g_gram_scratch in the current context. In host code the
// symbol's name is only a host-side stand-in, so the address is looked up with
// the device current, once per device and context, and cached.
int scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return relate::set_last_error(RELATE_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return relate::set_last_error(RELATE_ERR_UNSUPPORTED, "relate_gram_noalloc: device ordinal >= 64");
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_gram_scratch);
        if (e != cudaSuccess || !p)
            return relate::set_last_error(RELATE_ERR_CUDA, "relate_gram_noalloc: cudaGetSymbolAddress failed");
        g_scratch_ptr[dev] = static_cast<double *>(p);
        g_scratch_ctx[dev] = ctx;
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
    const cudaStream_t st = (cudaStream_t)stream;
    int *err = relate::gram_err_word(scratch);
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    const bool f = relate::fault_injected("gram_timeout");  // test hook: no tensor-core work is issued
    if (e == cudaSuccess) e = relate::launch_gram(A, I, R, dtype, scratch, G, err, st, f ? 100000000LL : 0, f ? 1 : 0);
    if (e != cudaSuccess) return relate::set_last_error(RELATE_ERR_CUDA, cudaGetErrorString(e));
    if (I > 0 && relate::gram_uses_tc(A, R, dtype)) {
        // the tensor-core kernel reports a given-up wait in the status word:
        // read it (this synchronises the stream)
        int flag = 0;
        if ((e = cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return relate::set_last_error(RELATE_ERR_CUDA, cudaGetErrorString(e));
        if (flag)
            return relate::set_last_error(RELATE_ERR_TIMEOUT,
                                          "relate_gram_noalloc: a bounded tensor-core wait timed out (G is NaN)");
    }
    return RELATE_OK;
}
