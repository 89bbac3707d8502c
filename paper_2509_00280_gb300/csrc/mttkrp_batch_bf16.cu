// mttkrp_batch_bf16.cu -- instantiations of the batched (multi-problem)
// MTTKRP kernel for __nv_bfloat16 factors (one translation unit per factor dtype so the
// build compiles them in parallel).
#include "mttkrp_impl.cuh"

namespace relate {

cudaError_t mttkrp_batch_bf16(const mk::BatchParams &bp, int N, int KW, int num_sms, cudaStream_t st) {
    return mk::dispatch_batch<__nv_bfloat16>(bp, N, KW, num_sms, st);
}

}  // namespace relate
