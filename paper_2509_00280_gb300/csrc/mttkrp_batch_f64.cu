// mttkrp_batch_f64.cu -- instantiations of the batched (multi-problem)
// MTTKRP kernel for double factors (one translation unit per factor dtype so the
// build compiles them in parallel).
#include "mttkrp_impl.cuh"

namespace relate {

cudaError_t mttkrp_batch_f64(const mk::BatchParams &bp, int N, int KW, int num_sms, cudaStream_t st) {
    return mk::dispatch_batch<double>(bp, N, KW, num_sms, st);
}

}  // namespace relate
