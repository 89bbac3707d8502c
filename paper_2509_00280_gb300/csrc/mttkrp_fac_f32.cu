// mttkrp_fac_f32.cu -- instantiations of the fiber-factored MTTKRP kernel for
// float factors (one translation unit per factor dtype so the build compiles
// them in parallel).
#include "mttkrp_impl.cuh"

namespace relate {

cudaError_t mttkrp_fac_f32(const MttkrpArgs &a, int KW, int64_t tiles, int num_sms, cudaStream_t st) {
    return mk::dispatch_fac<float>(a, KW, tiles, num_sms, st);
}

}  // namespace relate
