// mttkrp_fac_f64.cu -- instantiations of the fiber-factored MTTKRP kernel for
// double factors (one translation unit per factor dtype so the build compiles
// them in parallel).
#include "mttkrp_impl.cuh"

namespace relate {

cudaError_t mttkrp_fac_f64(const MttkrpArgs &a, int KW, int64_t tiles, int num_sms, cudaStream_t st) {
    return mk::dispatch_fac<double>(a, KW, tiles, num_sms, st);
}

}  // namespace relate
