// mttkrp_fac_bf16.cu -- instantiations of the fiber-factored MTTKRP kernel for
// __nv_bfloat16 factors (one translation unit per factor dtype so the build compiles
// them in parallel).
#include "mttkrp_impl.cuh"

namespace relate {

cudaError_t mttkrp_fac_bf16(const MttkrpArgs &a, int KW, int64_t tiles, int num_sms, cudaStream_t st) {
    return mk::dispatch_fac<__nv_bfloat16>(a, KW, tiles, num_sms, st);
}

}  // namespace relate
