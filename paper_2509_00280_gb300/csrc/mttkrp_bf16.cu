// mttkrp_bf16.cu -- instantiations of the MTTKRP kernel for __nv_bfloat16 factors
// (one translation unit per factor dtype so the build compiles them in parallel).
#include "mttkrp_impl.cuh"

namespace relate {

cudaError_t mttkrp_bf16(const MttkrpArgs &a, int KW, bool vec_ok, size_t acc_bytes, int grid, cudaStream_t st) {
    return mk::dispatch_ft<__nv_bfloat16>(a, KW, vec_ok, acc_bytes, grid, st);
}

}  // namespace relate
