// mttkrp_f64.cu -- instantiations of the MTTKRP kernel for double factors
// (one translation unit per factor dtype so the build compiles them in parallel).
#include "mttkrp_impl.cuh"

namespace relate {

cudaError_t mttkrp_f64(const MttkrpArgs &a, int KW, bool vec_ok, size_t acc_bytes, int grid, cudaStream_t st) {
    return mk::dispatch_ft<double>(a, KW, vec_ok, acc_bytes, grid, st);
}

}  // namespace relate
