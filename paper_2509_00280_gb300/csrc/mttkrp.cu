// mttkrp.cu -- host-side launch configuration of the MTTKRP kernel:
// grid sizing in multiples of the SM count, shared-memory accumulators,
// vector-path eligibility.
#include "mttkrp_impl.cuh"

namespace relate {

int mttkrp_acc_bytes(int factor_dtype) { return factor_dtype == RELATE_F64 ? 8 : 4; }

cudaError_t launch_mttkrp(const MttkrpArgs &a_in, int KW, int factor_dtype, int val_dtype, int smem_budget,
                          int num_sms, cudaStream_t st) {
    MttkrpArgs a = a_in;
    if (a.nnz == 0 || a.P == 0) return cudaSuccess;
    const int accb = mttkrp_acc_bytes(factor_dtype);
    const int fb = factor_dtype == RELATE_F64 ? 8 : factor_dtype == RELATE_F32 ? 4 : 2;

    // 16-byte vector path: every factor row starts 16-byte aligned
    bool vec_ok = (a.R * fb) % 16 == 0 && (reinterpret_cast<uintptr_t>(a.out) % 16) == 0;
    for (int k = 0; k < a.N; k++)
        if (k != a.mode && (reinterpret_cast<uintptr_t>(a.factors[k]) % 16) != 0) vec_ok = false;

    size_t smem = 0;
    int per_sm = kThreads == 256 ? 8 : 2048 / kThreads;  // resident blocks without shared accumulators
    if (a.strategy == RELATE_CONFLICT_PRIVATIZED) {
        smem = (size_t)a.In * a.R * accb;
        if (smem > (size_t)smem_budget) return cudaErrorInvalidValue;
        per_sm = (int)((228 * 1024) / (smem + 1024));
        if (per_sm < 1) per_sm = 1;
        if (per_sm > 8) per_sm = 8;
    } else if (a.strategy == RELATE_CONFLICT_SEGMENTED) {
        // a window of up to ~24 KB keeps 8 blocks resident per SM
        int rows = (24 * 1024) / (a.R * accb);
        if (rows < 1) rows = 1;
        a.window_rows = rows;
        smem = (size_t)rows * a.R * accb;
    }
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > a.P) grid = a.P;
    if (grid < 1) grid = 1;
    switch (factor_dtype) {
    case RELATE_F64: return mttkrp_f64(a, KW, val_dtype, vec_ok, smem, (int)grid, st);
    case RELATE_F32: return mttkrp_f32(a, KW, val_dtype, vec_ok, smem, (int)grid, st);
    default: return mttkrp_bf16(a, KW, val_dtype, vec_ok, smem, (int)grid, st);
    }
}

}  // namespace relate
