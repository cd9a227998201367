// Instantiations of the FP32-pair (FP64-accurate) local operator kernels.
#include "sem_ax_df.cuh"

namespace sem {

int dfl_set_coef(const float* cf, int lx) {
    const int off = dfl_coef_off(lx);
    if (off < 0) return fail(SEM_EINVAL, "line-transform coefficients exist for lx in {4, 6, 8, 10, 12}");
    const int P = lx / 2;
    cudaError_t e = cudaMemcpyToSymbol(c_dflcoef, cf, sizeof(float) * 8 * P * P, sizeof(float) * off);
    return e == cudaSuccess ? SEM_OK : cuda_fail(e, "cudaMemcpyToSymbol(line coefficients)");
}

int dispatch_ax_df_entry(sem_handle* h, int lx, const DfParams& a, bool fused, cudaStream_t s) {
    return fused ? dispatch_ax_df<true>(h, lx, a, s) : dispatch_ax_df<false>(h, lx, a, s);
}

int dispatch_ax_dfl_entry(sem_handle* h, int lx, const DflParams& a, bool fused, cudaStream_t s) {
    return fused ? dispatch_ax_dfl<true>(h, lx, a, s) : dispatch_ax_dfl<false>(h, lx, a, s);
}

int dispatch_ax_dfl_pair_entry(sem_handle* h, int lx, const DflParams& a, cudaStream_t s) {
    return dispatch_ax_dfl_pair(h, lx, a, s);
}

int dispatch_ax_dfl_batch_entry(sem_handle* h, int lx, const DflParams& a, bool fused, cudaStream_t s) {
    return fused ? dispatch_ax_dfl_batch<true>(h, lx, a, s) : dispatch_ax_dfl_batch<false>(h, lx, a, s);
}

}  // namespace sem
