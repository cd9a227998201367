// Instantiations of the native FP64 line-transform operator (variant 9).
#include "sem_ax_ln.cuh"

namespace sem {

int ln_set_coef(const double* cf, int lx) {
    const int off = ln_coef_off(lx);
    if (off < 0) return fail(SEM_EINVAL, "line-transform coefficients exist for lx in {4, 6, 8, 10, 12}");
    const int P = lx / 2;
    cudaError_t e = cudaMemcpyToSymbol(c_lncoef, cf, sizeof(double) * 4 * P * P, sizeof(double) * off);
    return e == cudaSuccess ? SEM_OK : cuda_fail(e, "cudaMemcpyToSymbol(FP64 line coefficients)");
}

int dispatch_ax_ln_entry(sem_handle* h, int lx, const AxParams<double>& a, bool fused, cudaStream_t s) {
    return fused ? dispatch_ax_ln<true>(h, lx, a, s) : dispatch_ax_ln<false>(h, lx, a, s);
}

}  // namespace sem
