// Instantiations of the CG-fused local operator kernels for double data.
#include "sem_ax.cuh"

namespace sem {

int dispatch_ax_f64_fused(sem_handle* h, int lx, const AxParams<double>& a, cudaStream_t s) {
    return dispatch_ax<double, true>(h, lx, a, s);
}

int dispatch_ax_f64(sem_handle* h, int lx, const AxParams<double>& a, bool fused, cudaStream_t s) {
    return fused ? dispatch_ax_f64_fused(h, lx, a, s) : dispatch_ax_f64_plain(h, lx, a, s);
}

}  // namespace sem
