// Instantiations of the CG-fused local operator kernels for float data.
#include "sem_ax.cuh"

namespace sem {

int dispatch_ax_f32_fused(sem_handle* h, int lx, const AxParams<float>& a, cudaStream_t s) {
    return dispatch_ax<float, true>(h, lx, a, s);
}

int dispatch_ax_f32(sem_handle* h, int lx, const AxParams<float>& a, bool fused, cudaStream_t s) {
    return fused ? dispatch_ax_f32_fused(h, lx, a, s) : dispatch_ax_f32_plain(h, lx, a, s);
}

}  // namespace sem
