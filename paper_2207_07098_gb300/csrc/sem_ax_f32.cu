// Instantiations of the plain local operator kernels for float data.
#include "sem_ax.cuh"

namespace sem {

int dispatch_ax_f32_plain(sem_handle* h, int lx, const AxParams<float>& a, cudaStream_t s) {
    return dispatch_ax<float, false>(h, lx, a, s);
}

}  // namespace sem
