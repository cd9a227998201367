// Instantiations of the plain local operator kernels for double data.
#include "sem_ax.cuh"

namespace sem {

int dispatch_ax_f64_plain(sem_handle* h, int lx, const AxParams<double>& a, cudaStream_t s) {
    return dispatch_ax<double, false>(h, lx, a, s);
}

}  // namespace sem
