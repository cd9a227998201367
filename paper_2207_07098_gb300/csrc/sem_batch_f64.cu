// Instantiations of the batched local operator kernels for double data.
#include "sem_batch.cuh"

namespace sem {

int dispatch_ax_batch_f64(sem_handle* h, int lx, const BatchAxParams<double>& a, bool fused, cudaStream_t s) {
    return fused ? dispatch_ax_batch<double, true>(h, lx, a, s) : dispatch_ax_batch<double, false>(h, lx, a, s);
}

}  // namespace sem
