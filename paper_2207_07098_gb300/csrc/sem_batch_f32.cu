// Instantiations of the batched local operator kernels for float data.
#include "sem_batch.cuh"

namespace sem {

int dispatch_ax_batch_f32(sem_handle* h, int lx, const BatchAxParams<float>& a, bool fused, cudaStream_t s) {
    return fused ? dispatch_ax_batch<float, true>(h, lx, a, s) : dispatch_ax_batch<float, false>(h, lx, a, s);
}

}  // namespace sem
