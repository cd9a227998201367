// Instantiations of the bulk-staged local operator kernels for float data.
#include "sem_ax_bulk.cuh"

namespace sem {

int dispatch_ax_bulk_f32(sem_handle* h, int lx, const AxParams<float>& a, bool fused, cudaStream_t s) {
    return fused ? dispatch_ax_bulk<float, true>(h, lx, a, s) : dispatch_ax_bulk<float, false>(h, lx, a, s);
}

int dispatch_ax_bulk_batch_f32(sem_handle* h, int lx, const AxParams<float>& a, bool fused, cudaStream_t s) {
    return fused ? dispatch_ax_bulk_batch<float, true>(h, lx, a, s) : dispatch_ax_bulk_batch<float, false>(h, lx, a, s);
}

int bulk_set_d_f32(const float* D, int lx) { return bulk_set_d<float>(D, lx); }

}  // namespace sem
