// Instantiations of the bulk-staged local operator kernels for double data.
#include "sem_ax_bulk.cuh"

namespace sem {

int dispatch_ax_bulk_f64(sem_handle* h, int lx, const AxParams<double>& a, bool fused, cudaStream_t s) {
    return fused ? dispatch_ax_bulk<double, true>(h, lx, a, s) : dispatch_ax_bulk<double, false>(h, lx, a, s);
}

int bulk_set_d_f64(const double* D, int lx) { return bulk_set_d<double>(D, lx); }

}  // namespace sem
