// Instantiations of the FP32-pair (FP64-accurate) local operator kernels.
#include "sem_ax_df.cuh"

namespace sem {

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
