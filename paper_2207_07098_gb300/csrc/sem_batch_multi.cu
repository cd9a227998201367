// Instantiations and launch of the multi-order batched operator kernel (one
// launch over the element groups of every order of a batch).
#include "sem_batch.cuh"

namespace sem {

template <typename T, bool FUSED>
static int launch_multi_t(sem_handle* h, const BatchAxParams<T>& a, const MultiOrder<T>& mo, size_t smem,
                          cudaStream_t s) {
    static size_t attr_smem = 0;  // dynamic shared memory the kernel was opened to
    static int per_sm = 0;
    if (smem > attr_smem) {
        cudaError_t e = cudaFuncSetAttribute(ax_batch_multi_kernel<T, FUSED>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(ax_batch_multi_kernel)");
        attr_smem = smem;
        per_sm = 0;
    }
    if (per_sm == 0) {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ax_batch_multi_kernel<T, FUSED>, kMultiThreads, smem);
        per_sm = nb > 0 ? nb : 1;
    }
    if (a.dry || a.ngroups == 0) return SEM_OK;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(a.ngroups, (int64_t)h->sm_count * per_sm));
    ax_batch_multi_kernel<T, FUSED><<<(int)grid, kMultiThreads, smem, s>>>(a, mo);
    SEM_LAUNCH_CHECK("ax_batch_multi_kernel");
    h->launches++;
    return SEM_OK;
}

int launch_ax_batch_multi_f64(sem_handle* h, const BatchAxParams<double>& a, const MultiOrder<double>& mo,
                              size_t smem, bool fused, cudaStream_t s) {
    return fused ? launch_multi_t<double, true>(h, a, mo, smem, s) : launch_multi_t<double, false>(h, a, mo, smem, s);
}

int launch_ax_batch_multi_f32(sem_handle* h, const BatchAxParams<float>& a, const MultiOrder<float>& mo,
                              size_t smem, bool fused, cudaStream_t s) {
    return fused ? launch_multi_t<float, true>(h, a, mo, smem, s) : launch_multi_t<float, false>(h, a, mo, smem, s);
}

}  // namespace sem
