// Gather-scatter QQ^T with the Dirichlet mask, and the weighted inner
// product over unique nodes (Sec. II-A of Karp et al.).
//
// QQ^T is deterministic and atomic-free: every node with several local copies
// is one segment whose copies are listed in ascending local index; one thread
// sums the segment in that order and writes the sum back to every copy.
#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

template <typename T>
__global__ void __launch_bounds__(256) gs_kernel(T* __restrict__ u, const int* __restrict__ seg_off,
                                                 const int* __restrict__ seg_idx, int64_t nseg_free,
                                                 int64_t nseg, const int* __restrict__ zero_idx,
                                                 int64_t nzero, int apply_mask) {
    const int64_t total = nseg + (apply_mask ? nzero : 0);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < nseg) {
            const int a = seg_off[t], b = seg_off[t + 1];
            if (apply_mask && t >= nseg_free) {
                for (int c = a; c < b; c++) u[seg_idx[c]] = T(0);
            } else {
                T s = u[seg_idx[a]];
                for (int c = a + 1; c < b; c++) s += u[seg_idx[c]];
                for (int c = a; c < b; c++) u[seg_idx[c]] = s;
            }
        } else {
            u[zero_idx[t - nseg]] = T(0);
        }
    }
}

int launch_gs(sem_handle* h, void* u, bool fp32, bool apply_mask, cudaStream_t s) {
    const GSLists& g = h->gs;
    const int64_t total = g.nseg + (apply_mask ? g.nzero : 0);
    if (total == 0) return SEM_OK;
    const int grid = grid_for(h, total, 256, 8);
    if (fp32)
        gs_kernel<float><<<grid, 256, 0, s>>>((float*)u, g.seg_off, g.seg_idx, g.nseg_free, g.nseg,
                                              g.zero_idx, g.nzero, apply_mask ? 1 : 0);
    else
        gs_kernel<double><<<grid, 256, 0, s>>>((double*)u, g.seg_off, g.seg_idx, g.nseg_free, g.nseg,
                                               g.zero_idx, g.nzero, apply_mask ? 1 : 0);
    SEM_LAUNCH_CHECK("gs_kernel");
    h->launches++;
    return SEM_OK;
}

// <a, b> = sum_L a_L b_L / mult_L in FP64, fixed-order grid reduction.
__global__ void __launch_bounds__(256) dot_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                                  const uint8_t* __restrict__ mult, int64_t n,
                                                  double* partials, unsigned int* counter, double* out) {
    __shared__ double inv[256];
    for (int m = threadIdx.x; m < 256; m += blockDim.x) inv[m] = m ? 1.0 / m : 0.0;
    __syncthreads();
    double v[1] = {0.0};
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x)
        v[0] = fma(a[L] * b[L], inv[mult[L]], v[0]);
    grid_sum_finalize<1>(v, partials, counter, [&](double (&acc)[1]) { *out = acc[0]; });
}

int launch_dot(sem_handle* h, const double* a, const double* b, double* out, cudaStream_t s) {
    // one reduction per mesh part (a batch handle returns one value per solve)
    for (int q = 0; q < h->nsolve; q++) {
        const MeshPart& p = h->parts[q];
        const int grid = grid_for(h, p.n_local, 256, 4);
        dot_kernel<<<grid, 256, 0, s>>>(a + p.loc_off, b + p.loc_off, h->mult + p.loc_off, p.n_local,
                                        h->partials, h->counters + 1, out + q);
        SEM_LAUNCH_CHECK("dot_kernel");
        h->launches++;
    }
    return SEM_OK;
}

}  // namespace sem

using namespace sem;

extern "C" {

SEM_API int sem_gs(sem_handle* h, void* u, int precision, int apply_mask, cudaStream_t s) {
    if (!h || !u) return fail(SEM_EINVAL, "null argument");
    if (precision != SEM_FP64 && precision != SEM_FP32 && precision != SEM_FP64_NATIVE)
        return fail(SEM_EINVAL, "unknown precision");
    return launch_gs(h, u, precision == SEM_FP32, apply_mask != 0, s);
}

SEM_API int sem_dot(sem_handle* h, const double* a, const double* b, double* result, cudaStream_t s) {
    if (!h || !a || !b || !result) return fail(SEM_EINVAL, "null argument");
    return launch_dot(h, a, b, result, s);
}

}  // extern "C"
