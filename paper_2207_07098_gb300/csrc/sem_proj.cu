// Projection onto previous solutions (Sec. II-B of Karp et al., after Fischer
// 1998): the pressure and velocity solves of successive time steps start from
// the A-orthogonal projection of the new solution onto the space spanned by
// earlier solution increments, which cuts the start residual and the
// iterations when the right-hand sides change slowly.
//
// The handle keeps up to L vectors xt_i, A-orthonormal in the unique-node
// inner product <a, b> = sum_L a_L b_L / mult_L, and bt_i = A xt_i (FP64).
//   start:  alpha_i = <xt_i, b>,  x0 = xbar = sum_i alpha_i xt_i
//   update: v = x - xbar, classical Gram-Schmidt twice against the space in
//           the A inner product (<bt_i, v> = xt_i^T A v), w = A v, then
//           xt = v / ||v||_A, bt = w / ||v||_A appended.
// When the space is full it restarts from the latest solution: it is cleared
// and x itself (A-normalised) becomes its first vector (the paper's GPU runs
// reset their space every 20 solves).  Every coefficient stays in
// device memory; the host reads two small arrays per update to decide
// whether the new direction is independent of the space.
#include <cmath>
#include <vector>

#include "sem_krylov.cuh"

namespace sem {

// dx = v / sqrt(nn), db = w / sqrt(nn)
__global__ void proj_normalise_kernel(const double* __restrict__ v, const double* __restrict__ w,
                                      double* __restrict__ dx, double* __restrict__ db, const double* nn,
                                      int64_t n) {
    const double s = 1.0 / sqrt(*nn);
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x) {
        dx[L] = v[L] * s;
        db[L] = w[L] * s;
    }
}

__global__ void proj_diff_kernel(double* __restrict__ v, const double* __restrict__ x,
                                 const double* __restrict__ xbar, int64_t n) {
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x)
        v[L] = x[L] - xbar[L];
}

static int ensure_space(sem_handle* h, int L) {
    ProjSpace& ps = h->proj;
    if (ps.L == L && ps.xt) return SEM_OK;
    free_projection(h);
    const size_t n = (size_t)h->n_local, ld = (n + 3) & ~(size_t)3;
    int rc = dalloc(h, &ps.xt, (size_t)L * ld);
    if (!rc) rc = dalloc(h, &ps.bt, (size_t)L * ld);
    if (!rc) rc = dalloc(h, &ps.xbar, n);
    if (!rc) rc = dalloc(h, &ps.coef, (size_t)L + 2);
    if (!rc) rc = dalloc(h, &ps.gpart, (size_t)(kGmNV + 1) * kMaxPartials);
    if (!rc && cudaMalloc(&ps.gcount, sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        ps.gcount = nullptr;
        rc = fail(SEM_ENOMEM, "cudaMalloc of the projection counter failed");
    }
    if (!rc && cudaMemset(ps.gcount, 0, sizeof(unsigned int)) != cudaSuccess) rc = fail(SEM_ECUDA, "cudaMemset");
    if (rc) {
        free_projection(h);
        return rc;
    }
    ps.L = L;
    ps.l = 0;
    ps.ld = (int64_t)ld;
    return SEM_OK;
}

void free_projection(sem_handle* h) {
    ProjSpace& ps = h->proj;
    const size_t n = (size_t)h->n_local;
    if (ps.xt)
        h->device_bytes -= sizeof(double) * ((size_t)2 * ps.L * (size_t)ps.ld + n + ps.L + 2 +
                                             (size_t)(kGmNV + 1) * kMaxPartials);
    cudaFree(ps.xt);
    cudaFree(ps.bt);
    cudaFree(ps.xbar);
    cudaFree(ps.coef);
    cudaFree(ps.gpart);
    cudaFree(ps.gcount);
    ps = ProjSpace{};
}

// x0 = xbar = sum_i <xt_i, b> xt_i into ws.x (and kept in the space's xbar)
int proj_start(sem_handle* h, int L, cudaStream_t s) {
    int rc = ensure_space(h, L);
    if (rc) return rc;
    ProjSpace& ps = h->proj;
    const int64_t n = h->n_local;
    SEM_CUDA_TRY(cudaMemsetAsync(h->ws.x, 0, sizeof(double) * n, s));
    if (ps.l > 0 &&
        ((rc = krylov_pass<double>(h, h->ws.b, ps.xt, ps.ld, 0, nullptr, ps.l, ps.coef, nullptr, ps.gpart,
                                   ps.gcount, s)) ||
         (rc = krylov_update<double>(h, h->ws.x, ps.xt, ps.ld, ps.coef, ps.l, s))))
        return rc;
    SEM_CUDA_TRY(cudaMemcpyAsync(ps.xbar, h->ws.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    return SEM_OK;
}

// Append the increment ws.x - xbar of the solve that just ended (uses ws.p,
// ws.w as scratch).  A full space restarts from the solution ws.x instead.
int proj_update(sem_handle* h, cudaStream_t s) {
    ProjSpace& ps = h->proj;
    if (!ps.xt) return SEM_OK;
    const int64_t n = h->n_local;
    double* v = h->ws.p;
    double* w = h->ws.w;
    if (ps.l >= ps.L) {
        ps.l = 0;
        SEM_CUDA_TRY(cudaMemcpyAsync(v, h->ws.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    } else {
        proj_diff_kernel<<<grid_for(h, n, 256, 8), 256, 0, s>>>(v, h->ws.x, ps.xbar, n);
        SEM_LAUNCH_CHECK("proj_diff_kernel");
        h->launches++;
    }
    double gsum = 0.0;
    std::vector<double> g((size_t)ps.L + 2);
    int rc;
    // classical Gram-Schmidt twice in the A inner product: g = bt^T v, v -= xt g
    for (int pass = 0; pass < 2 && ps.l > 0; pass++) {
        if ((rc = krylov_pass<double>(h, v, ps.bt, ps.ld, 0, nullptr, ps.l, ps.coef, nullptr, ps.gpart, ps.gcount,
                                      s)) ||
            (rc = krylov_pass<double>(h, v, ps.xt, ps.ld, ps.l, ps.coef, 0, nullptr, nullptr, ps.gpart, ps.gcount,
                                      s)))
            return rc;
        SEM_CUDA_TRY(cudaMemcpyAsync(g.data(), ps.coef, sizeof(double) * ps.l, cudaMemcpyDeviceToHost, s));
        SEM_CUDA_TRY(cudaStreamSynchronize(s));
        for (int i = 0; i < ps.l; i++) gsum += g[i] * g[i];
    }
    if ((rc = launch_ax_local(h, v, w, SEM_FP64, s)) || (rc = launch_gs(h, w, false, true, s)) ||
        (rc = launch_dot(h, v, w, ps.coef + ps.L, s)))
        return rc;
    double nn = 0.0;
    SEM_CUDA_TRY(cudaMemcpyAsync(&nn, ps.coef + ps.L, sizeof(double), cudaMemcpyDeviceToHost, s));
    SEM_CUDA_TRY(cudaStreamSynchronize(s));
    // a direction inside the span (numerically) is not appended
    if (!(nn > 1e-20 * (gsum + nn)) || !std::isfinite(nn)) return SEM_OK;
    proj_normalise_kernel<<<grid_for(h, n, 256, 8), 256, 0, s>>>(v, w, ps.xt + (int64_t)ps.l * ps.ld,
                                                                 ps.bt + (int64_t)ps.l * ps.ld, ps.coef + ps.L, n);
    SEM_LAUNCH_CHECK("proj_normalise_kernel");
    h->launches++;
    ps.l++;
    return SEM_OK;
}

}  // namespace sem

using namespace sem;

extern "C" {

SEM_API int sem_projection_reset(sem_handle* h) {
    if (!h) return fail(SEM_EINVAL, "null handle");
    h->proj.l = 0;
    return SEM_OK;
}

SEM_API int sem_projection_size(const sem_handle* h, int* count) {
    if (!h || !count) return fail(SEM_EINVAL, "null argument");
    *count = h->proj.l;
    return SEM_OK;
}

}  // extern "C"
