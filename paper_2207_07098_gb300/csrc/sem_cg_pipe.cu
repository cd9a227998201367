// Pipelined Jacobi-PCG (Ghysels and Vanroose 2014), the communication-reduced
// CG that the paper's solver work on reducing communication builds on (Sec.
// II-B): the iterates of PCG in exact arithmetic, with ONE reduction phase
// per iteration -- (r, u), (w, u) and (r, r) together -- that a distributed
// solve overlaps with the operator application n = A m.
//
// Per iteration (three launches, captured in graphs like the standard loop):
//   operator   n = mask QQ^T A_L m          (skipped once the solve is done)
//   gather-scatter on n
//   update     beta = gamma / gamma_prev,
//              alpha = gamma / (delta - beta gamma / alpha_prev)
//              z = n + beta z;  q = m + beta q;  s = w + beta s;  p = u + beta p
//              x += alpha p;  r -= alpha s;  u -= alpha q;  w -= alpha z;  m = Minv w
//              and the next gamma = (r, u), delta = (w, u), rr = (r, r)
// with u = Minv r, w = A u and m = Minv w kept as recurrences.  On one GPU the
// reductions already sit inside the kernels, so the pipelined form only adds
// vector traffic (20 vector accesses per point in the update against 8); it
// exists for parity with the paper's solver family and as the single-exchange
// form a multi-GPU build would overlap.  FP64 data, native FP64 operator.
// The solve runs in segments with residual replacement between them
// (launch_pipe_replace; the loop is in sem_cg.cu).
#include <algorithm>
#include <cmath>

#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

struct PipeVecs {
    double *x, *r, *u, *w, *m, *n, *z, *q, *s, *p;
    const double* minv;
    const double* b;
    const uint8_t* mult;
    int64_t nn;
    CGState* st;
    double* partials;
    unsigned int* counter;
};

// scalars of the pipelined recurrence in a CGState: rho = gamma, rho_old =
// gamma of the previous iteration, pap = delta, alpha = alpha of the previous
// iteration, scale = the delta of the first iteration (unused afterwards)

// start: u = Minv r, then (after w = A u) m = Minv w, gamma, delta, rr, bb
__global__ void pipe_u_kernel(const double* __restrict__ r, const double* __restrict__ minv, double* __restrict__ u,
                              int64_t n) {
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x)
        u[L] = minv[L] * r[L];
}

__global__ void __launch_bounds__(256) pipe_init_kernel(PipeVecs v, double tol, int max_iter) {
    __shared__ double inv[256];
    for (int m = threadIdx.x; m < 256; m += blockDim.x) inv[m] = m ? 1.0 / m : 0.0;
    __syncthreads();
    double acc4[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < v.nn; L += (int64_t)gridDim.x * blockDim.x) {
        const double rv = v.r[L], uv = v.u[L], wv = v.w[L], bv = v.b[L], iv = inv[v.mult[L]];
        v.m[L] = v.minv[L] * wv;
        v.z[L] = 0.0;
        v.q[L] = 0.0;
        v.s[L] = 0.0;
        v.p[L] = 0.0;
        acc4[0] = fma(rv * uv, iv, acc4[0]);
        acc4[1] = fma(wv * uv, iv, acc4[1]);
        acc4[2] = fma(rv * rv, iv, acc4[2]);
        acc4[3] = fma(bv * bv, iv, acc4[3]);
    }
    CGState* st = v.st;
    grid_sum_finalize<4>(acc4, v.partials, v.counter, [&](double (&a)[4]) {
        st->rho = a[0];
        st->pap = a[1];
        st->rr = a[2];
        st->bb = a[3];
        st->rho_old = 0.0;
        st->alpha = 0.0;
        st->tol2 = tol * tol * a[3];
        st->iter = 0;
        st->max_iter = max_iter;
        st->carry = 0;
        const bool conv = (a[3] == 0.0 || a[2] <= st->tol2);
        st->done = (conv || max_iter <= 0) ? 1 : 0;
        st->status = (conv || max_iter > 0) ? SEM_OK : SEM_ENOTCONV;
        if (!conv && (!isfinite(a[0]) || !isfinite(a[1]) || !isfinite(a[2]))) {
            st->done = 1;
            st->status = SEM_EBREAKDOWN;
        }
    });
}

__global__ void __launch_bounds__(256) pipe_update_kernel(PipeVecs v) {
    if (v.st->done) return;
    __shared__ double inv[256];
    __shared__ double s_ab[2];
    __shared__ int s_bad;
    for (int m = threadIdx.x; m < 256; m += blockDim.x) inv[m] = m ? 1.0 / m : 0.0;
    if (threadIdx.x == 0) {
        const CGState* st = v.st;
        double alpha, beta;
        if (st->iter == 0) {
            beta = 0.0;
            alpha = st->rho / st->pap;
        } else {
            beta = st->rho / st->rho_old;
            alpha = st->rho / (st->pap - beta * st->rho / st->alpha);
        }
        s_ab[0] = alpha;
        s_ab[1] = beta;
        s_bad = (!(alpha > 0.0) || !isfinite(alpha) || !isfinite(beta)) ? 1 : 0;
    }
    __syncthreads();
    const double alpha = s_ab[0], beta = s_ab[1];
    double acc3[3] = {0.0, 0.0, 0.0};
    if (!s_bad) {
        for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < v.nn;
             L += (int64_t)gridDim.x * blockDim.x) {
            const double zv = fma(beta, v.z[L], v.n[L]);
            const double qv = fma(beta, v.q[L], v.m[L]);
            const double wv0 = v.w[L];
            const double sv = fma(beta, v.s[L], wv0);
            const double pv = fma(beta, v.p[L], v.u[L]);
            const double xv = fma(alpha, pv, v.x[L]);
            const double rv = fma(-alpha, sv, v.r[L]);
            const double uv = fma(-alpha, qv, v.u[L]);
            const double wv = fma(-alpha, zv, wv0);
            v.z[L] = zv;
            v.q[L] = qv;
            v.s[L] = sv;
            v.p[L] = pv;
            v.x[L] = xv;
            v.r[L] = rv;
            v.u[L] = uv;
            v.w[L] = wv;
            v.m[L] = v.minv[L] * wv;
            const double iv = inv[v.mult[L]];
            acc3[0] = fma(rv * uv, iv, acc3[0]);
            acc3[1] = fma(wv * uv, iv, acc3[1]);
            acc3[2] = fma(rv * rv, iv, acc3[2]);
        }
    }
    CGState* st = v.st;
    const int bad = s_bad;
    grid_sum_finalize<3>(acc3, v.partials, v.counter, [&](double (&a)[3]) {
        if (bad) {
            st->done = 1;
            st->status = SEM_EBREAKDOWN;
            return;
        }
        st->rho_old = st->rho;
        st->alpha = alpha;
        st->rho = a[0];
        st->pap = a[1];
        st->rr = a[2];
        st->iter += 1;
        if (!isfinite(a[0]) || !isfinite(a[1]) || !isfinite(a[2])) {
            st->done = 1;
            st->status = SEM_EBREAKDOWN;
        } else if (a[2] <= st->tol2) {
            st->done = 1;
            st->status = SEM_OK;
        } else if (st->iter >= st->max_iter) {
            st->done = 1;
            st->status = SEM_ENOTCONV;
        }
    });
}

// residual replacement, last step: m = Minv w and the reductions gamma = <r, u>,
// delta = <w, u>, rr = <r, r> of the recomputed vectors; the scalars of the
// previous iteration (gamma_prev, alpha_prev) stay, so the next update
// continues the recurrence with the kept direction; seg more iterations
__global__ void __launch_bounds__(256) pipe_replace_kernel(PipeVecs v, int seg) {
    __shared__ double inv[256];
    for (int m = threadIdx.x; m < 256; m += blockDim.x) inv[m] = m ? 1.0 / m : 0.0;
    __syncthreads();
    double acc3[3] = {0.0, 0.0, 0.0};
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < v.nn; L += (int64_t)gridDim.x * blockDim.x) {
        const double rv = v.r[L], uv = v.u[L], wv = v.w[L], iv = inv[v.mult[L]];
        v.m[L] = v.minv[L] * wv;
        acc3[0] = fma(rv * uv, iv, acc3[0]);
        acc3[1] = fma(wv * uv, iv, acc3[1]);
        acc3[2] = fma(rv * rv, iv, acc3[2]);
    }
    CGState* st = v.st;
    grid_sum_finalize<3>(acc3, v.partials, v.counter, [&](double (&a)[3]) {
        st->rho = a[0];
        st->pap = a[1];
        st->rr = a[2];
        st->max_iter = st->iter + seg;
        const bool conv = a[2] <= st->tol2;
        st->done = (conv || seg <= 0) ? 1 : 0;
        st->status = SEM_OK;
        if (!conv && (!isfinite(a[0]) || !isfinite(a[1]) || !isfinite(a[2]))) {
            st->done = 1;
            st->status = SEM_EBREAKDOWN;
        }
    });
}

static PipeVecs pipe_vecs(sem_handle* h) {
    double** v = h->ws.pipe;
    return PipeVecs{h->ws.x, h->ws.r, v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7],
                    h->minv64, h->ws.b, h->mult, h->n_local, h->state, h->partials, h->counters + 6};
}

int ensure_pipe_workspace(sem_handle* h) {
    if (h->ws.pipe[0]) return SEM_OK;
    for (int q = 0; q < 8; q++) {
        int rc = dalloc(h, &h->ws.pipe[q], (size_t)h->n_local);
        if (rc) return rc;
    }
    return SEM_OK;
}

// start from ws.r = b - A x (the true residual): u = Minv r, w = A u, the rest
int launch_pipe_init(sem_handle* h, double tol, int max_iter, cudaStream_t s) {
    PipeVecs v = pipe_vecs(h);
    pipe_u_kernel<<<grid_for(h, h->n_local, 256, 8), 256, 0, s>>>(v.r, v.minv, v.u, v.nn);
    SEM_LAUNCH_CHECK("pipe_u_kernel");
    h->launches++;
    int rc = launch_ax_local(h, v.u, v.w, SEM_FP64, s);
    if (!rc) rc = launch_gs(h, v.w, false, true, s);
    if (rc) return rc;
    pipe_init_kernel<<<grid_for(h, h->n_local, 256, 4), 256, 0, s>>>(v, tol, max_iter);
    SEM_LAUNCH_CHECK("pipe_init_kernel");
    h->launches++;
    return SEM_OK;
}

// residual replacement (ws.r = b - A x already computed): u = Minv r, w = A u,
// s = A p, q = Minv s, z = A q, m = Minv w, the reductions, seg more iterations
int launch_pipe_replace(sem_handle* h, int seg, cudaStream_t s) {
    PipeVecs v = pipe_vecs(h);
    const int grid = grid_for(h, h->n_local, 256, 8);
    pipe_u_kernel<<<grid, 256, 0, s>>>(v.r, v.minv, v.u, v.nn);
    SEM_LAUNCH_CHECK("pipe_u_kernel");
    h->launches++;
    int rc = launch_ax_local(h, v.u, v.w, SEM_FP64, s);
    if (!rc) rc = launch_gs(h, v.w, false, true, s);
    if (!rc) rc = launch_ax_local(h, v.p, v.s, SEM_FP64, s);
    if (!rc) rc = launch_gs(h, v.s, false, true, s);
    if (rc) return rc;
    pipe_u_kernel<<<grid, 256, 0, s>>>(v.s, v.minv, v.q, v.nn);
    SEM_LAUNCH_CHECK("pipe_u_kernel");
    h->launches++;
    if ((rc = launch_ax_local(h, v.q, v.z, SEM_FP64, s)) || (rc = launch_gs(h, v.z, false, true, s))) return rc;
    pipe_replace_kernel<<<grid_for(h, h->n_local, 256, 4), 256, 0, s>>>(v, seg);
    SEM_LAUNCH_CHECK("pipe_replace_kernel");
    h->launches++;
    return SEM_OK;
}

// one pipelined iteration: n = A m (operator skipped once done), QQ^T, update
int launch_pipe_iteration(sem_handle* h, cudaStream_t s) {
    PipeVecs v = pipe_vecs(h);
    int rc = launch_ax_local_until_done(h, v.m, v.n, h->state, s);
    if (!rc) rc = launch_gs(h, v.n, false, true, s);
    if (rc) return rc;
    pipe_update_kernel<<<grid_for(h, h->n_local, 256, 4), 256, 0, s>>>(v);
    SEM_LAUNCH_CHECK("pipe_update_kernel");
    h->launches++;
    return SEM_OK;
}

}  // namespace sem
