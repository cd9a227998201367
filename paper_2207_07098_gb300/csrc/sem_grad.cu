// Gradient, divergence and curl of nodal fields by collocation, and the
// right-hand side of the pressure equation (Sec. II-A: the nodal GLL basis,
// the derivative matrix D, and eq. "pressure",
//   -lap p = -div(vhat) / dt + (1/Re) div(curl(omega)),
// whose weak right-hand side is b = mask QQ^T (B f) with f the point values of
// the right side, B the diagonal GLL mass).
//
// Derivatives in the reference coordinates come from D along each direction,
// (du/dr, du/ds, du/dt)_ijk = (sum_l D_il u_ljk, sum_l D_jl u_ilk, sum_l D_kl u_ijl)
// (indices as [k][j][i]), and become physical derivatives through the metric
// terms dr_s/dx_l that sem_setup keeps with SEM_FLAG_METRICS:
//   du/dx_l = sum_s (dr_s/dx_l) du/dr_s.
// All results are local (element by element): the derivative of a continuous
// field jumps across element faces.  These run once per time step, not in the
// solver loop: one thread per point.
#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

struct MetricPart {
    const double* D;     // [lx][lx]
    const double* M;     // [E][9][lx^3] dr_s/dx_l, s major, of this part
    int64_t E;
    int lx;
};

__device__ __forceinline__ void ref_derivs(const double* ue, const double* D, int lx, int i, int j, int k,
                                           double (&d)[3]) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int l = 0; l < lx; l++) {
        a = fma(D[i * lx + l], ue[(k * lx + j) * lx + l], a);
        b = fma(D[j * lx + l], ue[(k * lx + l) * lx + i], b);
        c = fma(D[k * lx + l], ue[(l * lx + j) * lx + i], c);
    }
    d[0] = a;
    d[1] = b;
    d[2] = c;
}

// physical gradient of u at local point L (element e, index q)
__device__ __forceinline__ void phys_grad(const double* u, const MetricPart& m, int64_t e, int q, double (&g)[3]) {
    const int lx = m.lx, n3 = lx * lx * lx;
    const int i = q % lx, j = (q / lx) % lx, k = q / (lx * lx);
    double d[3];
    ref_derivs(u + e * n3, m.D, lx, i, j, k, d);
    const double* Me = m.M + e * 9 * n3 + q;
#pragma unroll
    for (int l = 0; l < 3; l++)
        g[l] = fma(Me[(0 * 3 + l) * n3], d[0], fma(Me[(1 * 3 + l) * n3], d[1], Me[(2 * 3 + l) * n3] * d[2]));
}

__global__ void grad_kernel(const double* __restrict__ u, MetricPart m, double* gx, double* gy, double* gz) {
    const int n3 = m.lx * m.lx * m.lx;
    const int64_t n = m.E * n3;
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = L / n3;
        double g[3];
        phys_grad(u, m, e, (int)(L - e * n3), g);
        gx[L] = g[0];
        gy[L] = g[1];
        gz[L] = g[2];
    }
}

// out = cv * div(v)  (+ cw * div(w) when w0 is given)
__global__ void div_kernel(const double* v0, const double* v1, const double* v2, double cv, const double* w0,
                           const double* w1, const double* w2, double cw, const double* B, MetricPart m,
                           double* out) {
    const int n3 = m.lx * m.lx * m.lx;
    const int64_t n = m.E * n3;
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = L / n3;
        const int q = (int)(L - e * n3);
        double g0[3], g1[3], g2[3];
        phys_grad(v0, m, e, q, g0);
        phys_grad(v1, m, e, q, g1);
        phys_grad(v2, m, e, q, g2);
        double f = cv * (g0[0] + g1[1] + g2[2]);
        if (w0) {
            phys_grad(w0, m, e, q, g0);
            phys_grad(w1, m, e, q, g1);
            phys_grad(w2, m, e, q, g2);
            f = fma(cw, g0[0] + g1[1] + g2[2], f);
        }
        out[L] = B ? B[L] * f : f;
    }
}

__global__ void curl_kernel(const double* v0, const double* v1, const double* v2, MetricPart m, double* c0,
                            double* c1, double* c2) {
    const int n3 = m.lx * m.lx * m.lx;
    const int64_t n = m.E * n3;
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = L / n3;
        const int q = (int)(L - e * n3);
        double g0[3], g1[3], g2[3];
        phys_grad(v0, m, e, q, g0);
        phys_grad(v1, m, e, q, g1);
        phys_grad(v2, m, e, q, g2);
        c0[L] = g2[1] - g1[2];
        c1[L] = g0[2] - g2[0];
        c2[L] = g1[0] - g0[1];
    }
}

static MetricPart metric_part(const sem_handle* h, const MeshPart& p) {
    return MetricPart{h->D64[p.lx], h->drdx + 9 * p.loc_off, p.E, p.lx};
}

static int need_metrics(const sem_handle* h) {
    return h->drdx ? SEM_OK : fail(SEM_EINVAL, "the handle keeps no metric terms: set it up with SEM_FLAG_METRICS");
}

}  // namespace sem

using namespace sem;

extern "C" {

SEM_API int sem_grad(sem_handle* h, const double* u, double* gx, double* gy, double* gz, cudaStream_t s) {
    if (!h || !u || !gx || !gy || !gz) return fail(SEM_EINVAL, "null argument");
    int rc = need_metrics(h);
    if (rc) return rc;
    for (const MeshPart& p : h->parts) {
        const int64_t o = p.loc_off;
        grad_kernel<<<grid_for(h, p.n_local, 256, 8), 256, 0, s>>>(u + o, metric_part(h, p), gx + o, gy + o, gz + o);
        SEM_LAUNCH_CHECK("grad_kernel");
        h->launches++;
    }
    return SEM_OK;
}

SEM_API int sem_div(sem_handle* h, const double* vx, const double* vy, const double* vz, double* out,
                    cudaStream_t s) {
    if (!h || !vx || !vy || !vz || !out) return fail(SEM_EINVAL, "null argument");
    int rc = need_metrics(h);
    if (rc) return rc;
    for (const MeshPart& p : h->parts) {
        const int64_t o = p.loc_off;
        div_kernel<<<grid_for(h, p.n_local, 256, 8), 256, 0, s>>>(vx + o, vy + o, vz + o, 1.0, nullptr, nullptr,
                                                                 nullptr, 0.0, nullptr, metric_part(h, p), out + o);
        SEM_LAUNCH_CHECK("div_kernel");
        h->launches++;
    }
    return SEM_OK;
}

SEM_API int sem_curl(sem_handle* h, const double* vx, const double* vy, const double* vz, double* cx, double* cy,
                     double* cz, cudaStream_t s) {
    if (!h || !vx || !vy || !vz || !cx || !cy || !cz) return fail(SEM_EINVAL, "null argument");
    if (cx == vx || cx == vy || cx == vz || cy == vx || cy == vy || cy == vz || cz == vx || cz == vy || cz == vz)
        return fail(SEM_EINVAL, "the curl must not overwrite its input");
    int rc = need_metrics(h);
    if (rc) return rc;
    for (const MeshPart& p : h->parts) {
        const int64_t o = p.loc_off;
        curl_kernel<<<grid_for(h, p.n_local, 256, 8), 256, 0, s>>>(vx + o, vy + o, vz + o, metric_part(h, p), cx + o,
                                                                  cy + o, cz + o);
        SEM_LAUNCH_CHECK("curl_kernel");
        h->launches++;
    }
    return SEM_OK;
}

SEM_API int sem_pressure_rhs(sem_handle* h, const double* vx, const double* vy, const double* vz,
                             const double* wx, const double* wy, const double* wz, double dt, double Re, double* b,
                             cudaStream_t s) {
    if (!h || !vx || !vy || !vz || !b) return fail(SEM_EINVAL, "null argument");
    if ((wx || wy || wz) && !(wx && wy && wz)) return fail(SEM_EINVAL, "omega needs all three components");
    if (!(dt > 0.0) || !(Re > 0.0)) return fail(SEM_EINVAL, "dt and Re must be positive");
    int rc = need_metrics(h);
    if (!rc) rc = ensure_workspace(h, false);
    if (rc) return rc;
    // curl(omega) into the work vectors p, z, r (free between solves)
    double* c0 = h->ws.p;
    double* c1 = h->ws.z;
    double* c2 = h->ws.r;
    for (const MeshPart& p : h->parts) {
        const int64_t o = p.loc_off;
        if (wx) {
            curl_kernel<<<grid_for(h, p.n_local, 256, 8), 256, 0, s>>>(wx + o, wy + o, wz + o, metric_part(h, p),
                                                                      c0 + o, c1 + o, c2 + o);
            SEM_LAUNCH_CHECK("curl_kernel");
            h->launches++;
        }
        div_kernel<<<grid_for(h, p.n_local, 256, 8), 256, 0, s>>>(
            vx + o, vy + o, vz + o, -1.0 / dt, wx ? c0 + o : nullptr, wx ? c1 + o : nullptr, wx ? c2 + o : nullptr,
            1.0 / Re, h->B64 + o, metric_part(h, p), b + o);
        SEM_LAUNCH_CHECK("div_kernel");
        h->launches++;
    }
    return launch_gs(h, b, false, true, s);
}

}  // extern "C"
