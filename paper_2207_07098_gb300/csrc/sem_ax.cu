// Matrix-free local operator w = A_L u with A^e = D^T (h1 G^e) D
// (Sec. II-A of Karp et al., eq. "disclap"), in FP64 and FP32, plus the CG
// variant that fuses the search-direction update p = z + beta p and the
// partial sums of <p, A p> into the same pass (Sec. II-B, P-CG).
//
// Thread layout: a CTA owns EPC elements; each element is handled by lx^2
// threads, thread (i, j) owning the column u[:, j, i] in registers.  The
// element block u[k][j][i] is staged in shared memory; r- and s-derivatives
// read it from there, the t-derivative comes from the register column.  The
// six factors G are streamed once per point (coalesced along i), the
// weighted derivatives wr, ws go back to shared memory and the transposed
// contraction produces w.
#include "sem_ax.cuh"

namespace sem {

int launch_ax_local(sem_handle* h, const void* u, void* w, int precision, cudaStream_t s) {
    for (int q = 0; q < h->nsolve; q++) {
        const MeshPart& p = h->parts[q];
        int rc;
        if (precision == SEM_FP32) {
            AxParams<float> a = {};
            a.u = (const float*)u + p.loc_off;
            a.w = (float*)w + p.loc_off;
            a.G = h->G32 + 6 * p.loc_off;
            a.D = h->D32[p.lx];
            a.E = p.E;
            rc = dispatch_ax_f32(h, p.lx, a, false, s);
        } else {
            AxParams<double> a = {};
            a.u = (const double*)u + p.loc_off;
            a.w = (double*)w + p.loc_off;
            a.G = h->G64 + 6 * p.loc_off;
            a.D = h->D64[p.lx];
            a.E = p.E;
            rc = dispatch_ax_f64(h, p.lx, a, false, s);
        }
        if (rc) return rc;
    }
    return SEM_OK;
}

// K-A of a CG iteration on a single-mesh handle: p = z + beta p; w = A_L p;
// alpha = rho / <p, w>.
int launch_cg_pupdate_ax(sem_handle* h, int precision, cudaStream_t s) {
    const MeshPart& p = h->parts[0];
    if (precision == SEM_FP32) {
        AxParams<float> a = {};
        a.w = h->ws.w32;
        a.G = h->G32;
        a.D = h->D32[p.lx];
        a.E = p.E;
        a.z = h->ws.z32;
        a.p = h->ws.p32;
        a.st = h->state + 1;
        a.partials = h->partials;
        a.counter = h->counters + 2;
        return dispatch_ax_f32(h, p.lx, a, true, s);
    }
    AxParams<double> a = {};
    a.w = h->ws.w;
    a.G = h->G64;
    a.D = h->D64[p.lx];
    a.E = p.E;
    a.z = h->ws.z;
    a.p = h->ws.p;
    a.st = h->state;
    a.partials = h->partials;
    a.counter = h->counters + 2;
    return dispatch_ax_f64(h, p.lx, a, true, s);
}

// Set kernel attributes and cache occupancies of the CG kernels of this
// handle before any stream capture (those calls are kept out of captures).
int prepare_cg_kernels(sem_handle* h) {
    for (const MeshPart& p : h->parts) {
        AxParams<double> a = {};
        a.dry = 1;
        AxParams<float> b = {};
        b.dry = 1;
        int rc = dispatch_ax_f64(h, p.lx, a, true, 0);
        if (!rc) rc = dispatch_ax_f64(h, p.lx, a, false, 0);
        if (!rc) rc = dispatch_ax_f32(h, p.lx, b, true, 0);
        if (!rc) rc = dispatch_ax_f32(h, p.lx, b, false, 0);
        if (rc) return rc;
    }
    return SEM_OK;
}

// w = B u
template <typename T>
__global__ void mass_kernel(const T* __restrict__ u, const double* __restrict__ B, T* __restrict__ w, int64_t n) {
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x)
        w[L] = (T)(B[L] * (double)u[L]);
}

int launch_mass(sem_handle* h, const double* u, double* w, cudaStream_t s) {
    mass_kernel<double><<<grid_for(h, h->n_local, 256, 8), 256, 0, s>>>(u, h->B64, w, h->n_local);
    SEM_LAUNCH_CHECK("mass_kernel");
    h->launches++;
    return SEM_OK;
}

int launch_mass32(sem_handle* h, const float* u, float* w, cudaStream_t s) {
    mass_kernel<float><<<grid_for(h, h->n_local, 256, 8), 256, 0, s>>>(u, h->B64, w, h->n_local);
    SEM_LAUNCH_CHECK("mass_kernel");
    h->launches++;
    return SEM_OK;
}

}  // namespace sem

using namespace sem;

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

extern "C" {

SEM_API int sem_ax(sem_handle* h, void* w, const void* u, int precision, int assemble, cudaStream_t s) {
    if (!h || !w || !u) return fail(SEM_EINVAL, "null argument");
    if (precision != SEM_FP64 && precision != SEM_FP32 && precision != SEM_FP64_NATIVE)
        return fail(SEM_EINVAL, "unknown precision");
    if (w == u) return fail(SEM_EINVAL, "w must not alias u");
    if (!aligned16(w) || !aligned16(u)) return fail(SEM_EINVAL, "u and w must be 16-byte aligned");
    int rc = launch_ax_local(h, u, w, precision, s);
    if (rc == SEM_OK && assemble) rc = launch_gs(h, w, precision == SEM_FP32, true, s);
    return rc;
}

SEM_API int sem_mass(sem_handle* h, void* w, const void* u, int precision, int assemble, cudaStream_t s) {
    if (!h || !w || !u) return fail(SEM_EINVAL, "null argument");
    int rc;
    if (precision == SEM_FP32)
        rc = launch_mass32(h, (const float*)u, (float*)w, s);
    else if (precision == SEM_FP64 || precision == SEM_FP64_NATIVE)
        rc = launch_mass(h, (const double*)u, (double*)w, s);
    else
        return fail(SEM_EINVAL, "unknown precision");
    if (rc == SEM_OK && assemble) rc = launch_gs(h, w, precision == SEM_FP32, true, s);
    return rc;
}

}  // extern "C"
