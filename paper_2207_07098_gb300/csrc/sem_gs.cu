// Gather-scatter QQ^T with the Dirichlet mask, and the weighted inner
// product over unique nodes (Sec. II-A of Karp et al.).
//
// QQ^T is deterministic and atomic-free: every node with several local copies
// is one segment whose copies are listed in ascending local index; one thread
// sums the segment in that order and writes the sum back to every copy.
// Segments of 2, 4 and 8 copies (faces, edges, vertices of a hex mesh) carry
// their indices as int2 / int4 vectors, so one thread issues its index loads
// and value loads without a dependent offset lookup.
#include <algorithm>

#include "sem_device.cuh"
#include "sem_gs.cuh"
#include "sem_internal.h"

namespace sem {

// One launch covers free segments of 2, 4 and 8 copies (index vectors), free
// segments of other sizes (CSR), and either the zeroing of every Dirichlet copy
// (apply_mask) or the sums over Dirichlet segments.
// CTA ranges of the segment classes of one gather-scatter launch: the
// classes touch disjoint local points, so they run side by side, each CTA on
// one class (a thread walks one chain of dependent loads instead of one per
// class).  b[c] = first CTA after class c.
struct GsRanges {
    int b[6];
};
constexpr int kGsThreads = 256;
constexpr int kGsPairU = 4, kGsQuadU = 4, kGsZeroU = 4;

template <typename T>
__global__ void __launch_bounds__(kGsThreads) gs_kernel(T* __restrict__ u, GSLists g, int apply_mask, GsRanges rg,
                                                        GsSkip sk) {
    if (sk.done_st && sk.done_st->done) return;  // uniform over the grid
    const int b = blockIdx.x;
    int c = 0;
    while (c < 5 && b >= rg.b[c]) c++;
    const int b0 = c ? rg.b[c - 1] : 0;
    const int64_t t0 = (int64_t)(b - b0) * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)(rg.b[c] - b0) * blockDim.x;
    if (c == 0) {
        gs_pairs<T, kGsPairU>(u, g.pairs, g.npair, t0, stride, sk.sid[0], sk.st);
    } else if (c == 1) {
        gs_quads<T, kGsQuadU>(u, g.quads, g.nquad, t0, stride, sk.sid[1], sk.st);
    } else if (c == 2) {
        for (int64_t t = t0; t < g.noct; t += stride) {
            if (seg_done(sk.sid[2], sk.st, t)) continue;
            const int4 q0 = g.octs[2 * t], q1 = g.octs[2 * t + 1];
            const T a0 = u[q0.x], a1 = u[q0.y], a2 = u[q0.z], a3 = u[q0.w];
            const T a4 = u[q1.x], a5 = u[q1.y], a6 = u[q1.z], a7 = u[q1.w];
            const T sum = ((((((a0 + a1) + a2) + a3) + a4) + a5) + a6) + a7;
            u[q0.x] = sum; u[q0.y] = sum; u[q0.z] = sum; u[q0.w] = sum;
            u[q1.x] = sum; u[q1.y] = sum; u[q1.z] = sum; u[q1.w] = sum;
        }
    } else if (c == 3) {
        for (int64_t t = t0; t < g.noth; t += stride) {
            if (seg_done(sk.sid[3], sk.st, t)) continue;
            const int a = g.oth_off[t], e = g.oth_off[t + 1];
            T sum = u[g.oth_idx[a]];
            for (int q = a + 1; q < e; q++) sum += u[g.oth_idx[q]];
            for (int q = a; q < e; q++) u[g.oth_idx[q]] = sum;
        }
    } else if (c == 4) {
        if (apply_mask) {
            for (int64_t t = t0; t < g.nzero; t += stride * kGsZeroU) {
                int q[kGsZeroU];
#pragma unroll
                for (int k = 0; k < kGsZeroU; k++)
                    q[k] = (t + k * stride < g.nzero && !seg_done(sk.sid[4], sk.st, t + k * stride))
                               ? g.zero_idx[t + k * stride]
                               : -1;
#pragma unroll
                for (int k = 0; k < kGsZeroU; k++)
                    if (q[k] >= 0) u[q[k]] = T(0);
            }
        } else {
            for (int64_t t = t0; t < g.ndir; t += stride) {
                const int a = g.dir_off[t], e = g.dir_off[t + 1];
                T sum = u[g.dir_idx[a]];
                for (int q = a + 1; q < e; q++) sum += u[g.dir_idx[q]];
                for (int q = a; q < e; q++) u[g.dir_idx[q]] = sum;
            }
        }
    }
}

static int ctas_for(int64_t items, int per_thread) {
    const int64_t per_cta = (int64_t)kGsThreads * per_thread;
    return (int)std::min<int64_t>((items + per_cta - 1) / per_cta, 1 << 20);
}

static int launch_gs_impl(sem_handle* h, void* u, bool fp32, bool apply_mask, const GsSkip& sk, cudaStream_t s) {
    const GSLists& g = h->gs;
    const int64_t total = g.npair + g.nquad + g.noct + g.noth + (apply_mask ? g.nzero : g.ndir);
    if (total == 0) return SEM_OK;
    const int n[5] = {ctas_for(g.npair, kGsPairU), ctas_for(g.nquad, kGsQuadU), ctas_for(g.noct, 1),
                      ctas_for(g.noth, 1), apply_mask ? ctas_for(g.nzero, kGsZeroU) : ctas_for(g.ndir, 1)};
    GsRanges rg;
    int acc = 0;
    for (int c = 0; c < 5; c++) rg.b[c] = (acc += n[c]);
    rg.b[5] = acc;
    if (fp32)
        gs_kernel<float><<<acc, kGsThreads, 0, s>>>((float*)u, g, apply_mask ? 1 : 0, rg, sk);
    else
        gs_kernel<double><<<acc, kGsThreads, 0, s>>>((double*)u, g, apply_mask ? 1 : 0, rg, sk);
    SEM_LAUNCH_CHECK("gs_kernel");
    h->launches++;
    return SEM_OK;
}

int launch_gs(sem_handle* h, void* u, bool fp32, bool apply_mask, cudaStream_t s) {
    return launch_gs_impl(h, u, fp32, apply_mask, GsSkip{}, s);
}

int launch_gs_skip(sem_handle* h, void* u, bool fp32, const GsSkip& skip, cudaStream_t s) {
    return launch_gs_impl(h, u, fp32, true, skip, s);
}

int launch_gs_until_done(sem_handle* h, void* u, bool fp32, const CGState* st, cudaStream_t s) {
    GsSkip sk;
    sk.done_st = st;
    return launch_gs_impl(h, u, fp32, true, sk, s);
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
    if (!valid_precision(precision))
        return fail(SEM_EINVAL, "unknown precision");
    return launch_gs(h, u, is_f32(precision), apply_mask != 0, s);
}

SEM_API int sem_dot(sem_handle* h, const double* a, const double* b, double* result, cudaStream_t s) {
    if (!h || !a || !b || !result) return fail(SEM_EINVAL, "null argument");
    return launch_dot(h, a, b, result, s);
}

}  // extern "C"
