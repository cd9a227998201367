// FP64-mode CG with the vectors stored as float pairs (x = hi + lo, two float
// planes, the same 8 bytes per point as a double).  On GB300 the FP64 pipe
// (1/64 of the FP32 rate) bounds the plain FP64 vector update at ~7 FP64
// operations per point; in pair form the update, the gather-scatter sums and
// the operator run on the FP32 pipe with error-free transformations (products
// by FMA, sums by TwoSum), ~2^-44 relative per operation.  Doubles appear only
// at the solve boundaries (split of x0 and of the true residual, join of the
// solution) and in the scalar reductions, which are accumulated in FP64.
#include <algorithm>

#include "sem_ax_df.cuh"
#include "sem_internal.h"

namespace sem {

__device__ __forceinline__ void split_accurate(double x, float& h, float& l) {
    h = (float)x;
    l = (float)(x - (double)h);
}

__global__ void split_pairs_kernel(const double* __restrict__ x, float* __restrict__ h, float* __restrict__ l,
                                   int64_t n) {
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x)
        split_accurate(x[L], h[L], l[L]);
}

__global__ void join_pairs_kernel(const float* __restrict__ h, const float* __restrict__ l, double* __restrict__ x,
                                  int64_t n) {
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x)
        x[L] = (double)h[L] + (double)l[L];
}

// CG start from the true residual r (double): r and z = Minv r stored as
// pairs; rho = <r,z>, rr = <r,r>, bb = <b,b> in FP64.
__global__ void __launch_bounds__(256) init_pair_kernel(const double* __restrict__ b, const double* __restrict__ r,
                                                        const double* __restrict__ minv, const uint8_t* __restrict__ mult,
                                                        float* rh, float* rl, float* zh, float* zl, int64_t n,
                                                        double tol, int max_iter, CGState* st, double* partials,
                                                        unsigned int* counter) {
    __shared__ double inv[256];
    for (int m = threadIdx.x; m < 256; m += blockDim.x) inv[m] = m ? 1.0 / m : 0.0;
    __syncthreads();
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x) {
        const double rv = r[L], zv = minv[L] * rv, bv = b[L], iv = inv[mult[L]];
        split_accurate(rv, rh[L], rl[L]);
        split_accurate(zv, zh[L], zl[L]);
        v[0] = fma(rv * zv, iv, v[0]);
        v[1] = fma(rv * rv, iv, v[1]);
        v[2] = fma(bv * bv, iv, v[2]);
    }
    grid_sum_finalize<3>(v, partials, counter, [&](double (&acc)[3]) {
        st->rho = acc[0];
        st->rho_old = 1.0;
        st->rr = acc[1];
        st->bb = acc[2];
        st->tol2 = tol * tol * acc[2];
        st->alpha = 0.0;
        st->pap = 0.0;
        st->iter = 0;
        st->carry = 0;
        st->max_iter = max_iter;
        const bool conv = (acc[2] == 0.0 || acc[1] <= st->tol2);
        st->done = (conv || max_iter <= 0) ? 1 : 0;
        st->status = (conv || max_iter > 0) ? SEM_OK : SEM_ENOTCONV;
    });
}

struct PairVecs {
    float *xh, *xl, *ph, *pl, *rh, *rl, *wh, *wl, *zh, *zl;
    const float *mh, *ml;  // Minv pairs
    const uint8_t* mult;
    int64_t n;
    CGState* st;
    double* partials;
    unsigned int* counter;
};

// One point of K-C in pair form (FP64-accurate on the FP32 pipe).
__device__ __forceinline__ void upd_pair_point(float& xh, float& xl, float ph, float pl, float& rh, float& rl,
                                               float wh, float wl, float mh, float ml, float& zh, float& zl,
                                               float iv, dfl al, float& zS, float& zE, float& rS, float& rE) {
    float S = xh, E = xl;
    df_mac(S, E, al.h, al.l, ph, pl);
    const dfl x = df_norm(S, E);
    S = rh;
    E = rl;
    df_mac(S, E, -al.h, -al.l, wh, wl);
    const dfl r = df_norm(S, E);
    float zs = 0.f, ze = 0.f;
    df_mac(zs, ze, mh, ml, r.h, r.l);
    const dfl z = df_norm(zs, ze);
    xh = x.h;
    xl = x.l;
    rh = r.h;
    rl = r.l;
    zh = z.h;
    zl = z.l;
    df_mac(zS, zE, r.h * iv, r.l * iv, z.h, z.l);
    df_mac(rS, rE, r.h * iv, r.l * iv, r.h, r.l);
}

// K-C in pair form: x += alpha p; r -= alpha w; z = Minv r; <r,z>, <r,r>.
// Four points per thread and step (16-byte loads and stores of every plane).
__global__ void __launch_bounds__(256) cg_update_pair_kernel(PairVecs a) {
    if (a.st->done) return;
    __shared__ float inv[256];
    __shared__ float s_al[2];  // alpha as a float pair, split once by thread 0
    for (int m = threadIdx.x; m < 256; m += blockDim.x) inv[m] = m ? 1.0f / (float)m : 0.0f;
    if (threadIdx.x == 0) split_accurate(a.st->alpha, s_al[0], s_al[1]);
    __syncthreads();
    dfl al;
    al.h = s_al[0];
    al.l = s_al[1];
    float zS = 0.f, zE = 0.f, rS = 0.f, rE = 0.f;
    const int64_t nv = a.n / 4;
    auto ld4 = [](const float* p, int64_t q) { return reinterpret_cast<const float4*>(p)[q]; };
    auto ld4s = [](const float* p, int64_t q) { return ld_stream(reinterpret_cast<const float4*>(p) + q); };
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv; q += (int64_t)gridDim.x * blockDim.x) {
        float4 xh = ld4(a.xh, q), xl = ld4(a.xl, q), rh = ld4(a.rh, q), rl = ld4(a.rl, q);
        const float4 ph = ld4s(a.ph, q), pl = ld4s(a.pl, q), wh = ld4s(a.wh, q), wl = ld4s(a.wl, q);
        const float4 mh = ld4s(a.mh, q), ml = ld4s(a.ml, q);
        const uchar4 mu = reinterpret_cast<const uchar4*>(a.mult)[q];
        float4 zh, zl;
        upd_pair_point(xh.x, xl.x, ph.x, pl.x, rh.x, rl.x, wh.x, wl.x, mh.x, ml.x, zh.x, zl.x, inv[mu.x], al, zS, zE, rS, rE);
        upd_pair_point(xh.y, xl.y, ph.y, pl.y, rh.y, rl.y, wh.y, wl.y, mh.y, ml.y, zh.y, zl.y, inv[mu.y], al, zS, zE, rS, rE);
        upd_pair_point(xh.z, xl.z, ph.z, pl.z, rh.z, rl.z, wh.z, wl.z, mh.z, ml.z, zh.z, zl.z, inv[mu.z], al, zS, zE, rS, rE);
        upd_pair_point(xh.w, xl.w, ph.w, pl.w, rh.w, rl.w, wh.w, wl.w, mh.w, ml.w, zh.w, zl.w, inv[mu.w], al, zS, zE, rS, rE);
        reinterpret_cast<float4*>(a.xh)[q] = xh;
        reinterpret_cast<float4*>(a.xl)[q] = xl;
        reinterpret_cast<float4*>(a.rh)[q] = rh;
        reinterpret_cast<float4*>(a.rl)[q] = rl;
        reinterpret_cast<float4*>(a.zh)[q] = zh;
        reinterpret_cast<float4*>(a.zl)[q] = zl;
    }
    if (blockIdx.x == 0) {  // scalar tail
        for (int64_t L = nv * 4 + threadIdx.x; L < a.n; L += blockDim.x)
            upd_pair_point(a.xh[L], a.xl[L], a.ph[L], a.pl[L], a.rh[L], a.rl[L], a.wh[L], a.wl[L], a.mh[L], a.ml[L],
                           a.zh[L], a.zl[L], inv[a.mult[L]], al, zS, zE, rS, rE);
    }
    float h[2] = {zS, rS}, l[2] = {zE, rE};  // float pairs to the block sums: no FP64 per thread
    CGState* st = a.st;
    grid_sum_finalize_pair<2>(h, l, a.partials, a.counter, [&](double (&acc)[2]) { cg_set_rho(st, acc[0], acc[1]); });
}

// QQ^T + mask on pairs: copies summed in ascending local index with TwoSum.
__device__ __forceinline__ void pair_accumulate(float& S, float& E, float h, float l) {
    const float s = S + h;
    const float bb = s - S;
    const float err = (S - (s - bb)) + (h - bb);
    S = s;
    E += err + l;
}

__device__ __forceinline__ void seg_pair(float* uh, float* ul, const int* idx, int c) {
    float S = uh[idx[0]], E = ul[idx[0]];
    for (int q = 1; q < c; q++) pair_accumulate(S, E, uh[idx[q]], ul[idx[q]]);
    const dfl v = df_norm(S, E);
    for (int q = 0; q < c; q++) {
        uh[idx[q]] = v.h;
        ul[idx[q]] = v.l;
    }
}

// Pairs of copies, U segments per thread: all index and value loads of the U
// segments are issued before any sum is stored (the accesses are scattered
// and latency-bound).
template <int U>
__device__ __forceinline__ void gs_pair_pairs(float* __restrict__ uh, float* __restrict__ ul, const int2* idx,
                                              int64_t n, int64_t t0, int64_t stride) {
    for (int64_t t = t0; t < n; t += stride * U) {
        int2 q[U];
        float ah[U], al[U], bh[U], bl[U];
#pragma unroll
        for (int k = 0; k < U; k++) q[k] = (t + k * stride < n) ? idx[t + k * stride] : make_int2(-1, -1);
#pragma unroll
        for (int k = 0; k < U; k++)
            if (q[k].x >= 0) {
                ah[k] = uh[q[k].x];
                al[k] = ul[q[k].x];
                bh[k] = uh[q[k].y];
                bl[k] = ul[q[k].y];
            }
#pragma unroll
        for (int k = 0; k < U; k++)
            if (q[k].x >= 0) {
                float S = ah[k], E = al[k];
                pair_accumulate(S, E, bh[k], bl[k]);
                const dfl v = df_norm(S, E);
                uh[q[k].x] = v.h;
                ul[q[k].x] = v.l;
                uh[q[k].y] = v.h;
                ul[q[k].y] = v.l;
            }
    }
}

// CTA ranges of the segment classes (as in the FP32 gather-scatter): pairs
// (4 per thread), quads, octets, other sizes, Dirichlet zeroing.
struct GsPairRanges {
    int b[5];
};
constexpr int kGsPairU = 4;

// st: the pair CG's state; a graph launch past the end of the solve returns
// at once (uniform over the grid)
__global__ void __launch_bounds__(256) gs_pair_kernel(float* __restrict__ uh, float* __restrict__ ul, GSLists g,
                                                      GsPairRanges rg, const CGState* __restrict__ st) {
    if (st->done) return;
    const int b = blockIdx.x;
    int c = 0;
    while (c < 4 && b >= rg.b[c]) c++;
    const int b0 = c ? rg.b[c - 1] : 0;
    const int64_t t0 = (int64_t)(b - b0) * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)(rg.b[c] - b0) * blockDim.x;
    if (c == 0) {
        gs_pair_pairs<kGsPairU>(uh, ul, g.pairs, g.npair, t0, stride);
    } else if (c == 1) {
        for (int64_t t = t0; t < g.nquad; t += stride) {
            const int4 q = g.quads[t];
            const int ix[4] = {q.x, q.y, q.z, q.w};
            seg_pair(uh, ul, ix, 4);
        }
    } else if (c == 2) {
        for (int64_t t = t0; t < g.noct; t += stride) {
            const int4 q0 = g.octs[2 * t], q1 = g.octs[2 * t + 1];
            const int ix[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
            seg_pair(uh, ul, ix, 8);
        }
    } else if (c == 3) {
        for (int64_t t = t0; t < g.noth; t += stride) {
            const int a = g.oth_off[t], e = g.oth_off[t + 1];
            seg_pair(uh, ul, g.oth_idx + a, e - a);
        }
    } else {
        for (int64_t t = t0; t < g.nzero; t += stride) {
            const int L = g.zero_idx[t];
            uh[L] = 0.0f;
            ul[L] = 0.0f;
        }
    }
}

__global__ void split_minv_kernel(const double* minv, float* mh, float* ml, int64_t n) {
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x)
        split_accurate(minv[L], mh[L], ml[L]);
}

// ---------------------------------------------------------------------------

bool pair_cg_available(const sem_handle* h) {
    return h->nsolve == 1 && ax_variant_for(h, h->parts[0].lx, kClsPair) == kDflVariant;
}

// the pair planes of Minv follow a changed Jacobi diagonal (Helmholtz term)
int refresh_pair_minv(sem_handle* h, cudaStream_t s) {
    if (!h->ws.pv[10]) return SEM_OK;
    split_minv_kernel<<<grid_for(h, h->n_local, 256, 8), 256, 0, s>>>(h->minv64, h->ws.pv[10], h->ws.pv[11],
                                                                       h->n_local);
    SEM_LAUNCH_CHECK("split_minv_kernel");
    return SEM_OK;
}

int ensure_pair_workspace(sem_handle* h) {
    if (h->ws.pv[0]) return SEM_OK;
    const size_t n = (size_t)h->n_local;
    for (int q = 0; q < 12; q++) {
        int rc = dalloc(h, &h->ws.pv[q], n);
        if (rc) return rc;
    }
    split_minv_kernel<<<grid_for(h, h->n_local, 256, 8), 256>>>(h->minv64, h->ws.pv[10], h->ws.pv[11], h->n_local);
    SEM_LAUNCH_CHECK("split_minv_kernel");
    SEM_CUDA_TRY(cudaDeviceSynchronize());
    return SEM_OK;
}

static PairVecs pair_vecs(sem_handle* h) {
    float** v = h->ws.pv;
    return PairVecs{v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], v[8], v[9], v[10], v[11],
                    h->mult, h->n_local, h->state, h->partials, h->counters + 3};
}

int launch_pair_split_x(sem_handle* h, cudaStream_t s) {
    split_pairs_kernel<<<grid_for(h, h->n_local, 256, 8), 256, 0, s>>>(h->ws.x, h->ws.pv[0], h->ws.pv[1], h->n_local);
    SEM_LAUNCH_CHECK("split_pairs_kernel");
    h->launches++;
    return SEM_OK;
}

int launch_pair_join_x(sem_handle* h, cudaStream_t s) {
    join_pairs_kernel<<<grid_for(h, h->n_local, 256, 8), 256, 0, s>>>(h->ws.pv[0], h->ws.pv[1], h->ws.x, h->n_local);
    SEM_LAUNCH_CHECK("join_pairs_kernel");
    h->launches++;
    return SEM_OK;
}

int launch_pair_init(sem_handle* h, double tol, int max_iter, cudaStream_t s) {
    float** v = h->ws.pv;
    init_pair_kernel<<<grid_for(h, h->n_local, 256, 4), 256, 0, s>>>(h->ws.b, h->ws.r, h->minv64, h->mult, v[4], v[5],
                                                                     v[8], v[9], h->n_local, tol, max_iter, h->state,
                                                                     h->partials, h->counters + 5);
    SEM_LAUNCH_CHECK("init_pair_kernel");
    h->launches++;
    return SEM_OK;
}

// One CG iteration in pair form: K-A (line-transform operator, pair I/O),
// then K-B (pair gather-scatter + mask) and K-C (pair update).
int launch_pair_ka(sem_handle* h, cudaStream_t s) {
    const MeshPart& p = h->parts[0];
    float** v = h->ws.pv;
    DflParams d = {};
    d.zh = v[8];
    d.zl = v[9];
    d.ph = v[2];
    d.pl = v[3];
    d.wh = v[6];
    d.wl = v[7];
    d.G2 = h->G2;
    d.E = p.E;
    d.st = h->state;
    d.partials = h->partials;
    d.counter = h->counters + 2;
    return dispatch_ax_dfl_pair_entry(h, p.lx, d, s);
}

int launch_pair_rest(sem_handle* h, cudaStream_t s) {
    float** v = h->ws.pv;
    const GSLists& g = h->gs;
    const int64_t total = g.npair + g.nquad + g.noct + g.noth + g.nzero;
    if (total > 0) {
        auto ctas = [](int64_t items, int per_thread) {
            const int64_t per = 256LL * per_thread;
            return (int)std::min<int64_t>((items + per - 1) / per, 1 << 20);
        };
        GsPairRanges rg;
        const int n[5] = {ctas(g.npair, kGsPairU), ctas(g.nquad, 1), ctas(g.noct, 1), ctas(g.noth, 1),
                          ctas(g.nzero, 1)};
        int acc = 0;
        for (int c = 0; c < 5; c++) rg.b[c] = (acc += n[c]);
        gs_pair_kernel<<<acc, 256, 0, s>>>(v[6], v[7], g, rg, h->state);
        SEM_LAUNCH_CHECK("gs_pair_kernel");
        h->launches++;
    }
    cg_update_pair_kernel<<<grid_for(h, h->n_local / 4 + 1, 256, 4), 256, 0, s>>>(pair_vecs(h));
    SEM_LAUNCH_CHECK("cg_update_pair_kernel");
    h->launches++;
    return SEM_OK;
}

int prepare_pair_kernels(sem_handle* h) {
    DflParams d = {};
    d.dry = 1;
    return dispatch_ax_dfl_pair_entry(h, h->parts[0].lx, d, 0);
}

}  // namespace sem
