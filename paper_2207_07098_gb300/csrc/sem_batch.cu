// Batched Poisson solves over many independent meshes of different sizes and
// orders (one handle from sem_setup_batch).  Every CG iteration advances all
// unconverged solves with one set of launches: the fused p-update + ax_helm
// (one persistent launch per order present, over the element groups of every
// solve of that order), the gather-scatter over all meshes, and the x/r/z
// update over point tiles.  Each solve keeps its own scalars (CGState) and is
// reduced in a fixed order, so every member of a batch is bit-reproducible;
// converged solves are skipped.  The iterations are captured in CUDA graphs.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sem_ax_df.cuh"
#include "sem_batch.cuh"
#include "sem_internal.h"

namespace sem {

struct TileList {
    const int64_t* tloc;
    const int* tlen;
    const int* tsolve;
    int64_t ntiles;
    const int* stfirst;
    const int* stcount;
    double* tpart;
    unsigned int* scount;
};

// Per-tile partials -> per-solve sums in tile order, by the CTA that finishes
// the solve's last tile.  Returns true in thread 0 of that CTA with sums in acc.
template <int NV>
__device__ __forceinline__ bool tile_finalize_sums(const TileList& tl, int64_t t, int s, double (&v)[NV],
                                                   double (&acc)[NV], double* red, int* is_last);

template <int NV>
__device__ __forceinline__ bool tile_finalize(const TileList& tl, int64_t t, int s, double (&v)[NV],
                                              double (&acc)[NV], double* red, int* is_last) {
    block_sum<NV>(v, red);
    return tile_finalize_sums<NV>(tl, t, s, v, acc, red, is_last);
}

// As tile_finalize for per-thread float pairs (FP32 kernels): the block sum
// stays in FP32 pairs and only thread 0 converts it to FP64.
template <int NV>
__device__ __forceinline__ bool tile_finalize_pair(const TileList& tl, int64_t t, int s, float (&h)[NV],
                                                   float (&l)[NV], double (&acc)[NV], double* red, float* redf,
                                                   int* is_last) {
    block_sum_pair<NV>(h, l, redf);
    double v[NV];
#pragma unroll
    for (int q = 0; q < NV; q++) v[q] = threadIdx.x == 0 ? (double)h[q] + (double)l[q] : 0.0;
    return tile_finalize_sums<NV>(tl, t, s, v, acc, red, is_last);
}

// thread 0 holds the tile's block sums in v: store them; the last tile of the
// solve adds all of its tiles' sums in tile order (result in thread 0's acc)
template <int NV>
__device__ __forceinline__ bool tile_finalize_sums(const TileList& tl, int64_t t, int s, double (&v)[NV],
                                                   double (&acc)[NV], double* red, int* is_last) {
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; q++) tl.tpart[t * 3 + q] = v[q];
        __threadfence();
        *is_last = (atomicAdd(&tl.scount[s], 1u) == (unsigned)tl.stcount[s] - 1u) ? 1 : 0;
    }
    __syncthreads();
    if (!*is_last) return false;
    __threadfence();
    const int f = tl.stfirst[s], c = tl.stcount[s];
#pragma unroll
    for (int q = 0; q < NV; q++) acc[q] = 0.0;
    for (int k = threadIdx.x; k < c; k += blockDim.x)
#pragma unroll
        for (int q = 0; q < NV; q++) acc[q] += __ldcg(&tl.tpart[(int64_t)(f + k) * 3 + q]);
    block_sum<NV>(acc, red);
    if (threadIdx.x == 0) {
        tl.scount[s] = 0u;
        return true;
    }
    return false;
}

// K-C over tiles: x += alpha p; r -= alpha w; z = Minv r; <r,z>, <r,r> per solve.
template <typename T>
__global__ void __launch_bounds__(256) upd_batch_kernel(T* x, const T* p, T* r, const T* w, T* z, const T* minv,
                                                         const uint8_t* mult, CGState* st_base, TileList tl) {
    __shared__ T inv[256];
    __shared__ double red[64];
    __shared__ float redf[128];
    __shared__ int is_last;
    // 1/m per copy count; FP32 kernels divide in FP32 (the same correctly
    // rounded values for m < 256; an FP64 division per thread would occupy
    // GB300's slow FP64 pipe at every launch)
    for (int m = threadIdx.x; m < 256; m += blockDim.x)
        inv[m] = m ? (sizeof(T) == 4 ? (T)(1.0f / (float)m) : (T)(1.0 / m)) : T(0);
    __syncthreads();
    __shared__ T s_ta;  // the solve's alpha, converted once per tile by thread 0
    for (int64_t t = blockIdx.x; t < tl.ntiles; t += gridDim.x) {
        const int s = tl.tsolve[t];
        CGState* st = st_base + s;
        if (st->done) continue;  // uniform over the CTA
        if (threadIdx.x == 0) s_ta = (T)st->alpha;
        __syncthreads();
        const T ta = s_ta;
        const int64_t l0 = tl.tloc[t], l1 = l0 + tl.tlen[t];
        T lrz = T(0), lrr = T(0);
        auto point = [&](int64_t L) {
            const T xv = fma(ta, p[L], x[L]);
            const T rv = fma(-ta, w[L], r[L]);
            const T zv = minv[L] * rv;
            x[L] = xv;
            r[L] = rv;
            z[L] = zv;
            const T iv = inv[mult[L]];
            lrz = fma(rv * zv, iv, lrz);
            lrr = fma(rv * rv, iv, lrr);
        };
        bool vec = false;
        if constexpr (sizeof(T) == 4) {
            vec = (l0 & 3) == 0;  // 16-byte aligned tile: four points per thread and step
            const int64_t v0 = l0 / 4, v1 = vec ? l1 / 4 : v0;
            for (int64_t q = v0 + threadIdx.x; q < v1; q += blockDim.x) {
                float4 xv = reinterpret_cast<const float4*>(x)[q];
                float4 rv = reinterpret_cast<const float4*>(r)[q];
                const float4 pv = ld_stream(reinterpret_cast<const float4*>(p) + q);
                const float4 wv = ld_stream(reinterpret_cast<const float4*>(w) + q);
                const float4 mv = ld_stream(reinterpret_cast<const float4*>(minv) + q);
                const uchar4 mu = reinterpret_cast<const uchar4*>(mult)[q];
                float* xs = reinterpret_cast<float*>(&xv);
                float* rs = reinterpret_cast<float*>(&rv);
                const float* ps = reinterpret_cast<const float*>(&pv);
                const float* ws = reinterpret_cast<const float*>(&wv);
                const float* ms = reinterpret_cast<const float*>(&mv);
                const unsigned char* us = reinterpret_cast<const unsigned char*>(&mu);
                float4 zv;
                float* zs = reinterpret_cast<float*>(&zv);
#pragma unroll
                for (int c = 0; c < 4; c++) {  // the arithmetic of point(), one point at a time
                    xs[c] = fmaf(ta, ps[c], xs[c]);
                    rs[c] = fmaf(-ta, ws[c], rs[c]);
                    zs[c] = ms[c] * rs[c];
                    const float iv = inv[us[c]];
                    lrz = fmaf(rs[c] * zs[c], iv, lrz);
                    lrr = fmaf(rs[c] * rs[c], iv, lrr);
                }
                reinterpret_cast<float4*>(x)[q] = xv;
                reinterpret_cast<float4*>(r)[q] = rv;
                reinterpret_cast<float4*>(z)[q] = zv;
            }
            if (vec)
                for (int64_t L = v1 * 4 + threadIdx.x; L < l1; L += blockDim.x) point(L);  // ragged end
        }
        if (!vec)
            for (int64_t L = l0 + threadIdx.x; L < l1; L += blockDim.x) point(L);
        double acc[2];
        bool last;
        if constexpr (sizeof(T) == 4) {
            float h[2] = {lrz, lrr}, l[2] = {0.f, 0.f};
            last = tile_finalize_pair<2>(tl, t, s, h, l, acc, red, redf, &is_last);
        } else {
            double v[2] = {(double)lrz, (double)lrr};
            last = tile_finalize<2>(tl, t, s, v, acc, red, &is_last);
        }
        if (last) cg_set_rho(st, acc[0], acc[1]);
        __syncthreads();
    }
}

// CG start per solve: z = Minv r; rho, rr, bb.  Solves with act[s] == 0 are
// marked done without work.  carry (may be null): per solve, > 0 keeps the
// solve's direction p with that rescaling, as cg_init_kernel's carry_c.
template <typename T>
__global__ void __launch_bounds__(256) init_batch_kernel(const T* b, const T* r, T* z, const T* minv,
                                                          const uint8_t* mult, CGState* st_base, TileList tl,
                                                          const int* act, double tol, const double* tol_per_solve,
                                                          int max_iter, const double* carry = nullptr) {
    __shared__ double inv[256];
    __shared__ double red[96];
    __shared__ int is_last;
    for (int m = threadIdx.x; m < 256; m += blockDim.x) inv[m] = m ? 1.0 / m : 0.0;
    __syncthreads();
    for (int64_t t = blockIdx.x; t < tl.ntiles; t += gridDim.x) {
        const int s = tl.tsolve[t];
        CGState* st = st_base + s;
        if (act && !act[s]) {
            if (threadIdx.x == 0 && t == tl.stfirst[s]) {
                st->done = 1;
                st->status = SEM_OK;
                st->iter = 0;
                st->carry = 0;
                st->max_iter = max_iter;
            }
            continue;
        }
        const int64_t l0 = tl.tloc[t], l1 = l0 + tl.tlen[t];
        double v[3] = {0.0, 0.0, 0.0}, acc[3];
        for (int64_t L = l0 + threadIdx.x; L < l1; L += blockDim.x) {
            const T zv = minv[L] * r[L];
            z[L] = zv;
            const double rv = (double)r[L], bv = (double)b[L], iv = inv[mult[L]];
            v[0] = fma(rv * (double)zv, iv, v[0]);
            v[1] = fma(rv * rv, iv, v[1]);
            v[2] = fma(bv * bv, iv, v[2]);
        }
        if (tile_finalize<3>(tl, t, s, v, acc, red, &is_last)) {
            if (tol_per_solve) tol = tol_per_solve[s];
            const double cc = carry ? carry[s] : 0.0, rho_prev = st->rho_old;
            st->rho = acc[0];
            st->carry = cc > 0.0 ? 1 : 0;
            st->rho_old = cc > 0.0 ? rho_prev * cc : 1.0;
            st->rr = acc[1];
            st->bb = acc[2];
            st->tol2 = tol * tol * acc[2];
            st->alpha = 0.0;
            st->pap = 0.0;
            st->iter = 0;
            st->max_iter = max_iter;
            const bool conv = (acc[2] == 0.0 || acc[1] <= st->tol2);
            st->done = (conv || max_iter <= 0) ? 1 : 0;
            st->status = (conv || max_iter > 0) ? SEM_OK : SEM_ENOTCONV;
        }
        __syncthreads();
    }
}

// r = b - w in FP64; rrbb[2s] = <r,r>, rrbb[2s+1] = <b,b> per solve.
__global__ void __launch_bounds__(256) resid_batch_kernel(const double* b, const double* w, double* r,
                                                           const uint8_t* mult, TileList tl, double* rrbb) {
    __shared__ double inv[256];
    __shared__ double red[64];
    __shared__ int is_last;
    for (int m = threadIdx.x; m < 256; m += blockDim.x) inv[m] = m ? 1.0 / m : 0.0;
    __syncthreads();
    for (int64_t t = blockIdx.x; t < tl.ntiles; t += gridDim.x) {
        const int s = tl.tsolve[t];
        const int64_t l0 = tl.tloc[t], l1 = l0 + tl.tlen[t];
        double v[2] = {0.0, 0.0}, acc[2];
        for (int64_t L = l0 + threadIdx.x; L < l1; L += blockDim.x) {
            const double bv = b[L], rv = bv - w[L];
            r[L] = rv;
            const double iv = inv[mult[L]];
            v[0] = fma(rv * rv, iv, v[0]);
            v[1] = fma(bv * bv, iv, v[1]);
        }
        if (tile_finalize<2>(tl, t, s, v, acc, red, &is_last)) {
            rrbb[2 * s] = acc[0];
            rrbb[2 * s + 1] = acc[1];
        }
        __syncthreads();
    }
}

// Refinement, per active solve: b32 = r32 = float(r / ||r||), d32 = 0.
__global__ void prepare_batch_kernel(const double* r, float* b32, float* r32, float* d32, TileList tl,
                                     const int* act, const double* rrbb) {
    for (int64_t t = blockIdx.x; t < tl.ntiles; t += gridDim.x) {
        const int s = tl.tsolve[t];
        if (!act[s]) continue;
        const double sc = 1.0 / sqrt(rrbb[2 * s]);
        const int64_t l0 = tl.tloc[t], l1 = l0 + tl.tlen[t];
        for (int64_t L = l0 + threadIdx.x; L < l1; L += blockDim.x) {
            const float v = (float)(r[L] * sc);
            b32[L] = v;
            r32[L] = v;
            d32[L] = 0.0f;
        }
    }
}

// Refinement, per active solve: x += ||r|| d32.
__global__ void correct_batch_kernel(double* x, const float* d32, TileList tl, const int* act, const double* rrbb) {
    for (int64_t t = blockIdx.x; t < tl.ntiles; t += gridDim.x) {
        const int s = tl.tsolve[t];
        if (!act[s]) continue;
        const double sc = sqrt(rrbb[2 * s]);
        const int64_t l0 = tl.tloc[t], l1 = l0 + tl.tlen[t];
        for (int64_t L = l0 + threadIdx.x; L < l1; L += blockDim.x) x[L] = fma(sc, (double)d32[L], x[L]);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static int epc_of(int lx) { return std::max(1, 256 / (lx * lx)); }

static int batch_bulk_variant(const sem_handle* h, int lx);

// Cuts every solve of order lx into groups of at most epc_for(lx) elements
// (epc 0: no groups of that order), one list per order present, numbered
// globally; fills the per-solve first group and group count on the device.
template <typename EpcFor>
static int build_group_lists(sem_handle* h, const std::vector<int>& lxs, EpcFor epc_for,
                             std::vector<LxGroups>& lists, int64_t* total, int** d_first,
                             int** d_count, double** d_part) {
    const int ns = h->nsolve;
    std::vector<int> sgfirst(ns, 0), sgcount(ns, 0);
    int64_t goff = 0;
    int rc;
    for (int lx : lxs) {
        const int epc = epc_for(lx);
        const int64_t n3 = (int64_t)lx * lx * lx;
        std::vector<int64_t> loc;
        std::vector<int> cnt, sol;
        for (int q = 0; q < ns && epc > 0; q++) {
            const MeshPart& p = h->parts[q];
            if (p.lx != lx) continue;
            sgfirst[q] = (int)(goff + (int64_t)loc.size());
            for (int e0 = 0; e0 < p.E; e0 += epc) {
                loc.push_back(p.loc_off + (int64_t)e0 * n3);
                cnt.push_back(std::min(epc, p.E - e0));
                sol.push_back(q);
            }
            sgcount[q] = (int)(goff + (int64_t)loc.size()) - sgfirst[q];
        }
        LxGroups g;
        g.lx = lx;
        g.ngroups = (int64_t)loc.size();
        g.goff = goff;
        lists.push_back(g);
        LxGroups& gl = lists.back();
        if ((rc = dalloc(h, &gl.loc, loc.size())) || (rc = dalloc(h, &gl.cnt, cnt.size())) ||
            (rc = dalloc(h, &gl.solve, sol.size())))
            return rc;
        if (!loc.empty()) {
            SEM_CUDA_TRY(cudaMemcpy(gl.loc, loc.data(), loc.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
            SEM_CUDA_TRY(cudaMemcpy(gl.cnt, cnt.data(), cnt.size() * sizeof(int), cudaMemcpyHostToDevice));
            SEM_CUDA_TRY(cudaMemcpy(gl.solve, sol.data(), sol.size() * sizeof(int), cudaMemcpyHostToDevice));
        }
        goff += g.ngroups;
    }
    *total = goff;
    if ((rc = dalloc(h, d_first, ns)) || (rc = dalloc(h, d_count, ns)) || (rc = dalloc(h, d_part, (size_t)goff)))
        return rc;
    SEM_CUDA_TRY(cudaMemcpy(*d_first, sgfirst.data(), ns * sizeof(int), cudaMemcpyHostToDevice));
    SEM_CUDA_TRY(cudaMemcpy(*d_count, sgcount.data(), ns * sizeof(int), cudaMemcpyHostToDevice));
    return SEM_OK;
}

static int build_plan(sem_handle* h) {
    BatchPlan& bp = h->batch;
    if (bp.ready) return SEM_OK;
    const int ns = h->nsolve;
    std::vector<int> lxs;
    for (auto& p : h->parts) lxs.push_back(p.lx);
    std::sort(lxs.begin(), lxs.end());
    lxs.erase(std::unique(lxs.begin(), lxs.end()), lxs.end());
    int rc = build_group_lists(h, lxs, epc_of, bp.lxg, &bp.ngroups, &bp.sgfirst, &bp.sgcount, &bp.gpart);
    if (!rc)
        rc = build_group_lists(
            h, lxs,
            [&](int lx) {
                const int v = batch_bulk_variant(h, lx);
                return v > 0 ? kBulkCfg[v - 1][0] : 0;
            },
            bp.blxg, &bp.bngroups, &bp.bsgfirst, &bp.bsgcount, &bp.bgpart);
    if (rc) return rc;
    std::vector<int64_t> tloc;
    std::vector<int> tlen, tsol, stfirst(ns), stcount(ns);
    for (int q = 0; q < ns; q++) {
        const MeshPart& p = h->parts[q];
        stfirst[q] = (int)tloc.size();
        for (int64_t a = 0; a < p.n_local; a += kTile) {
            tloc.push_back(p.loc_off + a);
            tlen.push_back((int)std::min<int64_t>(kTile, p.n_local - a));
            tsol.push_back(q);
        }
        stcount[q] = (int)tloc.size() - stfirst[q];
    }
    bp.ntiles = (int64_t)tloc.size();
    if ((rc = dalloc(h, &bp.tloc, tloc.size())) || (rc = dalloc(h, &bp.tlen, tlen.size())) ||
        (rc = dalloc(h, &bp.tsolve, tsol.size())) || (rc = dalloc(h, &bp.stfirst, ns)) ||
        (rc = dalloc(h, &bp.stcount, ns)) || (rc = dalloc(h, &bp.tpart, (size_t)bp.ntiles * 3)) || (rc = dalloc(h, &bp.scount, ns)) ||
        (rc = dalloc(h, &bp.rrbb, (size_t)2 * ns)) || (rc = dalloc(h, &bp.act, ns)) ||
        (rc = dalloc(h, &bp.itol, ns)) || (rc = dalloc(h, &bp.carry, ns)))
        return rc;
    SEM_CUDA_TRY(cudaMemcpy(bp.tloc, tloc.data(), tloc.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    SEM_CUDA_TRY(cudaMemcpy(bp.tlen, tlen.data(), tlen.size() * sizeof(int), cudaMemcpyHostToDevice));
    SEM_CUDA_TRY(cudaMemcpy(bp.tsolve, tsol.data(), tsol.size() * sizeof(int), cudaMemcpyHostToDevice));
    SEM_CUDA_TRY(cudaMemcpy(bp.stfirst, stfirst.data(), ns * sizeof(int), cudaMemcpyHostToDevice));
    SEM_CUDA_TRY(cudaMemcpy(bp.stcount, stcount.data(), ns * sizeof(int), cudaMemcpyHostToDevice));
    SEM_CUDA_TRY(cudaMemset(bp.scount, 0, ns * sizeof(unsigned)));
    bp.ready = true;
    return SEM_OK;
}

static TileList tiles(sem_handle* h) {
    BatchPlan& bp = h->batch;
    return TileList{bp.tloc, bp.tlen, bp.tsolve, bp.ntiles, bp.stfirst, bp.stcount, bp.tpart, bp.scount};
}

static int grid_tiles(sem_handle* h) { return grid_for(h, h->batch.ntiles * 256, 256, 8); }

// FP64 batches use the FP32-pair line-transform operator for the orders it
// covers unless a native variant (0..4) was pinned at set-up.
static bool batch_uses_pair_arith(const sem_handle* h, int lx) {
    const int v = h->ax_variant[0][lx];
    return (lx % 2 == 0 && lx >= 4 && lx <= 12) && (v < 0 || v >= kDfVariant);
}

// FP32 batches use the bulk-staged operator for order lx only when a bulk
// variant was pinned at set-up, it fits, and every solve of that order starts
// on a 16-byte boundary (bulk copies need it; the elements of an even order
// keep it).  By default they use the slab kernel over the element-group
// lists: on the 256-box batch (N in {5, 7, 9}) it was faster than every bulk
// variant (mixed solve 2.97 s against 3.50-3.97 s).
static int batch_bulk_variant(const sem_handle* h, int lx) {
    for (const MeshPart& p : h->parts)
        if (p.lx == lx && (p.loc_off % 4) != 0) return 0;
    const int pinned = h->ax_variant[1][lx];
    if (pinned > 0 && pinned <= kBulkVariantsMax && bulk_fits(lx, pinned, true)) return pinned;
    return 0;
}

// K-A over every order present: fused (CG state slot base `st`) or plain.
static int batch_ax(sem_handle* h, bool fp32, bool fused, const void* u, CGState* st, cudaStream_t s) {
    BatchPlan& bp = h->batch;
    for (size_t li = 0; li < bp.lxg.size(); li++) {
        const LxGroups& g = bp.lxg[li];
        int rc;
        const int bv = batch_bulk_variant(h, g.lx);
        if (fp32 && bv > 0) {
            const LxGroups& gb = bp.blxg[li];
            AxParams<float> a = {};
            a.u = (const float*)u;
            a.z = h->ws.z32;
            a.p = h->ws.p32;
            a.w = h->ws.w32;
            a.G = h->G32;
            a.D = h->D32[g.lx];
            a.variant = bv;
            a.err = device_error_word(h);
            a.wait_budget = h->test_stall ? 100000000LL : 4000000000LL;
            a.tx_extra = h->test_stall ? 16u : 0u;
            a.loc = gb.loc; a.cnt = gb.cnt; a.solve = gb.solve; a.ngroups = gb.ngroups; a.goff = gb.goff;
            a.st = st; a.sgfirst = bp.bsgfirst; a.sgcount = bp.bsgcount; a.gpart = bp.bgpart; a.scount = bp.scount;
            rc = dispatch_ax_bulk_batch_f32(h, g.lx, a, fused, s);
        } else if (fp32) {
            BatchAxParams<float> a = {};
            a.u = (const float*)u;
            a.z = h->ws.z32;
            a.p = h->ws.p32;
            a.w = h->ws.w32;
            a.G = h->G32;
            a.D = h->D32[g.lx];
            a.loc = g.loc; a.cnt = g.cnt; a.solve = g.solve; a.ngroups = g.ngroups; a.goff = g.goff;
            a.st = st; a.sgfirst = bp.sgfirst; a.sgcount = bp.sgcount; a.gpart = bp.gpart; a.scount = bp.scount;
            rc = dispatch_ax_batch_f32(h, g.lx, a, fused, s);
        } else if (batch_uses_pair_arith(h, g.lx)) {
            DflParams d = {};
            d.u = (const double*)u;
            d.z = h->ws.z;
            d.p = h->ws.p;
            d.w = h->ws.w;
            d.G2 = h->G2;
            d.loc = g.loc; d.cnt = g.cnt; d.solve = g.solve; d.ngroups = g.ngroups; d.goff = g.goff;
            d.st = st; d.sgfirst = bp.sgfirst; d.sgcount = bp.sgcount; d.gpart = bp.gpart; d.scount = bp.scount;
            rc = dispatch_ax_dfl_batch_entry(h, g.lx, d, fused, s);
        } else {
            BatchAxParams<double> a = {};
            a.u = (const double*)u;
            a.z = h->ws.z;
            a.p = h->ws.p;
            a.w = h->ws.w;
            a.G = h->G64;
            a.D = h->D64[g.lx];
            a.loc = g.loc; a.cnt = g.cnt; a.solve = g.solve; a.ngroups = g.ngroups; a.goff = g.goff;
            a.st = st; a.sgfirst = bp.sgfirst; a.sgcount = bp.sgcount; a.gpart = bp.gpart; a.scount = bp.scount;
            rc = dispatch_ax_batch_f64(h, g.lx, a, fused, s);
        }
        if (rc) return rc;
    }
    return SEM_OK;
}

static int prepare_batch_kernels(sem_handle* h) {
    for (const LxGroups& g : h->batch.lxg) {
        BatchAxParams<double> a = {};
        a.dry = 1;
        BatchAxParams<float> b = {};
        b.dry = 1;
        int rc = dispatch_ax_batch_f64(h, g.lx, a, true, 0);
        if (!rc) rc = dispatch_ax_batch_f64(h, g.lx, a, false, 0);
        if (!rc && batch_bulk_variant(h, g.lx) > 0) {
            AxParams<float> c = {};
            c.dry = 1;
            c.variant = batch_bulk_variant(h, g.lx);
            rc = dispatch_ax_bulk_batch_f32(h, g.lx, c, true, 0);
            if (!rc) rc = dispatch_ax_bulk_batch_f32(h, g.lx, c, false, 0);
        }
        if (!rc && batch_uses_pair_arith(h, g.lx)) {
            DflParams d = {};
            d.dry = 1;
            rc = dispatch_ax_dfl_batch_entry(h, g.lx, d, true, 0);
            if (!rc) rc = dispatch_ax_dfl_batch_entry(h, g.lx, d, false, 0);
        }
        if (!rc) rc = dispatch_ax_batch_f32(h, g.lx, b, true, 0);
        if (!rc) rc = dispatch_ax_batch_f32(h, g.lx, b, false, 0);
        if (rc) return rc;
    }
    return SEM_OK;
}

// Solve of every gather-scatter segment (that of its first copy: segments
// never span two meshes), for the gather-scatter that skips converged solves.
// Built once per batch handle, before any graph capture.
static int ensure_segment_solves(sem_handle* h) {
    BatchPlan& bp = h->batch;
    if (bp.sid_ready || h->nsolve > 65535) return SEM_OK;
    const GSLists& g = h->gs;
    std::vector<int64_t> starts;
    for (const MeshPart& p : h->parts) starts.push_back(p.loc_off);
    auto solve_of = [&](int64_t L) {
        return (uint16_t)(std::upper_bound(starts.begin(), starts.end(), L) - starts.begin() - 1);
    };
    std::vector<uint16_t> sid[5];
    {
        std::vector<int2> v((size_t)g.npair);
        if (g.npair) SEM_CUDA_TRY(cudaMemcpy(v.data(), g.pairs, sizeof(int2) * g.npair, cudaMemcpyDeviceToHost));
        for (auto& q : v) sid[0].push_back(solve_of(q.x));
    }
    {
        std::vector<int4> v((size_t)g.nquad);
        if (g.nquad) SEM_CUDA_TRY(cudaMemcpy(v.data(), g.quads, sizeof(int4) * g.nquad, cudaMemcpyDeviceToHost));
        for (auto& q : v) sid[1].push_back(solve_of(q.x));
    }
    {
        std::vector<int4> v((size_t)(2 * g.noct));
        if (g.noct) SEM_CUDA_TRY(cudaMemcpy(v.data(), g.octs, sizeof(int4) * 2 * g.noct, cudaMemcpyDeviceToHost));
        for (int64_t t = 0; t < g.noct; t++) sid[2].push_back(solve_of(v[2 * t].x));
    }
    {
        std::vector<int> off((size_t)g.noth + 1), idx;
        if (g.noth) {
            SEM_CUDA_TRY(cudaMemcpy(off.data(), g.oth_off, sizeof(int) * (g.noth + 1), cudaMemcpyDeviceToHost));
            idx.resize((size_t)off[g.noth]);
            SEM_CUDA_TRY(cudaMemcpy(idx.data(), g.oth_idx, sizeof(int) * idx.size(), cudaMemcpyDeviceToHost));
        }
        for (int64_t t = 0; t < g.noth; t++) sid[3].push_back(solve_of(idx[off[t]]));
    }
    {
        std::vector<int> v((size_t)g.nzero);
        if (g.nzero) SEM_CUDA_TRY(cudaMemcpy(v.data(), g.zero_idx, sizeof(int) * g.nzero, cudaMemcpyDeviceToHost));
        for (int L : v) sid[4].push_back(solve_of(L));
    }
    for (int c = 0; c < 5; c++) {
        int rc = dalloc(h, &bp.sid[c], sid[c].size());
        if (rc) return rc;
        if (!sid[c].empty())
            SEM_CUDA_TRY(cudaMemcpy(bp.sid[c], sid[c].data(), sizeof(uint16_t) * sid[c].size(), cudaMemcpyHostToDevice));
    }
    bp.sid_ready = true;
    return SEM_OK;
}

// K-B and K-C of one batched iteration (K-B leaves the segments of the
// solves already done: their w is not used).
static int batch_kb_kc(sem_handle* h, bool fp32, CGState* st, cudaStream_t s) {
    void* w = fp32 ? (void*)h->ws.w32 : (void*)h->ws.w;
    int rc;
    if (h->batch.sid_ready) {
        GsSkip sk;
        for (int c = 0; c < 5; c++) sk.sid[c] = h->batch.sid[c];
        sk.st = st;
        rc = launch_gs_skip(h, w, fp32, sk, s);
    } else {
        rc = launch_gs(h, w, fp32, true, s);
    }
    if (rc) return rc;
    if (fp32)
        upd_batch_kernel<float><<<grid_tiles(h), 256, 0, s>>>(h->ws.d32, h->ws.p32, h->ws.r32, h->ws.w32, h->ws.z32,
                                                               h->minv32, h->mult, st, tiles(h));
    else
        upd_batch_kernel<double><<<grid_tiles(h), 256, 0, s>>>(h->ws.x, h->ws.p, h->ws.r, h->ws.w, h->ws.z,
                                                                h->minv64, h->mult, st, tiles(h));
    SEM_LAUNCH_CHECK("upd_batch_kernel");
    h->launches++;
    return SEM_OK;
}

static int batch_iteration(sem_handle* h, bool fp32, CGState* st, cudaStream_t s) {
    int rc = batch_ax(h, fp32, true, nullptr, st, s);
    return rc ? rc : batch_kb_kc(h, fp32, st, s);
}

static int batch_graph(sem_handle* h, bool fp32, CGState* st, int chunk, cudaGraphExec_t* out, int* per_launch) {
    GraphCache& g = h->graph;
    const int key = 100 + (fp32 ? 1 : 0);
    if (g.exec && g.key_prec == key && g.key_chunk == chunk && g.key_ptr == st) {
        *out = g.exec;
        *per_launch = (int)h->batch.lxg.size() + 2;
        return SEM_OK;
    }
    if (g.exec) {
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
    }
    if (!h->capture_stream) SEM_CUDA_TRY(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    int rc = prepare_batch_kernels(h);
    if (!rc) rc = ensure_segment_solves(h);  // no allocation during capture
    if (rc) return rc;
    for (auto& ev : h->ax_ev)
        if (!ev) SEM_CUDA_TRY(cudaEventCreate(&ev));
    cudaStream_t cs = h->capture_stream;
    const int64_t before = h->launches;
    SEM_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int it = 0; it < chunk && rc == SEM_OK; it++) {
        if (it == 0 && cudaEventRecordWithFlags(h->ax_ev[0], cs, cudaEventRecordExternal) != cudaSuccess)
            rc = fail(SEM_ECUDA, "event record");
        if (!rc) rc = batch_ax(h, fp32, true, nullptr, st, cs);
        if (it == 0 && !rc && cudaEventRecordWithFlags(h->ax_ev[1], cs, cudaEventRecordExternal) != cudaSuccess)
            rc = fail(SEM_ECUDA, "event record");
        if (!rc) rc = batch_kb_kc(h, fp32, st, cs);
    }
    h->launches = before;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g.exec = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    g.key_prec = key;
    g.key_chunk = chunk;
    g.key_ptr = st;
    *out = g.exec;
    *per_launch = (int)h->batch.lxg.size() + 2;
    return SEM_OK;
}

// Iterate until every state in [st, st + ns) is done.
static int batch_loop(sem_handle* h, bool fp32, CGState* st, const sem_solve_opts& o, cudaStream_t s,
                      std::vector<CGState>& hs, double* ax_ms_sum, int* ax_samples) {
    const int ns = h->nsolve;
    const int chunk = std::max(1, std::min(o.graph_chunk, 1024));
    cudaGraphExec_t exec = nullptr;
    int per_launch = 0;
    if (o.use_graph) {
        int rc = batch_graph(h, fp32, st, chunk, &exec, &per_launch);
        if (rc) return rc;
    }
    auto read = [&]() -> int {
        SEM_CUDA_TRY(cudaMemcpyAsync(h->state_host, st, sizeof(CGState) * ns, cudaMemcpyDeviceToHost, s));
        SEM_CUDA_TRY(cudaStreamSynchronize(s));
        std::copy(h->state_host, h->state_host + ns, hs.begin());
        return SEM_OK;
    };
    int rc = read();
    if (rc) return rc;
    auto all_done = [&]() {
        for (auto& x : hs)
            if (!x.done) return false;
        return true;
    };
    const int64_t max_rounds = (int64_t)o.max_iter / chunk + 3;
    for (int64_t round = 0; !all_done() && round < max_rounds; round++) {
        if (exec) {
            SEM_CUDA_TRY(cudaGraphLaunch(exec, s));
            h->launches += (int64_t)per_launch * chunk;
        } else {
            for (int it = 0; it < chunk; it++)
                if ((rc = batch_iteration(h, fp32, st, s))) return rc;
        }
        if ((rc = read())) return rc;
        if (exec) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, h->ax_ev[0], h->ax_ev[1]) == cudaSuccess) {
                *ax_ms_sum += ms;
                (*ax_samples)++;
            } else {
                cudaGetLastError();
            }
        }
    }
    if (!all_done()) return fail(SEM_ETIMEOUT, "batched CG loop did not finish within its iteration budget");
    return SEM_OK;
}

static int batch_true_residual(sem_handle* h, cudaStream_t s) {
    int rc = batch_ax(h, false, false, h->ws.x, nullptr, s);
    if (!rc) rc = launch_gs(h, h->ws.w, false, true, s);
    if (rc) return rc;
    resid_batch_kernel<<<grid_tiles(h), 256, 0, s>>>(h->ws.b, h->ws.w, h->ws.r, h->mult, tiles(h), h->batch.rrbb);
    SEM_LAUNCH_CHECK("resid_batch_kernel");
    h->launches++;
    return SEM_OK;
}

static bool host_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

static int solve_batch(sem_handle* h, double* x_user, const double* b_user, const sem_solve_opts& o,
                       sem_solve_stats* stats, cudaStream_t s) {
    int rc = ensure_workspace(h, o.mode == SEM_MODE_MIXED_IR);
    if (!rc) rc = build_plan(h);
    if (rc) return rc;
    const int ns = h->nsolve;
    const int64_t n = h->n_local;
    const size_t bytes = sizeof(double) * n;
    BatchPlan& bp = h->batch;
    const bool xh = host_ptr(x_user), bh = host_ptr(b_user);
    const int64_t launches0 = h->launches;
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, s);
    SEM_CUDA_TRY(cudaMemcpyAsync(h->ws.x, x_user, bytes, xh ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    SEM_CUDA_TRY(cudaMemcpyAsync(h->ws.b, b_user, bytes, bh ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    std::vector<CGState> hs(ns);
    std::vector<int> status(ns, SEM_OK), iters(ns, 0), outer(ns, 0);
    std::vector<double> rrbb(2 * ns);
    double ax_sum = 0.0;
    int ax_n = 0;
    auto read_rrbb = [&]() -> int {
        SEM_CUDA_TRY(cudaMemcpyAsync(rrbb.data(), bp.rrbb, sizeof(double) * 2 * ns, cudaMemcpyDeviceToHost, s));
        SEM_CUDA_TRY(cudaStreamSynchronize(s));
        return SEM_OK;
    };
    if ((rc = batch_true_residual(h, s))) return rc;
    if (o.mode == SEM_MODE_FP64) {
        // CG with residual replacement per solve (see the single-mesh solver)
        std::vector<int> act(ns, 1);
        for (int restart = 0;; restart++) {
            if (restart > 0) {
                if ((rc = batch_true_residual(h, s)) || (rc = read_rrbb())) return rc;
                int nact = 0;
                for (int q = 0; q < ns; q++) {
                    const double bb = rrbb[2 * q + 1];
                    const double rel = relative_residual(rrbb[2 * q], bb);
                    act[q] = (status[q] == SEM_OK && rel > o.tol && iters[q] < o.max_iter && restart <= 4) ? 1 : 0;
                    nact += act[q];
                }
                if (nact == 0) break;
                SEM_CUDA_TRY(cudaMemcpyAsync(bp.act, act.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
                init_batch_kernel<double><<<grid_tiles(h), 256, 0, s>>>(h->ws.b, h->ws.r, h->ws.z, h->minv64, h->mult,
                                                                         h->state, tiles(h), bp.act, o.tol, nullptr,
                                                                         o.max_iter);
            } else {
                init_batch_kernel<double><<<grid_tiles(h), 256, 0, s>>>(h->ws.b, h->ws.r, h->ws.z, h->minv64, h->mult,
                                                                         h->state, tiles(h), nullptr, o.tol, nullptr,
                                                                         o.max_iter);
            }
            SEM_LAUNCH_CHECK("init_batch_kernel");
            h->launches++;
            if ((rc = batch_loop(h, false, h->state, o, s, hs, &ax_sum, &ax_n))) return rc;
            for (int q = 0; q < ns; q++)
                if (act[q]) {
                    status[q] = hs[q].status;
                    iters[q] += hs[q].iter;
                }
        }
    } else {
        std::vector<double> prev(ns, INFINITY);
        std::vector<int> act(ns, 0), fin(ns, 0);
        std::vector<double> itol(ns, o.inner_tol), carry(ns, 0.0), rn_prev(ns, 0.0);
        std::vector<int> can_carry(ns, 0);
        if ((rc = read_rrbb())) return rc;
        CGState* inner = h->state + ns;
        for (int round = 0;; round++) {
            int nact = 0;
            for (int q = 0; q < ns; q++) {
                act[q] = 0;
                if (fin[q]) continue;
                const double bb = rrbb[2 * q + 1];
                const double rel = relative_residual(rrbb[2 * q], bb);
                if (!std::isfinite(rel)) { status[q] = SEM_EBREAKDOWN; fin[q] = 1; }
                else if (bb == 0.0 || rel <= o.tol) { status[q] = SEM_OK; fin[q] = 1; }
                else if (outer[q] >= o.max_outer) { status[q] = SEM_ENOTCONV; fin[q] = 1; }
                else if (outer[q] > 0 && rel > 0.5 * prev[q]) { status[q] = SEM_ESTAGNATE; fin[q] = 1; }
                else {
                    act[q] = 1;
                    prev[q] = rel;
                    itol[q] = inner_tolerance(o, rel);
                    // kept direction: its units were ||r_prev|| / ||r|| times smaller
                    const double rn = std::sqrt(rrbb[2 * q]);
                    carry[q] = (o.ir_carry && can_carry[q] && rn > 0.0) ? rn_prev[q] / rn : 0.0;
                    rn_prev[q] = rn;
                    nact++;
                }
            }
            if (nact == 0) break;
            SEM_CUDA_TRY(cudaMemcpyAsync(bp.act, act.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
            SEM_CUDA_TRY(cudaMemcpyAsync(bp.itol, itol.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s));
            SEM_CUDA_TRY(cudaMemcpyAsync(bp.carry, carry.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s));
            prepare_batch_kernel<<<grid_tiles(h), 256, 0, s>>>(h->ws.r, h->ws.b32, h->ws.r32, h->ws.d32, tiles(h),
                                                               bp.act, bp.rrbb);
            init_batch_kernel<float><<<grid_tiles(h), 256, 0, s>>>(h->ws.b32, h->ws.r32, h->ws.z32, h->minv32, h->mult,
                                                                    inner, tiles(h), bp.act, o.inner_tol, bp.itol,
                                                                    o.max_iter, bp.carry);
            SEM_LAUNCH_CHECK("batch refinement prepare");
            h->launches += 2;
            if ((rc = batch_loop(h, true, inner, o, s, hs, &ax_sum, &ax_n))) return rc;
            for (int q = 0; q < ns; q++)
                if (act[q]) {
                    iters[q] += hs[q].iter;
                    outer[q]++;
                    can_carry[q] = hs[q].status == SEM_OK && hs[q].iter > 0;
                }
            correct_batch_kernel<<<grid_tiles(h), 256, 0, s>>>(h->ws.x, h->ws.d32, tiles(h), bp.act, bp.rrbb);
            SEM_LAUNCH_CHECK("correct_batch_kernel");
            h->launches++;
            if ((rc = batch_true_residual(h, s)) || (rc = read_rrbb())) return rc;
        }
    }
    SEM_CUDA_TRY(cudaMemcpyAsync(x_user, h->ws.x, bytes, xh ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    cudaEventRecord(ev1, s);
    SEM_CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    int worst = SEM_OK;
    for (int q = 0; q < ns; q++) {
        if (status[q] != SEM_OK && (worst == SEM_OK || status[q] > worst)) worst = status[q];
        if (stats) {
            sem_solve_stats& st = stats[q];
            st = sem_solve_stats{};
            st.status = status[q];
            st.iterations = iters[q];
            st.outer_iterations = o.mode == SEM_MODE_MIXED_IR ? outer[q] : 0;
            const double bb = rrbb[2 * q + 1];
            st.relres = relative_residual(rrbb[2 * q], bb);
            st.relres_recursive = o.mode == SEM_MODE_FP64 && hs[q].bb > 0 ? std::sqrt(hs[q].rr / hs[q].bb) : st.relres;
            st.time_ms = ms;
            st.kernel_launches = h->launches - launches0;
            st.ax_samples = ax_n;
            st.ax_ms = ax_n ? ax_sum / ax_n : 0.0;
        }
    }
    if (worst != SEM_OK) set_error("at least one solve of the batch did not converge (see per-solve stats)");
    return worst;
}

}  // namespace sem

using namespace sem;

extern "C" {

SEM_API int sem_cg_solve_batch(sem_handle* h, double* x, const double* b, const sem_solve_opts* opts,
                               sem_solve_stats* stats, cudaStream_t s) {
    if (!h || !x || !b) return fail(SEM_EINVAL, "null argument");
    sem_solve_opts o;
    sem_solve_opts_default(&o);
    if (opts) o = *opts;
    if (!(o.tol > 0.0) || o.max_iter < 0 || (o.mode != SEM_MODE_FP64 && o.mode != SEM_MODE_MIXED_IR))
        return fail(SEM_EINVAL, "bad solve options");
    if (o.mode == SEM_MODE_MIXED_IR && !(o.inner_tol > 0.0 && o.inner_tol < 1.0))
        return fail(SEM_EINVAL, "inner_tol must be in (0, 1)");
    return solve_batch(h, x, b, o, stats, s);
}

}  // extern "C"
