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


// Cuts every solve of order lx into groups of at most epc_for(lx) elements
// (epc 0: no groups of that order), one list per order present, numbered
// globally; fills the per-solve first group and group count on the device.
struct UnifiedGroups {
    std::vector<int64_t> loc;
    std::vector<int> cnt, sol;
    std::vector<uint8_t> lx;
};

template <typename EpcFor>
static int build_group_lists(sem_handle* h, const std::vector<int>& lxs, EpcFor epc_for,
                             std::vector<LxGroups>& lists, int64_t* total, int** d_first,
                             int** d_count, double** d_part, UnifiedGroups* all = nullptr) {
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
        if (all) {
            all->loc.insert(all->loc.end(), loc.begin(), loc.end());
            all->cnt.insert(all->cnt.end(), cnt.begin(), cnt.end());
            all->sol.insert(all->sol.end(), sol.begin(), sol.end());
            all->lx.insert(all->lx.end(), loc.size(), (uint8_t)lx);
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

static std::vector<int> orders_present(const sem_handle* h) {
    std::vector<int> lxs;
    for (auto& p : h->parts) lxs.push_back(p.lx);
    std::sort(lxs.begin(), lxs.end());
    lxs.erase(std::unique(lxs.begin(), lxs.end()), lxs.end());
    return lxs;
}

static int build_plan(sem_handle* h) {
    BatchPlan& bp = h->batch;
    if (bp.ready) return SEM_OK;
    const int ns = h->nsolve;
    const std::vector<int> lxs = orders_present(h);
    UnifiedGroups all;
    int rc = build_group_lists(h, lxs, epc_of, bp.lxg, &bp.ngroups, &bp.sgfirst, &bp.sgcount, &bp.gpart, &all);
    if (rc) return rc;
    bp.multi_ok = lxs.back() <= kMultiMaxLx;
    if ((rc = dalloc(h, &bp.uloc, all.loc.size())) || (rc = dalloc(h, &bp.ucnt, all.cnt.size())) ||
        (rc = dalloc(h, &bp.usolve, all.sol.size())) || (rc = dalloc(h, &bp.ulx, all.lx.size())))
        return rc;
    if (!all.loc.empty()) {
        SEM_CUDA_TRY(cudaMemcpy(bp.uloc, all.loc.data(), all.loc.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
        SEM_CUDA_TRY(cudaMemcpy(bp.ucnt, all.cnt.data(), all.cnt.size() * sizeof(int), cudaMemcpyHostToDevice));
        SEM_CUDA_TRY(cudaMemcpy(bp.usolve, all.sol.data(), all.sol.size() * sizeof(int), cudaMemcpyHostToDevice));
        SEM_CUDA_TRY(cudaMemcpy(bp.ulx, all.lx.data(), all.lx.size(), cudaMemcpyHostToDevice));
    }
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

// FP64 batches with SEM_FP64_PAIR use the FP32-pair line-transform operator
// for the orders it covers; every other FP64 application (SEM_FP64, the true
// residual) uses the native FP64 batch kernel.
static bool batch_uses_pair_arith(const sem_handle* h, int lx, int precision) {
    // (the pair kernels carry no Helmholtz mass term)
    return precision == SEM_FP64_PAIR && !h->hmass64 && lx % 2 == 0 && lx >= 4 && lx <= 12;
}

// Bulk-staged operator variant v (1..4) can serve order lx of an FP32 batch:
// it fits, and every solve of that order starts on a 16-byte boundary (bulk
// copies need it; the elements of an even order keep it).
static bool batch_bulk_ok(const sem_handle* h, int lx, int v) {
    // (the bulk-staged kernels carry no Helmholtz mass term)
    if (v < 1 || v > kBulkVariantsMax || !bulk_fits(lx, v, true) || h->hmass64) return false;
    for (const MeshPart& p : h->parts)
        if (p.lx == lx && (p.loc_off % 4) != 0) return false;
    return true;
}

static int bulk_set_index(int epc) { return epc == 1 ? 0 : epc == 2 ? 1 : 2; }

// group lists cut to `epc` elements per group for every order present
static int ensure_bulk_set(sem_handle* h, int epc) {
    BatchPlan::BulkSet& bs = h->batch.bulk[bulk_set_index(epc)];
    if (bs.built) return SEM_OK;
    int rc = build_group_lists(h, orders_present(h), [&](int) { return epc; }, bs.lists, &bs.ngroups, &bs.sgfirst,
                               &bs.sgcount, &bs.gpart);
    if (rc) return rc;
    bs.built = true;
    return SEM_OK;
}

// K-A of one order lx (list index li) with operator variant v: fused (CG state
// slot base `st`) or plain.  precision: SEM_FP32, SEM_FP64 or SEM_FP64_PAIR.
static int batch_ax_order(sem_handle* h, int precision, size_t li, int v, bool fused, const void* u, CGState* st,
                          cudaStream_t s) {
    BatchPlan& bp = h->batch;
    const LxGroups& g = bp.lxg[li];
    if (precision == SEM_FP32 && v > 0) {
        const int epc = kBulkCfg[v - 1][0];
        int rc = ensure_bulk_set(h, epc);
        if (rc) return rc;
        const BatchPlan::BulkSet& bs = bp.bulk[bulk_set_index(epc)];
        const LxGroups& gb = bs.lists[li];
        AxParams<float> a = {};
        a.u = (const float*)u;
        a.z = h->ws.z32;
        a.p = h->ws.p32;
        a.w = h->ws.w32;
        a.G = h->G32;
        a.D = h->D32[g.lx];
        a.variant = v;
        a.err = device_error_word(h);
        a.wait_budget = h->test_stall ? 100000000LL : 4000000000LL;
        a.tx_extra = h->test_stall ? 16u : 0u;
        a.loc = gb.loc; a.cnt = gb.cnt; a.solve = gb.solve; a.ngroups = gb.ngroups; a.goff = gb.goff;
        a.st = st; a.sgfirst = bs.sgfirst; a.sgcount = bs.sgcount; a.gpart = bs.gpart; a.scount = bp.scount;
        return dispatch_ax_bulk_batch_f32(h, g.lx, a, fused, s);
    }
    if (precision == SEM_FP32) {
        BatchAxParams<float> a = {};
        a.u = (const float*)u;
        a.z = h->ws.z32;
        a.p = h->ws.p32;
        a.w = h->ws.w32;
        a.G = h->G32;
        a.D = h->D32[g.lx];
        a.loc = g.loc; a.cnt = g.cnt; a.solve = g.solve; a.ngroups = g.ngroups; a.goff = g.goff;
        a.st = st; a.sgfirst = bp.sgfirst; a.sgcount = bp.sgcount; a.gpart = bp.gpart; a.scount = bp.scount;
        a.mass = h->hmass32;
        return dispatch_ax_batch_f32(h, g.lx, a, fused, s);
    }
    if (batch_uses_pair_arith(h, g.lx, precision)) {
        DflParams d = {};
        d.u = (const double*)u;
        d.z = h->ws.z;
        d.p = h->ws.p;
        d.w = h->ws.w;
        d.G2 = h->G2;
        d.loc = g.loc; d.cnt = g.cnt; d.solve = g.solve; d.ngroups = g.ngroups; d.goff = g.goff;
        d.st = st; d.sgfirst = bp.sgfirst; d.sgcount = bp.sgcount; d.gpart = bp.gpart; d.scount = bp.scount;
        return dispatch_ax_dfl_batch_entry(h, g.lx, d, fused, s);
    }
    BatchAxParams<double> a = {};
    a.u = (const double*)u;
    a.z = h->ws.z;
    a.p = h->ws.p;
    a.w = h->ws.w;
    a.G = h->G64;
    a.D = h->D64[g.lx];
    a.loc = g.loc; a.cnt = g.cnt; a.solve = g.solve; a.ngroups = g.ngroups; a.goff = g.goff;
    a.st = st; a.sgfirst = bp.sgfirst; a.sgcount = bp.sgcount; a.gpart = bp.gpart; a.scount = bp.scount;
    a.mass = h->hmass64;
    return dispatch_ax_batch_f64(h, g.lx, a, fused, s);
}

// One slab launch over the groups of every order (SEM_FP32 or SEM_FP64).
static int batch_ax_multi(sem_handle* h, int precision, bool fused, const void* u, CGState* st, cudaStream_t s,
                          int dry = 0) {
    BatchPlan& bp = h->batch;
    bool present[kMaxLx + 1] = {};
    for (const LxGroups& g : bp.lxg) present[g.lx] = true;
    if (precision == SEM_FP32) {
        BatchAxParams<float> a = {};
        a.u = (const float*)u;
        a.z = h->ws.z32;
        a.p = h->ws.p32;
        a.w = h->ws.w32;
        a.G = h->G32;
        a.loc = bp.uloc; a.cnt = bp.ucnt; a.solve = bp.usolve; a.ngroups = bp.ngroups; a.goff = 0;
        a.st = st; a.sgfirst = bp.sgfirst; a.sgcount = bp.sgcount; a.gpart = bp.gpart; a.scount = bp.scount;
        a.dry = dry;
        a.mass = h->hmass32;
        MultiOrder<float> mo = {};
        for (int lx = 2; lx <= kMultiMaxLx; lx++) mo.D[lx] = present[lx] ? h->D32[lx] : nullptr;
        mo.lx = bp.ulx;
        return launch_ax_batch_multi_f32(h, a, mo, multi_smem_bytes<float>(present), fused, s);
    }
    BatchAxParams<double> a = {};
    a.u = (const double*)u;
    a.z = h->ws.z;
    a.p = h->ws.p;
    a.w = h->ws.w;
    a.G = h->G64;
    a.loc = bp.uloc; a.cnt = bp.ucnt; a.solve = bp.usolve; a.ngroups = bp.ngroups; a.goff = 0;
    a.st = st; a.sgfirst = bp.sgfirst; a.sgcount = bp.sgcount; a.gpart = bp.gpart; a.scount = bp.scount;
    a.dry = dry;
    a.mass = h->hmass64;
    MultiOrder<double> mo = {};
    for (int lx = 2; lx <= kMultiMaxLx; lx++) mo.D[lx] = present[lx] ? h->D64[lx] : nullptr;
    mo.lx = bp.ulx;
    return launch_ax_batch_multi_f64(h, a, mo, multi_smem_bytes<double>(present), fused, s);
}

// K-A over every order present with the class's chosen configuration.
static int batch_ax(sem_handle* h, int precision, bool fused, const void* u, CGState* st, cudaStream_t s) {
    BatchPlan& bp = h->batch;
    const int cls = precision == SEM_FP32 ? kClsF32 : kClsF64;
    if (precision != SEM_FP64_PAIR && bp.kcfg[cls] == 1) return batch_ax_multi(h, precision, fused, u, st, s);
    for (size_t li = 0; li < bp.lxg.size(); li++) {
        const int v = precision == SEM_FP64_PAIR ? 0 : bp.ovar[cls][bp.lxg[li].lx];
        int rc = batch_ax_order(h, precision, li, v, fused, u, st, s);
        if (rc) return rc;
    }
    return SEM_OK;
}

// K-A launches of one batched iteration
static int batch_ka_launches(const sem_handle* h, int precision) {
    const int cls = precision == SEM_FP32 ? kClsF32 : kClsF64;
    return (precision != SEM_FP64_PAIR && h->batch.kcfg[cls] == 1) ? 1 : (int)h->batch.lxg.size();
}

// Operator configuration of a batch for class cls (FP32 or native FP64):
// variants pinned at set-up are honoured (one launch per order, the pinned
// bulk-staged variant where it fits); otherwise, with autotuning, one slab
// launch per order and one multi-order slab launch over every group are
// timed on the handle's own data with the plain operator, and the faster is
// kept; without autotuning the multi-order launch is taken where it applies.
// The bulk-staged variants are not candidates: timed plain they beat the
// slab kernel on a batch, but inside the solve, where members converge at
// different iterations, they lost (256-box mixed batch, kept direction:
// 2.94-2.98 s against 2.33 s per-order slab and 2.46 s multi-order).  Runs
// once per handle and class, outside any capture.
static int batch_configure(sem_handle* h, int cls, bool autotune, cudaStream_t s) {
    BatchPlan& bp = h->batch;
    if (bp.kcfg[cls] >= 0) return SEM_OK;
    const bool fp32 = cls == kClsF32;
    const int precision = fp32 ? SEM_FP32 : SEM_FP64;
    bool pinned = false;
    for (const LxGroups& g : bp.lxg) {
        const int v = h->ax_variant[cls][g.lx];
        if (v >= 0 && v <= kBulkVariantsMax) {
            pinned = true;
            bp.ovar[cls][g.lx] = (fp32 && batch_bulk_ok(h, g.lx, v)) ? v : 0;
        } else {
            bp.ovar[cls][g.lx] = 0;
        }
    }
    if (pinned) {
        bp.kcfg[cls] = 0;
        return SEM_OK;
    }
    if (!autotune) {
        bp.kcfg[cls] = bp.multi_ok ? 1 : 0;
        return SEM_OK;
    }
    int rc = ensure_workspace(h, fp32);
    if (rc) return rc;
    const void* u = fp32 ? (const void*)h->ws.z32 : (const void*)h->ws.z;
    SEM_CUDA_TRY(cudaMemsetAsync(const_cast<void*>(u), 0, (fp32 ? 4 : 8) * (size_t)h->n_local, s));
    cudaEvent_t e0, e1;
    SEM_CUDA_TRY(cudaEventCreate(&e0));
    SEM_CUDA_TRY(cudaEventCreate(&e1));
    auto time_it = [&](auto&& launch, float* ms) -> int {
        int r = launch();  // warm-up (also sets kernel attributes outside any capture)
        if (r) return r;
        cudaEventRecord(e0, s);
        for (int k = 0; k < 3 && !r; k++) r = launch();
        cudaEventRecord(e1, s);
        if (r) return r;
        if (cudaEventSynchronize(e1) != cudaSuccess) return cuda_fail(cudaGetLastError(), "batch tuning");
        cudaEventElapsedTime(ms, e0, e1);
        return SEM_OK;
    };
    float per_order = 0.0f;
    rc = time_it(
        [&]() {
            for (size_t li = 0; li < bp.lxg.size(); li++) {
                int r = batch_ax_order(h, precision, li, 0, false, u, nullptr, s);
                if (r) return r;
            }
            return (int)SEM_OK;
        },
        &per_order);
    for (const LxGroups& g : bp.lxg) bp.ovar[cls][g.lx] = 0;
    int cfg = 0;
    if (!rc && bp.multi_ok) {
        float ms = 0.0f;
        rc = time_it([&]() { return batch_ax_multi(h, precision, false, u, nullptr, s); }, &ms);
        if (!rc && ms < per_order) cfg = 1;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    bp.kcfg[cls] = cfg;
    return SEM_OK;
}

static int prepare_batch_kernels(sem_handle* h) {
    BatchPlan& bp = h->batch;
    // group lists of the bulk-staged variants in use (allocation is not allowed during capture)
    for (const LxGroups& g : bp.lxg) {
        const int v = bp.ovar[kClsF32][g.lx];
        if (v > 0) {
            int rc = ensure_bulk_set(h, kBulkCfg[v - 1][0]);
            if (rc) return rc;
        }
    }
    for (int cls = 0; cls < 2; cls++) {
        if (bp.kcfg[cls] == 1) {
            const int prec = cls == kClsF32 ? SEM_FP32 : SEM_FP64;
            int rc = batch_ax_multi(h, prec, true, nullptr, nullptr, 0, 1);
            if (!rc) rc = batch_ax_multi(h, prec, false, nullptr, nullptr, 0, 1);
            if (rc) return rc;
        }
    }
    for (const LxGroups& g : bp.lxg) {
        BatchAxParams<double> a = {};
        a.dry = 1;
        BatchAxParams<float> b = {};
        b.dry = 1;
        int rc = dispatch_ax_batch_f64(h, g.lx, a, true, 0);
        if (!rc) rc = dispatch_ax_batch_f64(h, g.lx, a, false, 0);
        const int bv = bp.ovar[kClsF32][g.lx];
        if (!rc && bv > 0) {
            AxParams<float> c = {};
            c.dry = 1;
            c.variant = bv;
            rc = dispatch_ax_bulk_batch_f32(h, g.lx, c, true, 0);
            if (!rc) rc = dispatch_ax_bulk_batch_f32(h, g.lx, c, false, 0);
        }
        if (!rc && batch_uses_pair_arith(h, g.lx, SEM_FP64_PAIR)) {
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
static int batch_kb_kc(sem_handle* h, int precision, CGState* st, cudaStream_t s) {
    const bool fp32 = precision == SEM_FP32;
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

static int batch_iteration(sem_handle* h, int precision, CGState* st, cudaStream_t s) {
    int rc = batch_ax(h, precision, true, nullptr, st, s);
    return rc ? rc : batch_kb_kc(h, precision, st, s);
}

static int batch_graph(sem_handle* h, int precision, CGState* st, int chunk, cudaGraphExec_t* out,
                       int* per_launch) {
    GraphCache& g = h->graph;
    const int key = 100 + precision;
    if (g.exec && g.key_prec == key && g.key_chunk == chunk && g.key_ptr == st) {
        *out = g.exec;
        *per_launch = batch_ka_launches(h, precision) + 2;
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
        if (!rc) rc = batch_ax(h, precision, true, nullptr, st, cs);
        if (it == 0 && !rc && cudaEventRecordWithFlags(h->ax_ev[1], cs, cudaEventRecordExternal) != cudaSuccess)
            rc = fail(SEM_ECUDA, "event record");
        if (!rc) rc = batch_kb_kc(h, precision, st, cs);
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
    *per_launch = batch_ka_launches(h, precision) + 2;
    return SEM_OK;
}

// Iterate until every state in [st, st + ns) is done.
static int batch_loop(sem_handle* h, int precision, CGState* st, const sem_solve_opts& o, cudaStream_t s,
                      std::vector<CGState>& hs, double* ax_ms_sum, int* ax_samples) {
    const int ns = h->nsolve;
    const int chunk = std::max(1, std::min(o.graph_chunk, 1024));
    cudaGraphExec_t exec = nullptr;
    int per_launch = 0;
    if (o.use_graph) {
        int rc = batch_graph(h, precision, st, chunk, &exec, &per_launch);
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
                if ((rc = batch_iteration(h, precision, st, s))) return rc;
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

// r = b - A x per solve with the native FP64 operator, <r,r> and <b,b> per solve
static int batch_true_residual(sem_handle* h, cudaStream_t s) {
    int rc = batch_ax(h, SEM_FP64, false, h->ws.x, nullptr, s);
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
    // operator configuration of each class this solve uses (tuned once per handle)
    if (!rc) rc = batch_configure(h, kClsF64, o.autotune != 0, s);
    if (!rc && o.mode == SEM_MODE_MIXED_IR) rc = batch_configure(h, kClsF32, o.autotune != 0, s);
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
    if ((rc = batch_true_residual(h, s)) || (rc = read_rrbb())) return rc;
    std::vector<double> rel0(ns);
    for (int q = 0; q < ns; q++) rel0[q] = relative_residual(rrbb[2 * q], rrbb[2 * q + 1]);
    if (o.mode == SEM_MODE_FP64) {
        // SEM_FP64_NATIVE has no batched form of its own: the FP64 class serves it
        const int prec64 = o.precision == SEM_FP64_PAIR ? SEM_FP64_PAIR : SEM_FP64;
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
            if ((rc = batch_loop(h, prec64, h->state, o, s, hs, &ax_sum, &ax_n))) return rc;
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
        std::vector<int> can_carry(ns, 0), capped(ns, 0);
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
                else if (outer[q] > 0 && rel > 0.5 * prev[q] && !capped[q]) { status[q] = SEM_ESTAGNATE; fin[q] = 1; }
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
            if ((rc = batch_loop(h, SEM_FP32, inner, o, s, hs, &ax_sum, &ax_n))) return rc;
            for (int q = 0; q < ns; q++)
                if (act[q]) {
                    iters[q] += hs[q].iter;
                    outer[q]++;
                    // a step stopped by max_iter is not judged for stagnation and keeps its direction
                    capped[q] = hs[q].iter >= o.max_iter ? 1 : 0;
                    can_carry[q] = (hs[q].status == SEM_OK || hs[q].status == SEM_ENOTCONV) && hs[q].iter > 0;
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
        // SEM_OK promises the tolerance on the true residual of the returned x
        const double relq = relative_residual(rrbb[2 * q], rrbb[2 * q + 1]);
        if (status[q] == SEM_OK && !(relq <= o.tol)) status[q] = std::isfinite(relq) ? SEM_ENOTCONV : SEM_EBREAKDOWN;
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
            const int itprec = o.mode == SEM_MODE_MIXED_IR ? SEM_FP32 : (o.precision == SEM_FP64_PAIR ? SEM_FP64_PAIR : SEM_FP64);
            const int cls = itprec == SEM_FP32 ? kClsF32 : kClsF64;
            st.launches_per_iteration = batch_ka_launches(h, itprec) + 2;
            st.relres_start = rel0[q];
            st.ax_variant = (itprec == SEM_FP64_PAIR && !h->hmass64) ? kDflVariant
                            : bp.kcfg[cls] == 1 ? kMultiVariant : bp.ovar[cls][h->parts[q].lx];
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
    if (o.mode == SEM_MODE_FP64 && (!valid_precision(o.precision) || is_f32(o.precision)))
        return fail(SEM_EINVAL, "FP64 mode takes SEM_FP64, SEM_FP64_NATIVE or SEM_FP64_PAIR");
    if (o.projection != 0) return fail(SEM_EINVAL, "projection onto previous solutions: single-mesh handles only");
    return solve_batch(h, x, b, o, stats, s);
}

}  // extern "C"
