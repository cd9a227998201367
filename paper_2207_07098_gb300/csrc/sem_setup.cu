// Set-up of libsem handles: GLL basis, gather-scatter lists, geometric
// factors, mass and Jacobi diagonal (Sec. II-A and II-B of Karp et al.).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include "sem_ax.cuh"
#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return SEM_ECUDA;
}

int grid_for(sem_handle* h, int64_t work_items, int threads, int per_sm) {
    int64_t blocks = (work_items + threads - 1) / threads;
    int64_t cap = (int64_t)h->sm_count * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (blocks > kMaxPartials) blocks = kMaxPartials;
    return (int)blocks;
}

// ---------------------------------------------------------------------------
// GLL basis.  Nodes: -1, 1 and the roots of P_N'.  Here they are found as the
// roots of q = P_{N+1} - P_{N-1}, which vanishes exactly at the N+1 GLL nodes
// because P_{N+1} - P_{N-1} = (2N+1)/(N(N+1)) (x^2 - 1) P_N'; Newton uses
// q' = (2N+1) P_N.  Weights 2/(N(N+1) P_N^2); D_ij = l_j'(xi_i).
// ---------------------------------------------------------------------------
static void legendre_upto(int n, long double x, long double* P) {  // P[0..n]
    P[0] = 1.0L;
    if (n >= 1) P[1] = x;
    for (int m = 1; m < n; m++) P[m + 1] = ((2 * m + 1) * x * P[m] - m * P[m - 1]) / (m + 1);
}

static void gll_basis(int lx, double* xi, double* rho, double* D) {
    const int N = lx - 1;
    long double P[kMaxLx + 2];
    std::vector<long double> x(lx), PN(lx);
    const long double pi = 3.14159265358979323846264338327950288L;
    for (int i = 0; i <= N; i++) {
        long double t = -cosl(pi * (long double)i / (long double)N);
        if (i > 0 && i < N) {
            for (int it = 0; it < 60; it++) {
                legendre_upto(N + 1, t, P);
                long double q = P[N + 1] - P[N - 1];
                long double dq = (2 * N + 1) * P[N];
                long double step = q / dq;
                t -= step;
                if (fabsl(step) <= 4e-19L * (1.0L + fabsl(t))) break;
            }
        }
        x[i] = t;
        legendre_upto(N, t, P);
        PN[i] = P[N];
    }
    for (int i = 0; i <= N; i++) {
        if (xi) xi[i] = (double)x[i];
        if (rho) rho[i] = (double)(2.0L / ((long double)N * (N + 1) * PN[i] * PN[i]));
    }
    if (D) {
        for (int i = 0; i <= N; i++)
            for (int j = 0; j <= N; j++) {
                long double v;
                if (i != j)
                    v = PN[i] / (PN[j] * (x[i] - x[j]));
                else if (i == 0)
                    v = -0.25L * N * (N + 1);
                else if (i == N)
                    v = 0.25L * N * (N + 1);
                else
                    v = 0.0L;
                D[i * lx + j] = (double)v;
            }
    }
}

// ---------------------------------------------------------------------------
// set-up kernels (one thread per local point; run once, not on the hot path)
// ---------------------------------------------------------------------------
struct GeomArgs {
    const double* X;      // [3][n_local] (of this part)
    const double* h1;     // [n_local] or null
    const double* D;      // [lx][lx]
    const double* rho;    // [lx]
    double* G;            // [E][6][lx^3] (this part)
    double* B;            // [n_local]
    double* drdx;         // [E][9][lx^3] dr_s/dx_l (s major) of this part, or null
    int E, lx;
    int* bad;             // set to 1 on a non-positive Jacobian
};

__global__ void geometry_kernel(GeomArgs a) {
    const int lx = a.lx, n3 = lx * lx * lx;
    const int64_t n = (int64_t)a.E * n3;
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n;
         L += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = L / n3;
        const int q = (int)(L - e * n3);
        const int i = q % lx, j = (q / lx) % lx, k = q / (lx * lx);
        double d[3][3];
        for (int m = 0; m < 3; m++) {
            const double* c = a.X + (int64_t)m * n + e * n3;
            double dr = 0.0, ds = 0.0, dt = 0.0;
            for (int l = 0; l < lx; l++) {
                dr = fma(a.D[i * lx + l], c[(k * lx + j) * lx + l], dr);
                ds = fma(a.D[j * lx + l], c[(k * lx + l) * lx + i], ds);
                dt = fma(a.D[k * lx + l], c[(l * lx + j) * lx + i], dt);
            }
            d[m][0] = dr;
            d[m][1] = ds;
            d[m][2] = dt;
        }
        // cofactors of the Jacobian matrix dx/dr (rows x,y,z; columns r,s,t)
        const double c00 = d[1][1] * d[2][2] - d[1][2] * d[2][1];
        const double c01 = d[1][2] * d[2][0] - d[1][0] * d[2][2];
        const double c02 = d[1][0] * d[2][1] - d[1][1] * d[2][0];
        const double J = d[0][0] * c00 + d[0][1] * c01 + d[0][2] * c02;
        if (!(J > 0.0)) {
            *a.bad = 1;
            continue;
        }
        // gradients of r, s, t: rows of the inverse = columns of adj / J
        double g[3][3];
        g[0][0] = c00;
        g[0][1] = d[0][2] * d[2][1] - d[0][1] * d[2][2];
        g[0][2] = d[0][1] * d[1][2] - d[0][2] * d[1][1];
        g[1][0] = c01;
        g[1][1] = d[0][0] * d[2][2] - d[0][2] * d[2][0];
        g[1][2] = d[0][2] * d[1][0] - d[0][0] * d[1][2];
        g[2][0] = c02;
        g[2][1] = d[0][1] * d[2][0] - d[0][0] * d[2][1];
        g[2][2] = d[0][0] * d[1][1] - d[0][1] * d[1][0];
        const double wq = a.rho[i] * a.rho[j] * a.rho[k];
        const double hh = a.h1 ? a.h1[L] : 1.0;
        // G_st = w J (grad r_s . grad r_t) = w (adj_s . adj_t) / J
        const double s = wq * hh / J;
        double* Ge = a.G + e * 6 * n3 + q;
        const int ss[6] = {0, 0, 0, 1, 1, 2}, tt[6] = {0, 1, 2, 1, 2, 2};
        for (int c = 0; c < 6; c++) {
            const double dot = g[ss[c]][0] * g[tt[c]][0] + g[ss[c]][1] * g[tt[c]][1] +
                               g[ss[c]][2] * g[tt[c]][2];
            Ge[c * n3] = s * dot;
        }
        a.B[L] = wq * J;
        if (a.drdx) {
            double* Me = a.drdx + e * 9 * n3 + q;
            for (int c = 0; c < 9; c++) Me[c * n3] = g[c / 3][c % 3] / J;
        }
    }
}

// Local diagonal of A^e with the folded factors (h1 G):
// d = sum_l D_li^2 G11(l,j,k) + D_lj^2 G22(i,l,k) + D_lk^2 G33(i,j,l)
//   + 2 (D_ii D_jj G12 + D_ii D_kk G13 + D_jj D_kk G23)(i,j,k)
__global__ void jacobi_local_kernel(const double* G, const double* D, int E, int lx, double* d) {
    const int n3 = lx * lx * lx;
    const int64_t n = (int64_t)E * n3;
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n;
         L += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = L / n3;
        const int q = (int)(L - e * n3);
        const int i = q % lx, j = (q / lx) % lx, k = q / (lx * lx);
        const double* Ge = G + e * 6 * n3;
        double s = 0.0;
        for (int l = 0; l < lx; l++) {
            const double a = D[l * lx + i], b = D[l * lx + j], c = D[l * lx + k];
            s = fma(a * a, Ge[0 * n3 + (k * lx + j) * lx + l], s);
            s = fma(b * b, Ge[3 * n3 + (k * lx + l) * lx + i], s);
            s = fma(c * c, Ge[5 * n3 + (l * lx + j) * lx + i], s);
        }
        const double dii = D[i * lx + i], djj = D[j * lx + j], dkk = D[k * lx + k];
        s += 2.0 * (dii * djj * Ge[1 * n3 + q] + dii * dkk * Ge[2 * n3 + q] + djj * dkk * Ge[4 * n3 + q]);
        d[L] = s;
    }
}

__global__ void jacobi_invert_kernel(const double* d, const uint8_t* mask, int64_t n, double* minv,
                                     float* minv32) {
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n;
         L += (int64_t)gridDim.x * blockDim.x) {
        const double v = mask[L] ? 1.0 / d[L] : 0.0;
        minv[L] = v;
        minv32[L] = (float)v;
    }
}

// G2[e][c][q] = hi(G[e][c][q]), G2[e][6 + c][q] = lo = float(G - hi)
__global__ void split_factors_kernel(const double* G, float* G2, int64_t nelem_planes, int n3) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nelem_planes * n3;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ec = t / n3;  // element * 6 + c
        const int q = (int)(t - ec * n3);
        const int64_t e = ec / 6;
        const int c = (int)(ec - e * 6);
        const double v = G[t];
        const float hi = (float)v;
        G2[(e * 12 + c) * n3 + q] = hi;
        G2[(e * 12 + 6 + c) * n3 + q] = (float)(v - (double)hi);
    }
}

__global__ void to_float_kernel(const double* a, float* b, int64_t n) {
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n;
         L += (int64_t)gridDim.x * blockDim.x)
        b[L] = (float)a[L];
}

// ---------------------------------------------------------------------------
// host: stable LSD radix sort of (key, local index) pairs by key
// ---------------------------------------------------------------------------
static void radix_sort_pairs(std::vector<uint64_t>& key, std::vector<int32_t>& val) {
    const size_t n = key.size();
    if (n < 2) return;
    uint64_t mx = 0;
    for (uint64_t k : key) mx = std::max(mx, k);
    int bits = 0;
    while (bits < 64 && (mx >> bits) != 0) bits++;
    std::vector<uint64_t> k2(n);
    std::vector<int32_t> v2(n);
    std::vector<size_t> cnt(1 << 16);
    for (int shift = 0; shift < bits; shift += 16) {
        std::fill(cnt.begin(), cnt.end(), 0);
        for (size_t q = 0; q < n; q++) cnt[(key[q] >> shift) & 0xFFFF]++;
        size_t acc = 0;
        for (auto& c : cnt) {
            size_t t = c;
            c = acc;
            acc += t;
        }
        for (size_t q = 0; q < n; q++) {
            size_t pos = cnt[(key[q] >> shift) & 0xFFFF]++;
            k2[pos] = key[q];
            v2[pos] = val[q];
        }
        key.swap(k2);
        val.swap(v2);
    }
}

// Gather-scatter lists of one mesh, appended to host vectors (indices offset
// by loc_off).  Returns SEM_OK or SEM_EINVAL.
struct HostGS {
    std::vector<int32_t> free_off, free_idx, dir_off, dir_idx, zero;
    std::vector<uint8_t> mult;
};

static int build_gs_part(const MeshPart& part, int solve, const int64_t* gid, const uint8_t* mask,
                         HostGS& out, int64_t* n_unique, int64_t* n_free) {
    const int64_t n = part.n_local;
    int64_t gmin = INT64_MAX;
    for (int64_t L = 0; L < n; L++) gmin = std::min(gmin, gid[L]);
    std::vector<uint64_t> key(n);
    std::vector<int32_t> val(n);
    for (int64_t L = 0; L < n; L++) {
        key[L] = (uint64_t)(gid[L] - gmin);
        val[L] = (int32_t)L;
    }
    radix_sort_pairs(key, val);
    int64_t nu = 0, nf = 0;
    for (int64_t a = 0; a < n;) {
        int64_t b = a + 1;
        while (b < n && key[b] == key[a]) b++;
        const int cnt = (int)(b - a);
        if (cnt > 255) return fail(SEM_EINVAL, "a node has more than 255 local copies");
        const uint8_t m0 = mask[val[a]] ? 1 : 0;
        for (int64_t c = a; c < b; c++) {
            if ((mask[val[c]] ? 1 : 0) != m0)
                return fail(SEM_EINVAL, "Dirichlet mask differs between copies of a node");
            out.mult[part.loc_off + val[c]] = (uint8_t)cnt;
        }
        nu++;
        if (m0) nf++;
        if (cnt >= 2) {
            auto& off = m0 ? out.free_off : out.dir_off;
            auto& idx = m0 ? out.free_idx : out.dir_idx;
            off.push_back((int32_t)idx.size());
            for (int64_t c = a; c < b; c++) idx.push_back((int32_t)(part.loc_off + val[c]));
        } else if (!m0) {
            out.zero.push_back((int32_t)(part.loc_off + val[a]));
        }
        a = b;
    }
    *n_unique = nu;
    *n_free = nf;
    return SEM_OK;
}

static void free_handle(sem_handle* h) {
    if (!h) return;
    for (int l = 0; l <= kMaxLx; l++) {
        cudaFree(h->D64[l]);
        cudaFree(h->D32[l]);
        cudaFree(h->D2[l]);
    }
    cudaFree(h->G64);
    cudaFree(h->drdx);
    cudaFree(h->G32);
    cudaFree(h->G2);
    cudaFree(h->B64);
    cudaFree(h->minv64);
    cudaFree(h->hmass64);
    cudaFree(h->hmass32);
    cudaFree(h->minv32);
    cudaFree(h->mult);
    cudaFree(h->mask);
    GSLists& gl = h->gs;
    cudaFree(gl.pairs); cudaFree(gl.quads); cudaFree(gl.octs); cudaFree(gl.oth_off); cudaFree(gl.oth_idx);
    cudaFree(gl.dir_off); cudaFree(gl.dir_idx); cudaFree(gl.zero_idx);
    cudaFree(h->partials);
    cudaFree(h->counters);
    cudaFree(h->state);
    cudaFree(h->scratch);
    if (h->state_host) cudaFreeHost(h->state_host);
    if (h->loop_host) cudaFreeHost(h->loop_host);
    Workspace& w = h->ws;
    cudaFree(w.r); cudaFree(w.p); cudaFree(w.z); cudaFree(w.w); cudaFree(w.x); cudaFree(w.b);
    cudaFree(w.r32); cudaFree(w.p32); cudaFree(w.z32); cudaFree(w.w32); cudaFree(w.d32); cudaFree(w.b32);
    for (float* pv : w.pv) cudaFree(pv);
    for (double* pp : w.pipe) cudaFree(pp);
    BatchPlan& bp = h->batch;
    for (auto& g : bp.lxg) {
        cudaFree(g.loc); cudaFree(g.cnt); cudaFree(g.solve);
    }
    for (auto& bs : bp.bulk) {
        for (auto& g : bs.lists) {
            cudaFree(g.loc); cudaFree(g.cnt); cudaFree(g.solve);
        }
        cudaFree(bs.sgfirst); cudaFree(bs.sgcount); cudaFree(bs.gpart);
    }
    cudaFree(bp.uloc); cudaFree(bp.ucnt); cudaFree(bp.usolve); cudaFree(bp.ulx);
    for (auto* p : bp.sid) cudaFree(p);
    cudaFree(bp.sgfirst); cudaFree(bp.sgcount); cudaFree(bp.tloc); cudaFree(bp.tlen); cudaFree(bp.tsolve);
    cudaFree(bp.stfirst); cudaFree(bp.stcount); cudaFree(bp.gpart); cudaFree(bp.tpart); cudaFree(bp.scount);
    cudaFree(bp.rrbb); cudaFree(bp.act); cudaFree(bp.itol); cudaFree(bp.carry);
    free_projection(h);
    free_schwarz(h);
    if (h->graph.exec) cudaGraphExecDestroy(h->graph.exec);
    if (h->graph_tail.exec) cudaGraphExecDestroy(h->graph_tail.exec);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    for (auto& ev : h->ax_ev)
        if (ev) cudaEventDestroy(ev);
    delete h;
}

int ensure_workspace(sem_handle* h, bool fp32) {
    Workspace& w = h->ws;
    const size_t n = (size_t)h->n_local;
    int rc;
    if (!w.have64) {
        if ((rc = dalloc(h, &w.r, n)) || (rc = dalloc(h, &w.p, n)) || (rc = dalloc(h, &w.z, n)) ||
            (rc = dalloc(h, &w.w, n)) || (rc = dalloc(h, &w.x, n)) || (rc = dalloc(h, &w.b, n)))
            return rc;
        w.have64 = true;
    }
    if (fp32 && !w.have32) {
        if ((rc = dalloc(h, &w.r32, n)) || (rc = dalloc(h, &w.p32, n)) || (rc = dalloc(h, &w.z32, n)) ||
            (rc = dalloc(h, &w.w32, n)) || (rc = dalloc(h, &w.d32, n)) || (rc = dalloc(h, &w.b32, n)))
            return rc;
        w.have32 = true;
    }
    return SEM_OK;
}

static bool host_pointer(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

static int setup_common(sem_handle** out, int nsolve, const sem_mesh_desc* meshes, int flags, cudaStream_t s) {
    *out = nullptr;
    if (nsolve < 1 || !meshes) return fail(SEM_EINVAL, "nsolve must be >= 1");
    int64_t n_local = 0, E = 0;
    for (int q = 0; q < nsolve; q++) {
        const sem_mesh_desc& m = meshes[q];
        if (m.E < 1 || m.lx < 2 || m.lx > kMaxLx)
            return fail(SEM_EINVAL, "each mesh needs E >= 1 and 2 <= lx <= 16");
        if (!m.coords || !m.gid || !m.mask) return fail(SEM_EINVAL, "coords, gid and mask are required");
        if (!host_pointer(m.coords) || !host_pointer(m.gid) || !host_pointer(m.mask) ||
            (m.h1 && !host_pointer(m.h1)))
            return fail(SEM_EINVAL, "set-up arrays must be host pointers");
        n_local += (int64_t)m.E * m.lx * m.lx * m.lx;
        E += m.E;
    }
    if (n_local >= ((int64_t)1 << 31) - 64)
        return fail(SEM_EINVAL, "n_local must be below 2^31 (32-bit local indices)");
    const int forced = (flags & 0xF) - 1;  // pinned operator variant, -1 = autotune
    if (forced > kLnVariant || forced == kMultiVariant) return fail(SEM_EINVAL, "operator variant out of range");
    sem_handle* h = new sem_handle();
    // a pinned variant 0..4 serves the FP64 and FP32 classes, 5 or 6 the pair
    // class, 8 the FP32 class, 9 the FP64 class; the other classes stay autotuned
    for (int cls = 0; cls < 3; cls++) {
        const bool pair_pin = forced == kDfVariant || forced == kDflVariant;
        const bool applies = forced >= 0 && ((cls == kClsPair) == pair_pin) &&
                             (forced != kTcVariant || cls == kClsF32) && (forced != kLnVariant || cls == kClsF64);
        for (int& v : h->ax_variant[cls]) v = applies ? forced : -1;
    }
    h->test_stall = (flags & SEM_FLAG_TEST_STALL) ? 1 : 0;
    int rc = SEM_OK;
    auto bail = [&](int code) {
        free_handle(h);
        return code;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) return bail(fail(SEM_ECUDA, "no CUDA device"));
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    h->nsolve = nsolve;
    h->E = (int)E;
    h->n_local = n_local;
    h->lx = meshes[0].lx;
    for (int q = 1; q < nsolve; q++)
        if (meshes[q].lx != h->lx) h->lx = 0;
    // parts
    int64_t eoff = 0, loff = 0;
    for (int q = 0; q < nsolve; q++) {
        MeshPart p;
        p.E = meshes[q].E;
        p.lx = meshes[q].lx;
        p.elem_off = eoff;
        p.loc_off = loff;
        p.n_local = (int64_t)p.E * p.lx * p.lx * p.lx;
        h->parts.push_back(p);
        eoff += p.E;
        loff += p.n_local;
    }
    // gather-scatter lists
    HostGS hg;
    hg.mult.assign(n_local, 1);
    std::vector<uint8_t> mask_all(n_local);
    for (int q = 0; q < nsolve; q++) {
        MeshPart& p = h->parts[q];
        if ((rc = build_gs_part(p, q, meshes[q].gid, meshes[q].mask, hg, &p.n_unique, &p.n_free)))
            return bail(rc);
        for (int64_t L = 0; L < p.n_local; L++) mask_all[p.loc_off + L] = meshes[q].mask[L] ? 1 : 0;
        h->n_unique += p.n_unique;
        h->n_free += p.n_free;
    }
    GSLists& g = h->gs;
    // free segments by size class, each class ordered by first local index
    std::vector<int2> pairs;
    std::vector<int4> quads, octs;
    std::vector<int32_t> oth_off, oth_idx, dir_off, dir_idx, zero;
    {
        const int64_t nf = (int64_t)hg.free_off.size();
        std::vector<std::pair<int32_t, int64_t>> order(nf);
        for (int64_t q = 0; q < nf; q++) order[q] = {hg.free_idx[hg.free_off[q]], q};
        std::sort(order.begin(), order.end());
        for (auto& o : order) {
            const int64_t q = o.second;
            const int32_t a = hg.free_off[q];
            const int32_t b = q + 1 < nf ? hg.free_off[q + 1] : (int32_t)hg.free_idx.size();
            const int32_t* ix = hg.free_idx.data() + a;
            const int c = b - a;
            if (c == 2) {
                pairs.push_back(make_int2(ix[0], ix[1]));
            } else if (c == 4) {
                quads.push_back(make_int4(ix[0], ix[1], ix[2], ix[3]));
            } else if (c == 8) {
                octs.push_back(make_int4(ix[0], ix[1], ix[2], ix[3]));
                octs.push_back(make_int4(ix[4], ix[5], ix[6], ix[7]));
            } else {
                oth_off.push_back((int32_t)oth_idx.size());
                oth_idx.insert(oth_idx.end(), ix, ix + c);
            }
        }
        oth_off.push_back((int32_t)oth_idx.size());
        const int64_t nd = (int64_t)hg.dir_off.size();
        for (int64_t q = 0; q < nd; q++) {
            const int32_t a = hg.dir_off[q];
            const int32_t b = q + 1 < nd ? hg.dir_off[q + 1] : (int32_t)hg.dir_idx.size();
            dir_off.push_back((int32_t)dir_idx.size());
            dir_idx.insert(dir_idx.end(), hg.dir_idx.begin() + a, hg.dir_idx.begin() + b);
        }
        dir_off.push_back((int32_t)dir_idx.size());
        zero = hg.zero;
        zero.insert(zero.end(), hg.dir_idx.begin(), hg.dir_idx.end());
        std::sort(zero.begin(), zero.end());
    }
    g.npair = (int64_t)pairs.size();
    g.nquad = (int64_t)quads.size();
    g.noct = (int64_t)octs.size() / 2;
    g.noth = (int64_t)oth_off.size() - 1;
    g.ndir = (int64_t)dir_off.size() - 1;
    g.nzero = (int64_t)zero.size();
    g.n_shared = (int64_t)(hg.free_idx.size() + hg.dir_idx.size());
    if ((rc = dalloc(h, &g.pairs, pairs.size() + 1)) || (rc = dalloc(h, &g.quads, quads.size() + 1)) ||
        (rc = dalloc(h, &g.octs, octs.size() + 2)) || (rc = dalloc(h, &g.oth_off, oth_off.size())) ||
        (rc = dalloc(h, &g.oth_idx, oth_idx.size() + 1)) || (rc = dalloc(h, &g.dir_off, dir_off.size())) ||
        (rc = dalloc(h, &g.dir_idx, dir_idx.size() + 1)) || (rc = dalloc(h, &g.zero_idx, zero.size() + 1)) ||
        (rc = dalloc(h, &h->mult, n_local)) || (rc = dalloc(h, &h->mask, n_local)) ||
        (rc = dalloc(h, &h->G64, (size_t)6 * n_local)) || (rc = dalloc(h, &h->G32, (size_t)6 * n_local)) ||
        (rc = dalloc(h, &h->G2, (size_t)12 * n_local)) ||
        (rc = dalloc(h, &h->B64, n_local)) || (rc = dalloc(h, &h->minv64, n_local)) ||
        (rc = dalloc(h, &h->minv32, n_local)) || (rc = dalloc(h, &h->partials, (size_t)kMaxPartials * 4)) ||
        (rc = dalloc(h, &h->counters, 16)) || (rc = dalloc(h, &h->state, (size_t)2 * nsolve + 2)) ||
        (rc = dalloc(h, &h->scratch, 64)))
        return bail(rc);
    if ((flags & SEM_FLAG_METRICS) && (rc = dalloc(h, &h->drdx, (size_t)9 * n_local))) return bail(rc);
    if (cudaMallocHost((void**)&h->state_host, sizeof(CGState) * (2 * nsolve + 2)) != cudaSuccess ||
        cudaMallocHost((void**)&h->loop_host, sizeof(LoopReadback)) != cudaSuccess)
        return bail(fail(SEM_ENOMEM, "cudaMallocHost failed"));
#define UP(dst, src, bytes)                                                               \
    do {                                                                                  \
        if ((bytes) > 0) {                                                                \
            cudaError_t e_ = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s); \
            if (e_ != cudaSuccess) return bail(cuda_fail(e_, "upload"));                  \
        }                                                                                 \
    } while (0)
    UP(g.pairs, pairs.data(), pairs.size() * sizeof(int2));
    UP(g.quads, quads.data(), quads.size() * sizeof(int4));
    UP(g.octs, octs.data(), octs.size() * sizeof(int4));
    UP(g.oth_off, oth_off.data(), oth_off.size() * 4);
    UP(g.oth_idx, oth_idx.data(), oth_idx.size() * 4);
    UP(g.dir_off, dir_off.data(), dir_off.size() * 4);
    UP(g.dir_idx, dir_idx.data(), dir_idx.size() * 4);
    UP(g.zero_idx, zero.data(), zero.size() * 4);
    UP(h->mult, hg.mult.data(), (size_t)n_local);
    UP(h->mask, mask_all.data(), (size_t)n_local);
    if (cudaMemsetAsync(h->counters, 0, 16 * sizeof(unsigned), s) != cudaSuccess ||
        cudaMemsetAsync(h->scratch, 0, 64 * sizeof(double), s) != cudaSuccess)
        return bail(fail(SEM_ECUDA, "memset"));
    // basis per order
    for (int q = 0; q < nsolve; q++) {
        const int lx = h->parts[q].lx;
        if (h->D64[lx]) continue;
        double Dh[kMaxLx * kMaxLx];
        float Df[kMaxLx * kMaxLx], D2[2 * kMaxLx * kMaxLx];
        gll_basis(lx, nullptr, nullptr, Dh);
        for (int t = 0; t < lx * lx; t++) {
            Df[t] = (float)Dh[t];
            D2[t] = Df[t];
            D2[lx * lx + t] = (float)(Dh[t] - (double)Df[t]);
        }
        if ((rc = dalloc(h, &h->D64[lx], (size_t)lx * lx)) || (rc = dalloc(h, &h->D32[lx], (size_t)lx * lx)) ||
            (rc = dalloc(h, &h->D2[lx], (size_t)2 * lx * lx)))
            return bail(rc);
        UP(h->D64[lx], Dh, sizeof(double) * lx * lx);
        UP(h->D32[lx], Df, sizeof(float) * lx * lx);
        if ((rc = bulk_set_d_f64(Dh, lx)) || (rc = bulk_set_d_f32(Df, lx))) return bail(rc);
        UP(h->D2[lx], D2, sizeof(float) * 2 * lx * lx);
        if (lx % 2 == 0 && lx >= 4 && lx <= 12) {
            // even/odd line coefficients: [dir][A/B][hi/lo][P][P], dir 0 = D, 1 = D^T,
            // A_im = (M_im - M_{i,N-m}) / 2, B_im = (M_im + M_{i,N-m}) / 2
            const int P = lx / 2, N = lx - 1;
            std::vector<float> cf(8 * P * P);
            for (int dir = 0; dir < 2; dir++)
                for (int i = 0; i < P; i++)
                    for (int m = 0; m < P; m++) {
                        auto M = [&](int r, int c) { return dir == 0 ? Dh[r * lx + c] : Dh[c * lx + r]; };
                        const double A = 0.5 * (M(i, m) - M(i, N - m)), B = 0.5 * (M(i, m) + M(i, N - m));
                        const float Ah = (float)A, Bh = (float)B;
                        cf[((dir * 2 + 0) * 2 + 0) * P * P + i * P + m] = Ah;
                        cf[((dir * 2 + 0) * 2 + 1) * P * P + i * P + m] = (float)(A - (double)Ah);
                        cf[((dir * 2 + 1) * 2 + 0) * P * P + i * P + m] = Bh;
                        cf[((dir * 2 + 1) * 2 + 1) * P * P + i * P + m] = (float)(B - (double)Bh);
                    }
            if ((rc = dfl_set_coef(cf.data(), lx))) return bail(rc);
            // the same tables in FP64 for the native line-transform operator: [dir][A/B][P][P]
            std::vector<double> cd(4 * P * P);
            for (int dir = 0; dir < 2; dir++)
                for (int i = 0; i < P; i++)
                    for (int m = 0; m < P; m++) {
                        auto M = [&](int r, int c) { return dir == 0 ? Dh[r * lx + c] : Dh[c * lx + r]; };
                        cd[(dir * 2 + 0) * P * P + i * P + m] = 0.5 * (M(i, m) - M(i, N - m));
                        cd[(dir * 2 + 1) * P * P + i * P + m] = 0.5 * (M(i, m) + M(i, N - m));
                    }
            if ((rc = ln_set_coef(cd.data(), lx))) return bail(rc);
        }
    }
    // geometry, mass, Jacobi diagonal: one part at a time through a staging buffer
    int64_t maxn = 0;
    for (auto& p : h->parts) maxn = std::max(maxn, p.n_local);
    double *dX = nullptr, *dh1 = nullptr, *drho = nullptr, *dd = nullptr;
    int* dbad = nullptr;
    cudaError_t e1 = cudaMalloc((void**)&dX, sizeof(double) * 3 * maxn);
    cudaError_t e2 = cudaMalloc((void**)&dh1, sizeof(double) * maxn);
    cudaError_t e3 = cudaMalloc((void**)&drho, sizeof(double) * kMaxLx);
    cudaError_t e4 = cudaMalloc((void**)&dbad, sizeof(int));
    cudaError_t e5 = cudaMalloc((void**)&dd, sizeof(double) * n_local);
    auto free_tmp = [&]() {
        cudaFree(dX); cudaFree(dh1); cudaFree(drho); cudaFree(dbad); cudaFree(dd);
    };
    if (e1 || e2 || e3 || e4 || e5) {
        free_tmp();
        cudaGetLastError();
        return bail(fail(SEM_ENOMEM, "set-up staging allocation failed"));
    }
    int bad = 0;
    cudaMemsetAsync(dbad, 0, sizeof(int), s);
    for (int q = 0; q < nsolve && rc == SEM_OK; q++) {
        const MeshPart& p = h->parts[q];
        double rho[kMaxLx];
        gll_basis(p.lx, nullptr, rho, nullptr);
        cudaMemcpyAsync(drho, rho, sizeof(double) * p.lx, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(dX, meshes[q].coords, sizeof(double) * 3 * p.n_local, cudaMemcpyHostToDevice, s);
        if (meshes[q].h1)
            cudaMemcpyAsync(dh1, meshes[q].h1, sizeof(double) * p.n_local, cudaMemcpyHostToDevice, s);
        GeomArgs a;
        a.X = dX;
        a.h1 = meshes[q].h1 ? dh1 : nullptr;
        a.D = h->D64[p.lx];
        a.rho = drho;
        a.G = h->G64 + 6 * p.loc_off;
        a.drdx = h->drdx ? h->drdx + 9 * p.loc_off : nullptr;
        a.B = h->B64 + p.loc_off;
        a.E = p.E;
        a.lx = p.lx;
        a.bad = dbad;
        geometry_kernel<<<grid_for(h, p.n_local, 256, 8), 256, 0, s>>>(a);
        jacobi_local_kernel<<<grid_for(h, p.n_local, 256, 8), 256, 0, s>>>(
            h->G64 + 6 * p.loc_off, h->D64[p.lx], p.E, p.lx, dd + p.loc_off);
        // the staging buffers are reused by the next part: wait for this one
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "geometry kernels");
    }
    if (rc == SEM_OK) {
        cudaMemcpyAsync(&bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        if (bad) rc = fail(SEM_EINVAL, "non-positive Jacobian at some node (tangled or left-handed element)");
    }
    if (rc == SEM_OK) rc = launch_gs(h, dd, false, false, s);
    if (rc == SEM_OK) {
        jacobi_invert_kernel<<<grid_for(h, n_local, 256, 8), 256, 0, s>>>(dd, h->mask, n_local, h->minv64,
                                                                           h->minv32);
        to_float_kernel<<<grid_for(h, 6 * n_local, 256, 8), 256, 0, s>>>(h->G64, h->G32, 6 * n_local);
        for (const MeshPart& p : h->parts) {
            const int n3 = p.lx * p.lx * p.lx;
            split_factors_kernel<<<grid_for(h, 6 * p.n_local, 256, 8), 256, 0, s>>>(
                h->G64 + 6 * p.loc_off, h->G2 + 12 * p.loc_off, (int64_t)6 * p.E, n3);
        }
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "jacobi set-up");
    }
    free_tmp();
    if (rc != SEM_OK) return bail(rc);
    *out = h;
    return SEM_OK;
#undef UP
}

// ---------------------------------------------------------------------------
// Two-level Schwarz preconditioner set-up (host; the data for sem_gmres.cu)
// ---------------------------------------------------------------------------

// Eigenvalues and eigenvectors of a small symmetric matrix by cyclic Jacobi
// rotations (Golub and Van Loan, Sec. 8.5): A (n x n, row major) is
// overwritten; on return lam[m] and V[:, m] (V row major: V[i * n + m]).
static void sym_eigen(int n, std::vector<double>& A, std::vector<double>& lam, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; i++) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < n; p++)
            for (int q = 0; q < n; q++) (p == q ? diag : off) += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (off <= 1e-30 * diag) break;
        for (int p = 0; p < n - 1; p++)
            for (int q = p + 1; q < n; q++) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; k++) {  // columns p, q of A
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - sn * akq;
                    A[(size_t)k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {  // rows p, q
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - sn * aqk;
                    A[(size_t)q * n + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; k++) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - sn * vkq;
                    V[(size_t)k * n + q] = sn * vkp + c * vkq;
                }
            }
    }
    lam.resize(n);
    for (int i = 0; i < n; i++) lam[i] = A[(size_t)i * n + i];
}

// SEM_FLAG_SCHWARZ: box lengths and mean h1 per element, the coarse handle on
// the element corners, the reference interior modes (K S = W S Lambda,
// S^T W S = I on the interior GLL nodes) and the trilinear corner weights.
static int build_schwarz(sem_handle* h, const sem_mesh_desc& m, cudaStream_t s) {
    SchwarzData& sc = h->sch;
    const int lx = m.lx, N = lx - 1, n3 = lx * lx * lx, E = m.E;
    const int64_t n = (int64_t)E * n3;
    int corner[8];
    for (int q = 0; q < 8; q++) {
        const int i = (q & 1) ? N : 0, j = ((q >> 1) & 1) ? N : 0, k = ((q >> 2) & 1) ? N : 0;
        corner[q] = (k * lx + j) * lx + i;
    }
    std::vector<double> L((size_t)E * 3), h1m((size_t)E), cc((size_t)3 * E * 8), ch1;
    std::vector<int64_t> cg((size_t)E * 8);
    std::vector<uint8_t> cm((size_t)E * 8);
    if (m.h1) ch1.resize((size_t)E * 8);
    for (int e = 0; e < E; e++) {
        for (int q = 0; q < 8; q++) {
            const int64_t Lq = (int64_t)e * n3 + corner[q];
            for (int d = 0; d < 3; d++) cc[((size_t)d * E + e) * 8 + q] = m.coords[d * n + Lq];
            cg[(size_t)e * 8 + q] = m.gid[Lq];
            cm[(size_t)e * 8 + q] = m.mask[Lq];
            if (m.h1) ch1[(size_t)e * 8 + q] = m.h1[Lq];
        }
        for (int d = 0; d < 3; d++) {  // mean length of the element's four edges along direction d
            double acc = 0.0;
            for (int q = 0; q < 8; q++) {
                if ((q >> d) & 1) continue;
                const int q2 = q | (1 << d);
                double d2 = 0.0;
                for (int c = 0; c < 3; c++) {
                    const double dx = cc[((size_t)c * E + e) * 8 + q2] - cc[((size_t)c * E + e) * 8 + q];
                    d2 += dx * dx;
                }
                acc += std::sqrt(d2);
            }
            L[(size_t)e * 3 + d] = acc / 4.0;
        }
        double hs = 0.0;
        for (int q = 0; q < n3; q++) hs += m.h1 ? m.h1[(int64_t)e * n3 + q] : 1.0;
        h1m[e] = hs / n3;
    }
    sem_mesh_desc cmd;
    cmd.E = E;
    cmd.lx = 2;
    cmd.coords = cc.data();
    cmd.gid = cg.data();
    cmd.mask = cm.data();
    cmd.h1 = m.h1 ? ch1.data() : nullptr;
    int rc = setup_common(&sc.coarse, 1, &cmd, 0, s);
    if (!rc) rc = ensure_workspace(sc.coarse, false);
    if (!rc) rc = build_coarse_csr(h, cg.data(), cm.data());
    if (rc) return rc;
    // reference interior problem and trilinear weights
    std::vector<double> xi(lx), rho(lx), D((size_t)lx * lx);
    gll_basis(lx, xi.data(), rho.data(), D.data());
    const int ni = lx - 2;
    std::vector<double> S, lam;
    if (ni > 0) {
        std::vector<double> C((size_t)ni * ni);
        for (int a = 0; a < ni; a++)
            for (int b = 0; b < ni; b++) {
                double kab = 0.0;  // K = D^T diag(rho) D on [-1, 1], interior rows and columns
                for (int l = 0; l < lx; l++) kab += D[(size_t)l * lx + a + 1] * rho[l] * D[(size_t)l * lx + b + 1];
                C[(size_t)a * ni + b] = kab / std::sqrt(rho[a + 1] * rho[b + 1]);
            }
        std::vector<double> Vm;
        sym_eigen(ni, C, lam, Vm);
        S.resize((size_t)ni * ni);
        for (int a = 0; a < ni; a++)
            for (int b = 0; b < ni; b++) S[(size_t)a * ni + b] = Vm[(size_t)a * ni + b] / std::sqrt(rho[a + 1]);
    }
    std::vector<double> Pw((size_t)n3 * 8);
    for (int q = 0; q < n3; q++) {
        const int i = q % lx, j = (q / lx) % lx, k = q / (lx * lx);
        for (int c = 0; c < 8; c++) {
            const double fi = (c & 1) ? (1.0 + xi[i]) / 2.0 : (1.0 - xi[i]) / 2.0;
            const double fj = ((c >> 1) & 1) ? (1.0 + xi[j]) / 2.0 : (1.0 - xi[j]) / 2.0;
            const double fk = ((c >> 2) & 1) ? (1.0 + xi[k]) / 2.0 : (1.0 - xi[k]) / 2.0;
            Pw[(size_t)q * 8 + c] = fi * fj * fk;
        }
    }
    // per-element factors of the fast-diagonalisation solve: sqrt(2 / L_d) for
    // the three directions, then h1m 4 / L_d^2 (the box's 1-D stiffness scale)
    std::vector<double> fac((size_t)E * 6);
    for (int e = 0; e < E; e++)
        for (int d = 0; d < 3; d++) {
            const double Ld = L[(size_t)e * 3 + d];
            fac[(size_t)e * 6 + d] = std::sqrt(2.0 / Ld);
            fac[(size_t)e * 6 + 3 + d] = h1m[e] * 4.0 / (Ld * Ld);
        }
    if ((rc = dalloc(h, &sc.fac, fac.size())) || (rc = dalloc(h, &sc.fac32, fac.size())) ||
        (rc = dalloc(h, &sc.Pw, Pw.size())) || (rc = dalloc(h, &sc.Pw32, Pw.size())) ||
        (ni > 0 && ((rc = dalloc(h, &sc.S, S.size())) || (rc = dalloc(h, &sc.lam, lam.size())) ||
                    (rc = dalloc(h, &sc.S32, S.size())) || (rc = dalloc(h, &sc.lam32, lam.size())))))
        return rc;
    auto put = [](double* d, float* d32, const std::vector<double>& v) -> int {
        std::vector<float> f(v.begin(), v.end());
        SEM_CUDA_TRY(cudaMemcpy(d, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice));
        SEM_CUDA_TRY(cudaMemcpy(d32, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice));
        return SEM_OK;
    };
    if ((rc = put(sc.fac, sc.fac32, fac)) || (rc = put(sc.Pw, sc.Pw32, Pw))) return rc;
    if (ni > 0 && ((rc = put(sc.S, sc.S32, S)) || (rc = put(sc.lam, sc.lam32, lam)))) return rc;
    return SEM_OK;
}

// Helmholtz mass term: hm = h2 B (FP64 and FP32), d += hm on the local diagonal
__global__ void helmholtz_mass_kernel(const double* h2, const double* B, double* hm, float* hm32, double* d,
                                      int64_t n) {
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x) {
        const double v = h2[L] * B[L];
        hm[L] = v;
        hm32[L] = (float)v;
        d[L] += v;
    }
}

// Rebuild the Jacobi diagonal (and the Helmholtz mass term when h2 is given):
// d = diag(A_L) (+ h2 B), d <- QQ^T d, Minv = mask / d.
static int set_helmholtz(sem_handle* h, const double* h2_host, cudaStream_t s) {
    const int64_t n = h->n_local;
    double* dd = nullptr;
    double* dh2 = nullptr;
    int rc = dalloc(h, &dd, (size_t)n);
    if (!rc && h2_host) rc = dalloc(h, &dh2, (size_t)n);
    if (!rc && h2_host && !h->hmass64) {
        rc = dalloc(h, &h->hmass64, (size_t)n);
        if (!rc) rc = dalloc(h, &h->hmass32, (size_t)n);
    }
    auto done = [&](int code) {
        if (dd) { cudaFree(dd); h->device_bytes -= sizeof(double) * n; }
        if (dh2) { cudaFree(dh2); h->device_bytes -= sizeof(double) * n; }
        return code;
    };
    if (rc) return done(rc);
    for (const MeshPart& p : h->parts)
        jacobi_local_kernel<<<grid_for(h, p.n_local, 256, 8), 256, 0, s>>>(h->G64 + 6 * p.loc_off, h->D64[p.lx],
                                                                            p.E, p.lx, dd + p.loc_off);
    if (h2_host) {
        if (cudaMemcpyAsync(dh2, h2_host, sizeof(double) * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return done(cuda_fail(cudaGetLastError(), "copy of h2"));
        helmholtz_mass_kernel<<<grid_for(h, n, 256, 8), 256, 0, s>>>(dh2, h->B64, h->hmass64, h->hmass32, dd, n);
    } else if (h->hmass64) {
        cudaFree(h->hmass64);
        cudaFree(h->hmass32);
        h->hmass64 = nullptr;
        h->hmass32 = nullptr;
        h->device_bytes -= (sizeof(double) + sizeof(float)) * n;
    }
    rc = launch_gs(h, dd, false, false, s);
    if (!rc) {
        jacobi_invert_kernel<<<grid_for(h, n, 256, 8), 256, 0, s>>>(dd, h->mask, n, h->minv64, h->minv32);
        rc = refresh_pair_minv(h, s);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "Helmholtz set-up");
    // captured graphs hold the old operator's arguments; the batch operator
    // configuration is chosen again for the new operator
    for (GraphCache* g : {&h->graph, &h->graph_tail})
        if (g->exec) {
            cudaGraphExecDestroy(g->exec);
            g->exec = nullptr;
        }
    h->batch.kcfg[0] = h->batch.kcfg[1] = -1;
    return done(rc);
}

}  // namespace sem

using namespace sem;

extern "C" {

SEM_API int sem_set_helmholtz(sem_handle* h, const double* h2, cudaStream_t stream) {
    if (!h) return fail(SEM_EINVAL, "null handle");
    if (h2 && !host_pointer(h2)) return fail(SEM_EINVAL, "h2 must be a host pointer");
    if (h2)
        for (int64_t L = 0; L < h->n_local; L++)
            if (!(h2[L] >= 0.0) || !std::isfinite(h2[L]))
                return fail(SEM_EINVAL, "h2 must be finite and non-negative");
    return set_helmholtz(h, h2, stream);
}

SEM_API const char* sem_last_error(void) { return g_err.c_str(); }

SEM_API void sem_solve_opts_default(sem_solve_opts* o) {
    if (!o) return;
    o->tol = 1e-10;
    o->max_iter = 100000;
    o->mode = SEM_MODE_FP64;
    o->inner_tol = 1e-5;
    o->max_outer = 100;
    o->precision = SEM_FP64;
    o->use_graph = 1;
    o->graph_chunk = 32;
    o->autotune = 1;
    o->ir_carry = 0;
    o->persistent = 0;
    o->projection = 0;
    o->tc_split = 0;
    o->pipelined = 0;
    o->gmres_restart = 20;
    o->precond_precision = SEM_FP64;
    o->gmres_orth = 2;
}

SEM_API int sem_gll(int lx, double* xi, double* rho, double* D) {
    if (lx < 2 || lx > kMaxLx) return fail(SEM_EINVAL, "lx must be in [2, 16]");
    gll_basis(lx, xi, rho, D);
    return SEM_OK;
}

SEM_API int sem_setup(sem_handle** h, int E, int lx, const double* coords, const int64_t* gid,
                      const uint8_t* mask, const double* h1, int flags, cudaStream_t stream) {
    if (!h) return fail(SEM_EINVAL, "null handle pointer");
    sem_mesh_desc m;
    m.E = E;
    m.lx = lx;
    m.coords = coords;
    m.gid = gid;
    m.mask = mask;
    m.h1 = h1;
    int rc = setup_common(h, 1, &m, flags & ~SEM_FLAG_SCHWARZ, stream);
    if (rc == SEM_OK && (flags & SEM_FLAG_SCHWARZ) && (rc = build_schwarz(*h, m, stream)) != SEM_OK) {
        free_handle(*h);
        *h = nullptr;
    }
    return rc;
}

SEM_API int sem_setup_batch(sem_handle** h, int nsolve, const sem_mesh_desc* meshes, int flags,
                            cudaStream_t stream) {
    if (!h) return fail(SEM_EINVAL, "null handle pointer");
    return setup_common(h, nsolve, meshes, flags, stream);
}

SEM_API int sem_destroy(sem_handle* h) {
    if (h) {
        cudaDeviceSynchronize();
        free_handle(h);
    }
    return SEM_OK;
}

SEM_API int sem_get_info(const sem_handle* h, sem_info* info) {
    if (!h || !info) return fail(SEM_EINVAL, "null argument");
    info->nsolve = h->nsolve;
    info->E = h->E;
    info->lx = h->lx;
    info->n_local = h->n_local;
    info->n_unique = h->n_unique;
    info->n_free = h->n_free;
    info->n_shared = h->gs.n_shared;
    info->device_bytes = h->device_bytes;
    return SEM_OK;
}

SEM_API int sem_get_offsets(const sem_handle* h, int64_t* offsets) {
    if (!h || !offsets) return fail(SEM_EINVAL, "null argument");
    for (int q = 0; q < h->nsolve; q++) offsets[q] = h->parts[q].loc_off;
    offsets[h->nsolve] = h->n_local;
    return SEM_OK;
}

SEM_API int sem_get_geometry(const sem_handle* h, double* G, double* B, cudaStream_t s) {
    if (!h) return fail(SEM_EINVAL, "null handle");
    if (G) SEM_CUDA_TRY(cudaMemcpyAsync(G, h->G64, sizeof(double) * 6 * h->n_local, cudaMemcpyDeviceToDevice, s));
    if (B) SEM_CUDA_TRY(cudaMemcpyAsync(B, h->B64, sizeof(double) * h->n_local, cudaMemcpyDeviceToDevice, s));
    return SEM_OK;
}

SEM_API int sem_get_jacobi(const sem_handle* h, double* minv, cudaStream_t s) {
    if (!h || !minv) return fail(SEM_EINVAL, "null argument");
    SEM_CUDA_TRY(cudaMemcpyAsync(minv, h->minv64, sizeof(double) * h->n_local, cudaMemcpyDeviceToDevice, s));
    return SEM_OK;
}

}  // extern "C"
