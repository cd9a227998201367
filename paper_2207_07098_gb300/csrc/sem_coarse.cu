// The coarse-grid solve of the Schwarz preconditioner (Sec. II-B: 10 P-CG
// iterations on the coarse problem) on the ASSEMBLED coarse matrix.
//
// The coarse space is the elements' corners (N = 1).  At set-up the local
// element matrices A_e (8 x 8) are read off the coarse handle's own operator
// (eight applications to the corner unit vectors of every element at once)
// and assembled on the host into CSR over the free unique corner nodes, with
// the entries of every row summed in a fixed order.  A Jacobi-PCG iteration
// is then two launches over the free coarse nodes instead of three over the
// 8 E element-local points plus a gather-scatter:
//   spmv:    p = z + beta p_prev (on the fly for every column), q = A p, <p, q>
//   update:  x += alpha p, r -= alpha q, z = Dinv r, <r, z>
// with the CG scalars in device memory and p double-buffered (a row reads its
// neighbours' previous p).  The right-hand side is gathered from the
// element-corner restriction (the sum of every node's copies, in ascending
// local index); the last iteration writes x back to the element corners for
// the prolongation.
// Deterministic: fixed-order row sums and grid reductions.  The whole CG can
// also run as one cooperative launch with bounded grid barriers
// (coarse_cg_persist_kernel, opts.persistent in GMRES mode).
#include <algorithm>
#include <vector>

#include "sem_krylov.cuh"

namespace sem {

// scalars of the coarse CG in CoarseCsr::st
constexpr int kCsRho = 0, kCsRhoOld = 1, kCsPq = 2;

// b_i = sum of row i's element-corner copies of rc; x = 0; r = b; z = Dinv b; <r, z>
template <typename T>
__global__ void __launch_bounds__(256) coarse_gather_kernel(const T* __restrict__ rc, const int* __restrict__ gptr,
                                                            const int* __restrict__ gidx, const T* __restrict__ dinv,
                                                            int nc, T* __restrict__ x, T* __restrict__ r,
                                                            T* __restrict__ z, double* st, double* partials,
                                                            unsigned int* counter) {
    T d[1] = {(T)0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
        T b = (T)0;
        for (int q = gptr[i]; q < gptr[i + 1]; q++) b += rc[gidx[q]];
        const T zi = dinv[i] * b;
        x[i] = (T)0;
        r[i] = b;
        z[i] = zi;
        d[0] = fma(b, zi, d[0]);
    }
    gm_grid_sum<T, 1>(d, partials, counter, [&](const double* t) {
        st[kCsRho] = t[0];
        st[kCsRhoOld] = 0.0;
    });
}

// p = z + beta p_prev (beta = rho / rho_old after the first iteration),
// q = A p, <p, q>
template <typename T>
__global__ void __launch_bounds__(256) coarse_spmv_kernel(const int* __restrict__ rowptr, const int* __restrict__ col,
                                                          const T* __restrict__ val, const T* __restrict__ z,
                                                          const T* __restrict__ p_prev, T* __restrict__ p,
                                                          T* __restrict__ q, int nc, int first, double* st,
                                                          double* partials, unsigned int* counter) {
    __shared__ T beta_s;
    if (threadIdx.x == 0) {
        const double ro = st[kCsRhoOld];
        beta_s = (!first && ro > 0.0) ? (T)(st[kCsRho] / ro) : (T)0;
    }
    __syncthreads();
    const T beta = beta_s;
    T d[1] = {(T)0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
        T acc = (T)0;
        // (the first iteration does not read p_prev: it holds the last solve's p)
#pragma unroll 4
        for (int k = rowptr[i]; k < rowptr[i + 1]; k++) {
            const int j = col[k];
            acc = fma(val[k], first ? z[j] : fma(beta, p_prev[j], z[j]), acc);
        }
        const T pi = first ? z[i] : fma(beta, p_prev[i], z[i]);
        p[i] = pi;
        q[i] = acc;
        d[0] = fma(pi, acc, d[0]);
    }
    gm_grid_sum<T, 1>(d, partials, counter, [&](const double* t) { st[kCsPq] = t[0]; });
}

// alpha = rho / <p, q>; x += alpha p; r -= alpha q; z = Dinv r; rho_old = rho;
// rho = <r, z>; the last iteration also writes x to the row's element-corner
// copies in xl (xl != null; its Dirichlet corners stay zero)
template <typename T>
__global__ void __launch_bounds__(256) coarse_update_kernel(T* __restrict__ x, T* __restrict__ r, T* __restrict__ z,
                                                            const T* __restrict__ p, const T* __restrict__ q,
                                                            const T* __restrict__ dinv, int nc, T* __restrict__ xl,
                                                            const int* __restrict__ gptr,
                                                            const int* __restrict__ gidx, double* st,
                                                            double* partials, unsigned int* counter) {
    __shared__ T alpha_s;
    if (threadIdx.x == 0) {
        const double pq = st[kCsPq];
        alpha_s = pq > 0.0 ? (T)(st[kCsRho] / pq) : (T)0;  // a zero or broken direction changes nothing
    }
    __syncthreads();
    const T alpha = alpha_s;
    T d[1] = {(T)0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
        const T xi = fma(alpha, p[i], x[i]);
        x[i] = xi;
        if (xl)
            for (int c = gptr[i]; c < gptr[i + 1]; c++) xl[gidx[c]] = xi;
        const T ri = fma(-alpha, q[i], r[i]);
        const T zi = dinv[i] * ri;
        r[i] = ri;
        z[i] = zi;
        d[0] = fma(ri, zi, d[0]);
    }
    gm_grid_sum<T, 1>(d, partials, counter, [&](const double* t) {
        st[kCsRhoOld] = st[kCsRho];
        st[kCsRho] = t[0];
    });
}

// The whole coarse CG (gather and `iters` iterations) as ONE cooperative
// launch of at most one CTA per SM: the phases are separated by bounded grid
// barriers (sem_device.cuh), each reduction is a block sum into a slot per
// CTA, a barrier, and every CTA adding all slots in block order (so all CTAs
// hold the same value; consecutive reductions alternate between two slot
// arrays).  The arithmetic per row is that of the three kernels above.
template <typename T>
struct CoarseRun {
    const int* rowptr;
    const int* col;
    const T* val;
    const T* dinv;
    const int* gptr;
    const int* gidx;
    const T* rc;
    T *x, *r, *z, *p0, *p1, *q, *xl;
    int nc, iters;
    double* part;        // [2][kMaxPartials]
    unsigned int* bar;   // [0] arrivals, [1] generation
    int* err;
    long long budget;
};

template <typename T>
__device__ __forceinline__ bool coarse_allreduce(T v, double* slot, const CoarseRun<T>& a, double& out) {
    __shared__ double red[8];
    __shared__ double tot;
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid] = (double)v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < nw; w++) sum += red[w];
        slot[blockIdx.x] = sum;
        __threadfence();
    }
    if (!grid_barrier(a.bar, a.err, a.budget, &s_ok)) return false;
    if (wid == 0) {
        double acc = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) acc += __ldcg(slot + b);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) tot = acc;
    }
    __syncthreads();
    out = tot;
    __syncthreads();  // red and tot are rewritten by the next reduction
    return true;
}

template <typename T>
__global__ void __launch_bounds__(256) coarse_cg_persist_kernel(CoarseRun<T> a) {
    const int stride = gridDim.x * blockDim.x, i0 = blockIdx.x * blockDim.x + threadIdx.x;
    T d = (T)0;
    for (int i = i0; i < a.nc; i += stride) {
        T b = (T)0;
        for (int c = a.gptr[i]; c < a.gptr[i + 1]; c++) b += a.rc[a.gidx[c]];
        const T zi = a.dinv[i] * b;
        a.x[i] = (T)0;
        a.r[i] = b;
        a.z[i] = zi;
        d = fma(b, zi, d);
    }
    double rho = 0.0, rho_old = 0.0, pq = 0.0;
    int k = 0;  // reductions so far: slot array k & 1
    if (!coarse_allreduce(d, a.part + (size_t)(k++ & 1) * kMaxPartials, a, rho)) return;
    const T* pp = a.p0;
    T* pn = a.p1;
    for (int it = 0; it < a.iters; it++) {
        const bool first = it == 0;
        const T beta = (!first && rho_old > 0.0) ? (T)(rho / rho_old) : (T)0;
        d = (T)0;
        for (int i = i0; i < a.nc; i += stride) {
            T acc = (T)0;
#pragma unroll 4
            for (int kk = a.rowptr[i]; kk < a.rowptr[i + 1]; kk++) {
                const int j = a.col[kk];
                acc = fma(a.val[kk], first ? a.z[j] : fma(beta, pp[j], a.z[j]), acc);
            }
            const T pi = first ? a.z[i] : fma(beta, pp[i], a.z[i]);
            pn[i] = pi;
            a.q[i] = acc;
            d = fma(pi, acc, d);
        }
        if (!coarse_allreduce(d, a.part + (size_t)(k++ & 1) * kMaxPartials, a, pq)) return;
        const T alpha = pq > 0.0 ? (T)(rho / pq) : (T)0;
        const bool last = it == a.iters - 1;
        d = (T)0;
        for (int i = i0; i < a.nc; i += stride) {
            const T xi = fma(alpha, pn[i], a.x[i]);
            a.x[i] = xi;
            if (last)
                for (int c = a.gptr[i]; c < a.gptr[i + 1]; c++) a.xl[a.gidx[c]] = xi;
            const T ri = fma(-alpha, a.q[i], a.r[i]);
            const T zi = a.dinv[i] * ri;
            a.r[i] = ri;
            a.z[i] = zi;
            d = fma(ri, zi, d);
        }
        if (last) break;
        rho_old = rho;
        if (!coarse_allreduce(d, a.part + (size_t)(k++ & 1) * kMaxPartials, a, rho)) return;
        T* t = const_cast<T*>(pp);
        pp = pn;
        pn = t;
    }
}

template <typename T>
static T* csr_vec(const CoarseCsr& cc, int which) {  // x, r, z, p0, p1, q
    T* base = static_cast<T*>(cc.vec[std::is_same<T, float>::value ? 1 : 0]);
    return base + (size_t)which * cc.nc;
}
template <typename T>
static const T* csr_val(const CoarseCsr& cc) {
    if constexpr (std::is_same<T, float>::value)
        return cc.val32;
    else
        return cc.val64;
}
template <typename T>
static const T* csr_dinv(const CoarseCsr& cc) {
    if constexpr (std::is_same<T, float>::value)
        return cc.dinv32;
    else
        return cc.dinv64;
}

// the coarse CG as one cooperative launch (coarse_cg_persist_kernel); false
// when the device cannot launch it (the caller then takes the launch chain)
template <typename T>
static bool coarse_csr_solve_coop(sem_handle* h, const T* rc, int iters, cudaStream_t s, int* rc_out) {
    CoarseCsr& cc = h->sch.csr;
    static int per_sm = -1;
    if (per_sm < 0) {
        int coop = 0, nb = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
        if (coop) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, coarse_cg_persist_kernel<T>, 256, 0);
        per_sm = nb;
    }
    if (per_sm < 1) return false;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((cc.nc + 255) / 256, (int64_t)h->sm_count));
    CoarseRun<T> a;
    a.rowptr = cc.rowptr;
    a.col = cc.col;
    a.val = csr_val<T>(cc);
    a.dinv = csr_dinv<T>(cc);
    a.gptr = cc.gptr;
    a.gidx = cc.gidx;
    a.rc = rc;
    a.x = csr_vec<T>(cc, 0);
    a.r = csr_vec<T>(cc, 1);
    a.z = csr_vec<T>(cc, 2);
    a.p0 = csr_vec<T>(cc, 3);
    a.p1 = csr_vec<T>(cc, 4);
    a.q = csr_vec<T>(cc, 5);
    a.xl = static_cast<T*>(cc.xl[std::is_same<T, float>::value ? 1 : 0]);
    a.nc = cc.nc;
    a.iters = iters;
    a.part = cc.partials;
    a.bar = cc.bar;
    a.err = device_error_word(h->sch.coarse);
    a.budget = h->test_stall ? 100000000LL : 4000000000LL;  // ~50 ms / ~2 s at 2 GHz
    void* args[] = {&a};
    const cudaError_t e = cudaLaunchCooperativeKernel((const void*)coarse_cg_persist_kernel<T>, grid, 256, args, 0, s);
    *rc_out = e == cudaSuccess ? SEM_OK : cuda_fail(e, "cudaLaunchCooperativeKernel(coarse_cg_persist_kernel)");
    h->launches++;
    return true;
}

template <typename T>
int coarse_csr_solve(sem_handle* h, const T* rc, int iters, bool coop, cudaStream_t s) {
    CoarseCsr& cc = h->sch.csr;
    if (cc.nc == 0) return SEM_OK;
    int crc = SEM_OK;
    if (coop && coarse_csr_solve_coop<T>(h, rc, iters, s, &crc)) return crc;
    // at most one CTA per SM: the launches fit beside the local-solve kernel
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((cc.nc + 255) / 256, (int64_t)h->sm_count));
    T* x = csr_vec<T>(cc, 0);
    T* r = csr_vec<T>(cc, 1);
    T* z = csr_vec<T>(cc, 2);
    T* p[2] = {csr_vec<T>(cc, 3), csr_vec<T>(cc, 4)};
    T* q = csr_vec<T>(cc, 5);
    const T* dinv = csr_dinv<T>(cc);
    T* xl = static_cast<T*>(cc.xl[std::is_same<T, float>::value ? 1 : 0]);
    coarse_gather_kernel<T><<<grid, 256, 0, s>>>(rc, cc.gptr, cc.gidx, dinv, cc.nc, x, r, z, cc.st, cc.partials,
                                                 cc.counter);
    SEM_LAUNCH_CHECK("coarse_gather_kernel");
    h->launches++;
    for (int it = 0; it < iters; it++) {
        T* pn = p[(it + 1) & 1];
        coarse_spmv_kernel<T><<<grid, 256, 0, s>>>(cc.rowptr, cc.col, csr_val<T>(cc), z, p[it & 1], pn, q, cc.nc,
                                                   it == 0 ? 1 : 0, cc.st, cc.partials, cc.counter);
        SEM_LAUNCH_CHECK("coarse_spmv_kernel");
        coarse_update_kernel<T><<<grid, 256, 0, s>>>(x, r, z, pn, q, dinv, cc.nc, it == iters - 1 ? xl : nullptr,
                                                     cc.gptr, cc.gidx, cc.st, cc.partials, cc.counter);
        SEM_LAUNCH_CHECK("coarse_update_kernel");
        h->launches += 2;
    }
    return SEM_OK;
}
template int coarse_csr_solve<double>(sem_handle*, const double*, int, bool, cudaStream_t);
template int coarse_csr_solve<float>(sem_handle*, const float*, int, bool, cudaStream_t);

template <typename T>
const T* coarse_csr_x(const sem_handle* h) {  // element-corner values [E][8]
    return static_cast<const T*>(h->sch.csr.xl[std::is_same<T, float>::value ? 1 : 0]);
}
template const double* coarse_csr_x<double>(const sem_handle*);
template const float* coarse_csr_x<float>(const sem_handle*);

void free_coarse_csr(CoarseCsr& cc) {
    cudaFree(cc.rowptr);
    cudaFree(cc.col);
    cudaFree(cc.val64);
    cudaFree(cc.val32);
    cudaFree(cc.dinv64);
    cudaFree(cc.dinv32);
    cudaFree(cc.gptr);
    cudaFree(cc.gidx);
    cudaFree(cc.vec[0]);
    cudaFree(cc.vec[1]);
    cudaFree(cc.xl[0]);
    cudaFree(cc.xl[1]);
    cudaFree(cc.st);
    cudaFree(cc.partials);
    cudaFree(cc.counter);
    cudaFree(cc.bar);
    cc = CoarseCsr{};
}

template <typename T>
static int upload(sem_handle* h, T** d, const std::vector<T>& v) {
    int rc = dalloc(h, d, std::max<size_t>(v.size(), 1));
    if (rc) return rc;
    if (!v.empty()) SEM_CUDA_TRY(cudaMemcpy(*d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return SEM_OK;
}

// Assemble the coarse CSR of handle h from its coarse handle (lx = 2, one
// element per fine element; cgid / cmask: the corners' global ids and
// Dirichlet mask, element-major [E][8]).
int build_coarse_csr(sem_handle* h, const int64_t* cgid, const uint8_t* cmask) {
    sem_handle* hc = h->sch.coarse;
    CoarseCsr& cc = h->sch.csr;
    const int64_t E = hc->parts[0].E, nl = E * 8;
    // element matrices: column c of every A_e = A_L applied to corner c's unit vector
    std::vector<double> Ae((size_t)nl * 8), e_c((size_t)nl), w_c((size_t)nl);
    double *du = nullptr, *dw = nullptr;
    if (cudaMalloc(&du, sizeof(double) * nl) != cudaSuccess || cudaMalloc(&dw, sizeof(double) * nl) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(du);
        return fail(SEM_ENOMEM, "cudaMalloc for the coarse element matrices failed");
    }
    int rc = SEM_OK;
    for (int c = 0; c < 8 && !rc; c++) {
        for (int64_t L = 0; L < nl; L++) e_c[(size_t)L] = (L % 8) == c ? 1.0 : 0.0;
        if (cudaMemcpy(du, e_c.data(), sizeof(double) * nl, cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = fail(SEM_ECUDA, "cudaMemcpy of a coarse unit vector");
            break;
        }
        if ((rc = launch_ax_local(hc, du, dw, SEM_FP64, 0))) break;
        if (cudaMemcpy(w_c.data(), dw, sizeof(double) * nl, cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = fail(SEM_ECUDA, "cudaMemcpy of a coarse operator column");
            break;
        }
        for (int64_t e = 0; e < E; e++)
            for (int a = 0; a < 8; a++) Ae[(size_t)(e * 8 + a) * 8 + c] = w_c[(size_t)(e * 8 + a)];
    }
    cudaFree(du);
    cudaFree(dw);
    if (rc) return rc;
    // rows: the free unique corner nodes in ascending global id
    std::vector<int64_t> ids;
    ids.reserve((size_t)nl);
    for (int64_t L = 0; L < nl; L++)
        if (cmask[L]) ids.push_back(cgid[L]);
    std::sort(ids.begin(), ids.end());
    ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
    const int nc = (int)ids.size();
    std::vector<int> cmap((size_t)nl, -1);
    for (int64_t L = 0; L < nl; L++)
        if (cmask[L]) cmap[(size_t)L] = (int)(std::lower_bound(ids.begin(), ids.end(), cgid[L]) - ids.begin());
    // entries summed in (row, column, element, corner pair) order
    struct Ent {
        int64_t key;  // row << 32 | column
        int64_t ord;  // e * 64 + a * 8 + b
        double v;
    };
    std::vector<Ent> ent;
    ent.reserve((size_t)E * 64);
    for (int64_t e = 0; e < E; e++)
        for (int a = 0; a < 8; a++) {
            const int ra = cmap[(size_t)(e * 8 + a)];
            if (ra < 0) continue;
            for (int b = 0; b < 8; b++) {
                const int cb = cmap[(size_t)(e * 8 + b)];
                if (cb < 0) continue;
                ent.push_back({((int64_t)ra << 32) | (int64_t)cb, e * 64 + a * 8 + b, Ae[(size_t)(e * 8 + a) * 8 + b]});
            }
        }
    std::sort(ent.begin(), ent.end(),
              [](const Ent& x, const Ent& y) { return x.key != y.key ? x.key < y.key : x.ord < y.ord; });
    std::vector<int> rowptr((size_t)nc + 1, 0), col;
    std::vector<double> val, dinv((size_t)nc, 0.0);
    for (size_t q = 0; q < ent.size();) {
        size_t q2 = q;
        double sum = 0.0;
        while (q2 < ent.size() && ent[q2].key == ent[q].key) sum += ent[q2++].v;
        const int row = (int)(ent[q].key >> 32), cl = (int)(ent[q].key & 0xffffffff);
        col.push_back(cl);
        val.push_back(sum);
        rowptr[(size_t)row + 1]++;
        if (row == cl) dinv[(size_t)row] = sum;
        q = q2;
    }
    for (int i = 0; i < nc; i++) {
        rowptr[(size_t)i + 1] += rowptr[(size_t)i];
        if (!(dinv[(size_t)i] > 0.0)) return fail(SEM_EINVAL, "coarse matrix with a non-positive diagonal entry");
        dinv[(size_t)i] = 1.0 / dinv[(size_t)i];
    }
    // each row's element-corner copies, in ascending local index
    std::vector<int> gptr((size_t)nc + 1, 0), gidx;
    for (int64_t L = 0; L < nl; L++)
        if (cmap[(size_t)L] >= 0) gptr[(size_t)cmap[(size_t)L] + 1]++;
    for (int i = 0; i < nc; i++) gptr[(size_t)i + 1] += gptr[(size_t)i];
    gidx.resize((size_t)gptr[(size_t)nc]);
    std::vector<int> fill(gptr.begin(), gptr.end() - 1);
    for (int64_t L = 0; L < nl; L++)
        if (cmap[(size_t)L] >= 0) gidx[(size_t)fill[(size_t)cmap[(size_t)L]]++] = (int)L;
    std::vector<float> val32(val.begin(), val.end()), dinv32(dinv.begin(), dinv.end());
    cc.nc = nc;
    if ((rc = upload(h, &cc.rowptr, rowptr)) || (rc = upload(h, &cc.col, col)) || (rc = upload(h, &cc.val64, val)) ||
        (rc = upload(h, &cc.val32, val32)) || (rc = upload(h, &cc.dinv64, dinv)) ||
        (rc = upload(h, &cc.dinv32, dinv32)) || (rc = upload(h, &cc.gptr, gptr)) ||
        (rc = upload(h, &cc.gidx, gidx)))
        return rc;
    const size_t nv = (size_t)6 * (size_t)std::max(nc, 1);
    double* v64 = nullptr;
    float* v32 = nullptr;
    if ((rc = dalloc(h, &v64, nv)) || (rc = dalloc(h, &v32, nv)) || (rc = dalloc(h, &cc.st, 4)) ||
        (rc = dalloc(h, &cc.partials, (size_t)2 * kMaxPartials)))
        return rc;
    cc.vec[0] = v64;
    cc.vec[1] = v32;
    SEM_CUDA_TRY(cudaMemset(v64, 0, sizeof(double) * nv));
    SEM_CUDA_TRY(cudaMemset(v32, 0, sizeof(float) * nv));
    double* xl64 = nullptr;
    float* xl32 = nullptr;
    if ((rc = dalloc(h, &xl64, (size_t)nl)) || (rc = dalloc(h, &xl32, (size_t)nl))) return rc;
    cc.xl[0] = xl64;
    cc.xl[1] = xl32;
    SEM_CUDA_TRY(cudaMemset(xl64, 0, sizeof(double) * nl));  // Dirichlet corners stay zero
    SEM_CUDA_TRY(cudaMemset(xl32, 0, sizeof(float) * nl));
    SEM_CUDA_TRY(cudaMalloc(&cc.counter, sizeof(unsigned int)));
    SEM_CUDA_TRY(cudaMemset(cc.counter, 0, sizeof(unsigned int)));
    SEM_CUDA_TRY(cudaMalloc(&cc.bar, 2 * sizeof(unsigned int)));
    SEM_CUDA_TRY(cudaMemset(cc.bar, 0, 2 * sizeof(unsigned int)));
    return SEM_OK;
}

}  // namespace sem
