// Jacobi-PCG of Sec. II-B (Karp et al.) as ONE persistent launch for meshes
// small enough to stay in L2, where the three launches of a CG iteration cost
// more than their work (a 32 K-point mesh: ~9 us of launch latency each).
//
// The CTAs of a cooperative launch (all resident at once) run every iteration
// of the solve, with a grid barrier between the phases that read what other
// CTAs wrote:
//   K-A  p = z + beta p;  w = A_L p;  partial <p, w>            | barrier
//        alpha = rho / <p, w> (every CTA sums the partials in CTA order);
//   K-B  w = mask QQ^T w (segments split over the grid)          | barrier
//   K-C  x += alpha p; r -= alpha w; z = Minv r; partials       | barrier
//        rho = <r, z>, rr = <r, r>: convergence and beta, in every CTA.
// Every CTA computes the scalars from the same partials in the same order, so
// all take the same decisions without another exchange, and a solve is
// bit-reproducible.  The operator is the shared-slab kernel's ax_group and
// the gather-scatter the same segment sums as the QQ^T launch.
//
// The grid barrier is bounded: a CTA that waits longer than its budget sets
// the device error word and returns, so a barrier that can never complete
// ends in SEM_ETIMEOUT instead of a hang.
#include <algorithm>

#include "sem_ax.cuh"
#include "sem_gs.cuh"

namespace sem {

template <typename T>
struct PersistParams {
    T* x;
    T* p;
    T* r;
    T* w;
    T* z;
    const T* minv;
    const uint8_t* mult;
    const T* G;
    const T* D;
    int64_t E;
    int64_t n;
    GSLists g;
    CGState* st;
    double* part;        // [3][kMaxPartials] per-CTA partial sums
    unsigned int* bar;   // [0] arrivals, [1] generation
    int* err;
    long long budget;    // clock cycles a CTA waits at one barrier
    int stall;           // test of the bounded barrier: CTA 0 never arrives at the first one
    const T* mass;       // [n] Helmholtz term h2 B, null for Poisson
};


// Sum over the CTAs of partial q (CTA order, fixed tree): valid in thread 0.
template <int NV>
__device__ __forceinline__ void sum_partials(const double* part, const int (&q)[NV], double (&acc)[NV],
                                             double* red) {
#pragma unroll
    for (int k = 0; k < NV; k++) acc[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; k++) acc[k] += __ldcg(&part[q[k] * kMaxPartials + b]);
    block_sum<NV>(acc, red);
}

template <typename T, int LX>
__global__ void __launch_bounds__(AxCfg<LX>::THREADS) cg_persist_kernel(PersistParams<T> a) {
    using C = AxCfg<LX>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const AxSmem<T, LX> sm(smem_raw);
    __shared__ double red[3 * 32];
    __shared__ float redf[2 * 3 * 32];
    __shared__ T s_inv[256];
    __shared__ T s_tbeta, s_ta;
    __shared__ int s_done, s_first, s_ok;
    // scalars of the solve, in shared memory (only thread 0 of each CTA touches
    // them; identical in all CTAs), so they hold no registers in the loop
    __shared__ double rho, rho_old, rr, pap, alpha, tol2;
    __shared__ int iter, max_iter, status;
    for (int m = threadIdx.x; m < 256; m += blockDim.x)
        s_inv[m] = m ? (sizeof(T) == 4 ? (T)(1.0f / (float)m) : (T)(1.0 / m)) : T(0);
    ax_load_d<T, LX>(sm.sD, a.D);
    if (threadIdx.x == 0) {  // the state the CG start left
        const CGState* st = a.st;
        rho = st->rho;
        rho_old = st->rho_old;
        rr = st->rr;
        tol2 = st->tol2;
        iter = st->iter;
        max_iter = st->max_iter;
        status = st->status;
        s_done = st->done;
        s_first = cg_first(st) ? 1 : 0;
    }
    __syncthreads();
    const AxThread<LX> th;
    const int64_t ngroups = (a.E + C::EPC - 1) / C::EPC;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    bool failed = false;
    while (!s_done) {
        if (threadIdx.x == 0) s_tbeta = s_first ? T(0) : (T)(rho / rho_old);
        __syncthreads();
        const T tbeta = s_tbeta;
        const bool first = s_first != 0;
        // K-A over this CTA's element groups
        float ph = 0.f, pl = 0.f;
        double pd = 0.0;
        for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
            const int64_t e = g * C::EPC + th.el;
            const bool valid = th.active && e < a.E;
            const T pw = ax_group<T, LX, true>(sm, th, e, valid, nullptr, a.z, a.p, a.w, a.G, tbeta, first, a.mass);
            if constexpr (sizeof(T) == 4)
                fpair_add(ph, pl, pw);
            else
                pd += (double)pw;
            __syncthreads();
        }
        {
            double v[1];
            if constexpr (sizeof(T) == 4) {
                float hh[1] = {ph}, ll[1] = {pl};
                block_sum_pair<1>(hh, ll, redf);
                v[0] = threadIdx.x == 0 ? (double)hh[0] + (double)ll[0] : 0.0;
            } else {
                v[0] = pd;
                block_sum<1>(v, red);
            }
            if (threadIdx.x == 0) a.part[0 * kMaxPartials + blockIdx.x] = v[0];
        }
        if (a.stall && blockIdx.x == 0) return;  // the other CTAs' first barrier expires
        if (!grid_barrier(a.bar, a.err, a.budget, &s_ok)) {
            failed = true;
            break;
        }
        {
            const int q[1] = {0};
            double acc[1];
            sum_partials<1>(a.part, q, acc, red);
            if (threadIdx.x == 0) {
                pap = acc[0];
                if (!(pap > 0.0) || !isfinite(pap)) {
                    alpha = 0.0;
                    status = SEM_EBREAKDOWN;
                    s_done = 1;
                } else {
                    alpha = rho / pap;
                }
                s_ta = (T)alpha;
            }
            __syncthreads();
        }
        if (s_done) break;
        // K-B: w = mask QQ^T w, the segments split over the whole grid
        gs_pairs<T, 1>(a.w, a.g.pairs, a.g.npair, t0, nthr);
        gs_quads<T, 1>(a.w, a.g.quads, a.g.nquad, t0, nthr);
        gs_rest<T>(a.w, a.g, t0, nthr);
        if (!grid_barrier(a.bar, a.err, a.budget, &s_ok)) {
            failed = true;
            break;
        }
        // K-C over this thread's points
        {
            const T ta = s_ta;
            float h2[2] = {0.f, 0.f}, l2[2] = {0.f, 0.f};
            double d2[2] = {0.0, 0.0};
            for (int64_t L = t0; L < a.n; L += nthr) {
                const T xv = fma(ta, a.p[L], a.x[L]);
                const T rv = fma(-ta, a.w[L], a.r[L]);
                const T zv = a.minv[L] * rv;
                a.x[L] = xv;
                a.r[L] = rv;
                a.z[L] = zv;
                const T iv = s_inv[a.mult[L]];
                if constexpr (sizeof(T) == 4) {
                    fpair_add(h2[0], l2[0], rv * zv * iv);
                    fpair_add(h2[1], l2[1], rv * rv * iv);
                } else {
                    d2[0] = fma(rv * zv, iv, d2[0]);
                    d2[1] = fma(rv * rv, iv, d2[1]);
                }
            }
            double v[2];
            if constexpr (sizeof(T) == 4) {
                block_sum_pair<2>(h2, l2, redf);
                v[0] = threadIdx.x == 0 ? (double)h2[0] + (double)l2[0] : 0.0;
                v[1] = threadIdx.x == 0 ? (double)h2[1] + (double)l2[1] : 0.0;
            } else {
                v[0] = d2[0];
                v[1] = d2[1];
                block_sum<2>(v, red);
            }
            if (threadIdx.x == 0) {
                a.part[1 * kMaxPartials + blockIdx.x] = v[0];
                a.part[2 * kMaxPartials + blockIdx.x] = v[1];
            }
        }
        if (!grid_barrier(a.bar, a.err, a.budget, &s_ok)) {
            failed = true;
            break;
        }
        {
            const int q[2] = {1, 2};
            double acc[2];
            sum_partials<2>(a.part, q, acc, red);
            if (threadIdx.x == 0) {  // the scalar step of cg_set_rho
                rho_old = rho;
                rho = acc[0];
                rr = acc[1];
                iter++;
                if (!isfinite(rr) || !isfinite(rho)) {
                    status = SEM_EBREAKDOWN;
                    s_done = 1;
                } else if (rr <= tol2) {
                    status = SEM_OK;
                    s_done = 1;
                } else if (iter >= max_iter) {
                    status = SEM_ENOTCONV;
                    s_done = 1;
                }
                s_first = 0;
            }
            // the next loop test reads s_done; the K-A of the next iteration
            // starts after the __syncthreads() that publishes s_tbeta
            __syncthreads();
        }
    }
    if (!failed && blockIdx.x == 0 && threadIdx.x == 0) {
        CGState* st = a.st;
        st->rho = rho;
        st->rho_old = rho_old;
        st->rr = rr;
        st->pap = pap;
        st->alpha = alpha;
        st->iter = iter;
        st->status = status;
        st->done = 1;
    }
}

template <typename T, int LX>
static int launch_persist_t(sem_handle* h, PersistParams<T> a, cudaStream_t s) {
    using C = AxCfg<LX>;
    constexpr size_t smem = ax_smem_bytes<T, LX>();
    static int per_sm = -1;
    if (per_sm < 0) {
        cudaError_t e = cudaFuncSetAttribute(cg_persist_kernel<T, LX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(cg_persist_kernel)");
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cg_persist_kernel<T, LX>, C::THREADS, smem);
        per_sm = nb;
    }
    if (per_sm < 1) return fail(SEM_EINVAL, "persistent CG kernel cannot be resident");
    const int64_t ngroups = (a.E + C::EPC - 1) / C::EPC;
    // at least one CTA per element group, more (up to the resident capacity)
    // to spread the gather-scatter and the vector update
    const int64_t want = std::max<int64_t>(ngroups, (a.n + 4 * C::THREADS - 1) / (4 * C::THREADS));
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>({want, (int64_t)h->sm_count * per_sm, (int64_t)kMaxPartials}));
    SEM_CUDA_TRY(cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned int), s));
    void* args[] = {&a};
    SEM_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)cg_persist_kernel<T, LX>, dim3(grid), dim3(C::THREADS),
                                             args, smem, s));
    h->launches++;
    return SEM_OK;
}

template <typename T>
static int dispatch_persist(sem_handle* h, int lx, const PersistParams<T>& a, cudaStream_t s) {
    switch (lx) {
        case 2: return launch_persist_t<T, 2>(h, a, s);
        case 3: return launch_persist_t<T, 3>(h, a, s);
        case 4: return launch_persist_t<T, 4>(h, a, s);
        case 5: return launch_persist_t<T, 5>(h, a, s);
        case 6: return launch_persist_t<T, 6>(h, a, s);
        case 7: return launch_persist_t<T, 7>(h, a, s);
        case 8: return launch_persist_t<T, 8>(h, a, s);
        case 9: return launch_persist_t<T, 9>(h, a, s);
        case 10: return launch_persist_t<T, 10>(h, a, s);
        default: return fail(SEM_EINVAL, "persistent CG covers lx <= 10");
    }
}

bool persist_available(const sem_handle* h) {
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
    return coop && h->nsolve == 1 && h->parts[0].lx <= kPersistMaxLx;
}

// The whole CG of state slot `slot` (started by cg_init_kernel) in one
// cooperative launch: precision SEM_FP32 (inner vectors) or the native FP64
// class (FP64 vectors).
int launch_cg_persist(sem_handle* h, int precision, int slot, cudaStream_t s) {
    const MeshPart& pt = h->parts[0];
    const GSLists& g = h->gs;
    const long long budget = h->test_stall ? 100000000LL : 4000000000LL;  // ~50 ms / ~2 s at 2 GHz
    if (is_f32(precision)) {
        PersistParams<float> a = {h->ws.d32, h->ws.p32, h->ws.r32, h->ws.w32, h->ws.z32, h->minv32, h->mult,
                                  h->G32, h->D32[pt.lx], pt.E, h->n_local, g, h->state + slot, h->partials,
                                  h->counters + 10, device_error_word(h), budget, h->test_stall, h->hmass32};
        return dispatch_persist<float>(h, pt.lx, a, s);
    }
    PersistParams<double> a = {h->ws.x, h->ws.p, h->ws.r, h->ws.w, h->ws.z, h->minv64, h->mult,
                               h->G64, h->D64[pt.lx], pt.E, h->n_local, g, h->state + slot, h->partials,
                               h->counters + 10, device_error_word(h), budget, h->test_stall, h->hmass64};
    return dispatch_persist<double>(h, pt.lx, a, s);
}

}  // namespace sem
