// Template of the matrix-free local operator kernels (see sem_ax.cu for the
// description); instantiated per precision in sem_ax_f64.cu and sem_ax_f32.cu.
#pragma once

#include <algorithm>
#include <type_traits>

#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

template <int LX>
struct AxCfg {
    static constexpr int N2 = LX * LX;
    static constexpr int N3 = LX * LX * LX;
    static constexpr int EPC = (256 / N2) > 0 ? (256 / N2) : 1;
    static constexpr int USED = EPC * N2;
    static constexpr int THREADS = ((USED + 31) / 32) * 32;
    static constexpr int DP = LX + 1;  // padded row of D in shared memory
};

template <typename T>
struct AxParams {
    const T* u;   // input (plain variant)
    T* w;         // output
    const T* G;   // [E][6][lx^3], h1 folded in
    const T* D;   // [lx][lx]
    int64_t E;
    const T* mass;  // [n] Helmholtz term h2 B (w += mass u), null for Poisson
    const CGState* skip_st;  // plain kernels: return at once when skip_st->done (null: never)
    // fused CG variant: u = z + beta p, p <- u, partial <p, w>
    const T* z;
    T* p;
    CGState* st;
    double* partials;
    unsigned int* counter;
    int* err;     // set to 1 when a bounded wait of a staged kernel expires
    int dry;      // 1: only prepare the kernel (attributes, occupancy); no launch
    int variant;  // 0: shared-slab kernel; 1..kBulkVariants: bulk-staged (EPC, stages)
    long long wait_budget;  // clock cycles a staged kernel waits for a stage
    unsigned tx_extra;      // bytes announced beyond the copies (test of the bounded wait)
    // batched form (bulk kernel): element-group list of one order, per-solve
    // CG states (st is the base) and partials
    const int64_t* loc;
    const int* cnt;
    const int* solve;
    int64_t ngroups;
    int64_t goff;
    const int* sgfirst;
    const int* sgcount;
    double* gpart;
    unsigned int* scount;
};

template <typename T, int LX>
constexpr size_t ax_smem_bytes() {
    return sizeof(T) * ((size_t)LX * AxCfg<LX>::DP + 3 * (size_t)AxCfg<LX>::EPC * AxCfg<LX>::N3);
}

// Shared-memory carve-up of one CTA: D (padded rows), then EPC element slots
// of u, wr and ws.
template <typename T, int LX>
struct AxSmem {
    T* sD;
    T* su;
    T* sr;
    T* ss;
    __device__ __forceinline__ explicit AxSmem(unsigned char* raw) {
        using C = AxCfg<LX>;
        sD = reinterpret_cast<T*>(raw);
        su = sD + LX * C::DP;
        sr = su + C::EPC * C::N3;
        ss = sr + C::EPC * C::N3;
    }
    // D (padded rows) at d, the EPC element slots of u, wr, ws from `slots` on
    __device__ __forceinline__ AxSmem(T* d, T* slots) {
        using C = AxCfg<LX>;
        sD = d;
        su = slots;
        sr = su + C::EPC * C::N3;
        ss = sr + C::EPC * C::N3;
    }
};

// Thread coordinates inside a CTA: element slot `el`, column (i, j).
template <int LX>
struct AxThread {
    int el, ij, i, j, so;
    bool active;
    __device__ __forceinline__ AxThread() {
        using C = AxCfg<LX>;
        el = threadIdx.x / C::N2;
        ij = threadIdx.x - el * C::N2;
        i = ij % LX;
        j = ij / LX;
        active = el < C::EPC;
        so = (active ? el : 0) * C::N3;
    }
};

template <typename T, int LX>
__device__ __forceinline__ void ax_load_d(T* sD, const T* D) {
    constexpr int DP = AxCfg<LX>::DP;
    for (int t = threadIdx.x; t < LX * LX; t += blockDim.x) sD[(t / LX) * DP + (t % LX)] = D[t];
}

// One group of up to EPC elements.  Element `e` of this thread (relative to
// the pointers) is processed when `valid`.  Plain: w = A_L u.  FUSED:
// u = z + beta p (p <- u; old p ignored on the first iteration), w = A_L u,
// and the thread's partial sum of u.w is returned.  mass (may be null): the
// Helmholtz term h2 B per point, added as w += mass u.  Contains two
// __syncthreads(); every thread of the CTA must call it.
template <typename T, int LX, bool FUSED>
__device__ __forceinline__ T ax_group(const AxSmem<T, LX>& sm, const AxThread<LX>& th, int64_t e, bool valid,
                                      const T* __restrict__ u, const T* __restrict__ z, T* __restrict__ p,
                                      T* __restrict__ w, const T* __restrict__ G, T tbeta, bool first,
                                      const T* __restrict__ mass = nullptr) {
    using C = AxCfg<LX>;
    constexpr int N2 = C::N2, N3 = C::N3, DP = C::DP;
    const T* sD = sm.sD;
    T* su = sm.su;
    T* sr = sm.sr;
    T* ss = sm.ss;
    const int so = th.so, ij = th.ij, i = th.i, j = th.j;
    const int64_t base = e * N3 + ij;
    T ucol[LX];
    // all loads of the column first, then the p stores: no load waits on a store
#pragma unroll
    for (int k = 0; k < LX; k++) {
        if (FUSED) {
            ucol[k] = valid ? ld_stream(z + base + k * N2) : T(0);
        } else {
            ucol[k] = valid ? ld_stream(u + base + k * N2) : T(0);
        }
    }
    if (FUSED) {
        T pold[LX];
#pragma unroll
        for (int k = 0; k < LX; k++) pold[k] = (valid && !first) ? p[base + k * N2] : T(0);
#pragma unroll
        for (int k = 0; k < LX; k++) {
            ucol[k] = fma(tbeta, pold[k], ucol[k]);
            if (valid) p[base + k * N2] = ucol[k];
        }
    }
#pragma unroll
    for (int k = 0; k < LX; k++)
        if (th.active) su[so + k * N2 + ij] = ucol[k];
    __syncthreads();
    T wt[LX];
    const T* Ge = G + e * 6 * N3 + ij;
#pragma unroll
    for (int k = 0; k < LX; k++) {
        T ur = T(0), us = T(0), ut = T(0);
#pragma unroll
        for (int l = 0; l < LX; l++) {
            ur = fma(sD[i * DP + l], su[so + k * N2 + j * LX + l], ur);
            us = fma(sD[j * DP + l], su[so + k * N2 + l * LX + i], us);
            ut = fma(sD[k * DP + l], ucol[l], ut);
        }
        T g11 = T(0), g12 = T(0), g13 = T(0), g22 = T(0), g23 = T(0), g33 = T(0);
        if (valid) {
            g11 = ld_stream(Ge + 0 * N3 + k * N2);
            g12 = ld_stream(Ge + 1 * N3 + k * N2);
            g13 = ld_stream(Ge + 2 * N3 + k * N2);
            g22 = ld_stream(Ge + 3 * N3 + k * N2);
            g23 = ld_stream(Ge + 4 * N3 + k * N2);
            g33 = ld_stream(Ge + 5 * N3 + k * N2);
        }
        const T wr = fma(g11, ur, fma(g12, us, g13 * ut));
        const T ws = fma(g12, ur, fma(g22, us, g23 * ut));
        wt[k] = fma(g13, ur, fma(g23, us, g33 * ut));
        if (th.active) {
            sr[so + k * N2 + ij] = wr;
            ss[so + k * N2 + ij] = ws;
        }
    }
    __syncthreads();
    T pw = T(0);
#pragma unroll
    for (int k = 0; k < LX; k++) {
        T acc = T(0);
        if constexpr (sizeof(T) == 4 && FUSED) {
            // FP32 CG kernel: three independent chains (r, s, t), summed at the
            // end, a third of the dependent-FMA latency per point (measured
            // 1.6% faster; the plain operator keeps one chain, which measured
            // no slower)
            T ar = T(0), as = T(0), at = T(0);
#pragma unroll
            for (int l = 0; l < LX; l++) {
                ar = fma(sD[l * DP + i], sr[so + k * N2 + j * LX + l], ar);
                as = fma(sD[l * DP + j], ss[so + k * N2 + l * LX + i], as);
                at = fma(sD[l * DP + k], wt[l], at);
            }
            acc = (ar + as) + at;
        } else {
            // one chain (FP64: the FP64 pipe's throughput, not latency, bounds it)
#pragma unroll
            for (int l = 0; l < LX; l++) {
                acc = fma(sD[l * DP + i], sr[so + k * N2 + j * LX + l], acc);
                acc = fma(sD[l * DP + j], ss[so + k * N2 + l * LX + i], acc);
                acc = fma(sD[l * DP + k], wt[l], acc);
            }
        }
        if (valid) {
            // Helmholtz mass term: u is read back from its shared slot, so the
            // column need not stay in registers through this loop
            if (mass) acc = fma(ld_stream(mass + base + k * N2), su[so + k * N2 + ij], acc);
            st_keep<FUSED>(w + base + k * N2, acc);
            if (FUSED) pw = fma(ucol[k], acc, pw);
        }
    }
    return pw;
}

template <typename T, int LX, bool FUSED>
__global__ void __launch_bounds__(AxCfg<LX>::THREADS) ax_kernel(AxParams<T> a) {
    using C = AxCfg<LX>;
    constexpr int EPC = C::EPC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const AxSmem<T, LX> sm(smem_raw);
    bool first = false;
    __shared__ T s_tbeta;  // beta, divided and converted once by thread 0 (GB300's FP64 pipe is slow)
    if (FUSED) {
        if (a.st->done) return;  // uniform over the grid
        if (threadIdx.x == 0) s_tbeta = (T)cg_beta(a.st);
        first = cg_first(a.st);
    } else if (a.skip_st && a.skip_st->done) {
        return;  // uniform over the grid
    }
    ax_load_d<T, LX>(sm.sD, a.D);
    const AxThread<LX> th;
    const int64_t ngroups = (a.E + EPC - 1) / EPC;
    double pap = 0.0;
    float paph = 0.f, papl = 0.f;  // FP32 kernels: <p, A p> as a float pair (no FP64 per group)
    __syncthreads();
    const T tbeta = FUSED ? s_tbeta : T(0);
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const int64_t e = g * EPC + th.el;
        const bool valid = th.active && e < a.E;
        const T pw = ax_group<T, LX, FUSED>(sm, th, e, valid, a.u, a.z, a.p, a.w, a.G, tbeta, first, a.mass);
        if (FUSED) {
            if constexpr (sizeof(T) == 4)
                fpair_add(paph, papl, pw);
            else
                pap += (double)pw;
        }
        __syncthreads();
    }
    if (FUSED) {
        CGState* st = a.st;
        if constexpr (sizeof(T) == 4) {
            float h[1] = {paph}, l[1] = {papl};
            grid_sum_finalize_pair<1>(h, l, a.partials, a.counter,
                                      [&](double (&acc)[1]) { cg_set_alpha(st, acc[0]); });
        } else {
            double v[1] = {pap};
            grid_sum_finalize<1>(v, a.partials, a.counter, [&](double (&acc)[1]) { cg_set_alpha(st, acc[0]); });
        }
    }
}

template <typename T, int LX, bool FUSED>
inline int launch_ax_t(sem_handle* h, const AxParams<T>& a, cudaStream_t s) {
    using C = AxCfg<LX>;
    constexpr size_t smem = ax_smem_bytes<T, LX>();
    static int per_sm = -1;  // occupancy of this instantiation (same device for the process)
    if (per_sm < 0) {
        cudaFuncSetAttribute(ax_kernel<T, LX, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ax_kernel<T, LX, FUSED>, C::THREADS, smem);
        per_sm = nb > 0 ? nb : 1;
    }
    if (a.dry) return SEM_OK;
    const int64_t ngroups = (a.E + C::EPC - 1) / C::EPC;
    int64_t grid = std::min<int64_t>(ngroups, (int64_t)h->sm_count * per_sm);
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, kMaxPartials));
    ax_kernel<T, LX, FUSED><<<(int)grid, C::THREADS, smem, s>>>(a);
    SEM_LAUNCH_CHECK("ax_kernel");
    h->launches++;
    return SEM_OK;
}

template <typename T, bool FUSED>
inline int dispatch_ax(sem_handle* h, int lx, const AxParams<T>& a, cudaStream_t s) {
    switch (lx) {
        case 2: return launch_ax_t<T, 2, FUSED>(h, a, s);
        case 3: return launch_ax_t<T, 3, FUSED>(h, a, s);
        case 4: return launch_ax_t<T, 4, FUSED>(h, a, s);
        case 5: return launch_ax_t<T, 5, FUSED>(h, a, s);
        case 6: return launch_ax_t<T, 6, FUSED>(h, a, s);
        case 7: return launch_ax_t<T, 7, FUSED>(h, a, s);
        case 8: return launch_ax_t<T, 8, FUSED>(h, a, s);
        case 9: return launch_ax_t<T, 9, FUSED>(h, a, s);
        case 10: return launch_ax_t<T, 10, FUSED>(h, a, s);
        case 11: return launch_ax_t<T, 11, FUSED>(h, a, s);
        case 12: return launch_ax_t<T, 12, FUSED>(h, a, s);
        case 13: return launch_ax_t<T, 13, FUSED>(h, a, s);
        case 14: return launch_ax_t<T, 14, FUSED>(h, a, s);
        case 15: return launch_ax_t<T, 15, FUSED>(h, a, s);
        case 16: return launch_ax_t<T, 16, FUSED>(h, a, s);
        default: return fail(SEM_EINVAL, "lx out of range");
    }
}


// Bulk-staged variants (sem_ax_bulk.cuh): variant v = 1..kBulkVariants uses
// (elements per CTA, stages) = kBulkCfg[v - 1]; only even lx in {4,6,8,10,12}.
constexpr int kBulkVariants = kBulkVariantsMax;
constexpr int kBulkCfg[kBulkVariants][2] = {{1, 3}, {2, 2}, {2, 3}, {4, 2}};
int dispatch_ax_bulk_f64(sem_handle* h, int lx, const AxParams<double>& a, bool fused, cudaStream_t s);
int bulk_set_d_f64(const double* D, int lx);
int bulk_set_d_f32(const float* D, int lx);
// fills the constant-bank line-transform tables of order lx (sem_ax_df.cu)
int dfl_set_coef(const float* cf, int lx);
int dispatch_ax_bulk_batch_f32(sem_handle* h, int lx, const AxParams<float>& a, bool fused, cudaStream_t s);
int dispatch_ax_bulk_f32(sem_handle* h, int lx, const AxParams<float>& a, bool fused, cudaStream_t s);
inline bool bulk_supported(int lx) { return lx == 4 || lx == 6 || lx == 8 || lx == 10 || lx == 12; }
// Shared memory of the fused (larger) bulk kernel of variant v fits in a CTA.
inline bool bulk_fits(int lx, int v, bool fp32) {
    if (v < 1 || v > kBulkVariants || !bulk_supported(lx)) return false;
    const size_t epc = kBulkCfg[v - 1][0], nst = kBulkCfg[v - 1][1];
    const size_t n3 = (size_t)lx * lx * lx, el = fp32 ? 4 : 8;
    const size_t bytes = el * ((size_t)lx * (lx + 1) + 3 * epc * n3 + nst * epc * n3 * 8) + 16 * nst + 64;
    return bytes <= 227 * 1024 && epc * lx * lx <= 1024;
}

// native FP64 line-transform operator (variant 9; sem_ax_ln.cu) and its
// constant-bank even/odd tables of order lx ([dir][A/B][P][P])
int dispatch_ax_ln_entry(sem_handle* h, int lx, const AxParams<double>& a, bool fused, cudaStream_t s);
int ln_set_coef(const double* cf, int lx);

// BF16 split-precision tensor-core operator for FP32 data, lx = 8 (sem_ax_tc.cu)
int dispatch_ax_tc(sem_handle* h, int lx, const AxParams<float>& a, bool fused, cudaStream_t s);

// per-precision entry points (sem_ax_f64.cu, sem_ax_f32.cu)
int dispatch_ax_f64(sem_handle* h, int lx, const AxParams<double>& a, bool fused, cudaStream_t s);
int dispatch_ax_f64_plain(sem_handle* h, int lx, const AxParams<double>& a, cudaStream_t s);
int dispatch_ax_f32_plain(sem_handle* h, int lx, const AxParams<float>& a, cudaStream_t s);
int dispatch_ax_f32(sem_handle* h, int lx, const AxParams<float>& a, bool fused, cudaStream_t s);

}  // namespace sem
