// Local operator kernels with bulk-copy staging: each CTA walks its element
// groups through a ring of NST shared-memory stages.  One elected thread
// fills a stage with cp.async.bulk copies (the group's u, or z and p, and its
// six factor blocks, each one contiguous run of global memory) that signal an
// mbarrier; the CTA computes group g while the copies of the next NST-1
// groups are in flight, and refills the stage as soon as phase 1 has consumed
// it.  The arithmetic is that of ax_group (sem_ax.cuh): same contractions,
// same order.  Only for even lx (element blocks are multiples of 16 bytes).
#pragma once

#include <type_traits>

#include "sem_ax.cuh"

namespace sem {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar` for at most ~`budget` clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long budget) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > budget) return false;
    return true;
}

constexpr long long kWaitBudget = 4000000000LL;  // about two seconds at 2 GHz

// D of every order in constant memory (one copy per translation unit, filled
// at set-up): entries indexed with compile-time (k, l) become constant-bank
// operands of the FMAs instead of shared-memory loads.
static __constant__ float c_bulkD32[kMaxLx + 1][kMaxLx * kMaxLx];
static __constant__ double c_bulkD64[kMaxLx + 1][kMaxLx * kMaxLx];

template <typename T>
__device__ __forceinline__ T bulk_d(int lx, int idx) {
    if constexpr (sizeof(T) == 4)
        return c_bulkD32[lx][idx];
    else
        return c_bulkD64[lx][idx];
}

// LX consecutive values of shared memory into registers with the widest
// aligned vector loads (rows start on multiples of LX*sizeof(T) bytes).
template <typename T, int LX>
__device__ __forceinline__ void load_row(const T* p, T (&r)[LX]) {
    if constexpr (sizeof(T) == 4 && LX % 4 == 0) {
#pragma unroll
        for (int q = 0; q < LX / 4; q++) {
            const float4 v = reinterpret_cast<const float4*>(p)[q];
            r[4 * q] = v.x;
            r[4 * q + 1] = v.y;
            r[4 * q + 2] = v.z;
            r[4 * q + 3] = v.w;
        }
    } else if constexpr (sizeof(T) == 4 && LX % 2 == 0) {
#pragma unroll
        for (int q = 0; q < LX / 2; q++) {
            const float2 v = reinterpret_cast<const float2*>(p)[q];
            r[2 * q] = v.x;
            r[2 * q + 1] = v.y;
        }
    } else if constexpr (sizeof(T) == 8 && LX % 2 == 0) {
#pragma unroll
        for (int q = 0; q < LX / 2; q++) {
            const double2 v = reinterpret_cast<const double2*>(p)[q];
            r[2 * q] = v.x;
            r[2 * q + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < LX; q++) r[q] = p[q];
    }
}

template <typename T, int LX, int EPC, int NST, bool FUSED>
struct BulkCfg {
    static constexpr int N2 = LX * LX, N3 = LX * LX * LX, DP = LX + 1;
    static constexpr int USED = EPC * N2;
    static constexpr int THREADS = ((USED + 31) / 32) * 32;
    static constexpr int IN = FUSED ? 2 : 1;                   // u, or z and p
    static constexpr size_t STAGE = (size_t)EPC * N3 * (IN + 6);  // elements of T per stage
    static constexpr size_t WORK = (size_t)LX * DP + 3 * (size_t)EPC * N3;
    static constexpr size_t BYTES = sizeof(T) * (WORK + NST * STAGE) + 16 * NST + 64;
    static_assert(LX % 2 == 0, "bulk staging needs even lx");
};

template <typename T, int LX, int EPC, int NST, bool FUSED, bool BATCH = false>
__global__ void __launch_bounds__(BulkCfg<T, LX, EPC, NST, FUSED>::THREADS)
    ax_bulk_kernel(AxParams<T> a) {
    using C = BulkCfg<T, LX, EPC, NST, FUSED>;
    constexpr int N2 = C::N2, N3 = C::N3, DP = C::DP;
    extern __shared__ __align__(128) unsigned char smem_bulk[];
    T* sD = reinterpret_cast<T*>(smem_bulk);
    T* su = sD + ((LX * DP + 3) & ~3);  // 16-byte aligned
    T* sr = su + EPC * N3;
    T* ss = sr + EPC * N3;
    T* stage0 = ss + EPC * N3;          // EPC*N3*sizeof(T) is a multiple of 16 for even LX
    uint64_t* bars = reinterpret_cast<uint64_t*>(stage0 + NST * C::STAGE);
    __shared__ int abort_flag;

    double beta = 0.0;
    bool first = false;
    __shared__ T s_tbeta;  // beta, divided and converted once by thread 0 (GB300's FP64 pipe is slow)
    if (FUSED && !BATCH) {
        if (a.st->done) return;  // uniform over the grid
        if (threadIdx.x == 0) s_tbeta = (T)cg_beta(a.st);
        first = cg_first(a.st);
    } else if (!FUSED && a.skip_st && a.skip_st->done) {
        return;  // uniform over the grid
    }
    T tbeta = T(0);
    const int64_t ngroups = BATCH ? a.ngroups : (a.E + EPC - 1) / EPC;
    __shared__ double red[32];
    __shared__ int is_last;
    const int tid = threadIdx.x;
    const int el = tid / N2;
    const int ij = tid - el * N2;
    const int i = ij % LX, j = ij / LX;
    const bool active = el < EPC;
    const int so = (active ? el : 0) * N3;

    // stage s of group g: [in0 | in1 | G], each in element order
    // local index of the first element of group g, and its element count
    auto group_off = [&](int64_t g) -> int64_t { return BATCH ? a.loc[g] : g * EPC * N3; };
    auto group_cnt = [&](int64_t g) -> int {
        return BATCH ? a.cnt[g] : (int)(a.E - g * EPC < EPC ? a.E - g * EPC : EPC);
    };
    auto issue = [&](int s, int64_t g) {
        const int64_t off = group_off(g);
        const int cnt = group_cnt(g);
        T* st = stage0 + s * C::STAGE;
        const uint32_t bin = (uint32_t)(cnt * N3 * sizeof(T));
        const uint32_t bG = 6u * bin;
        mbar_expect_tx(&bars[s], (uint32_t)C::IN * bin + bG + a.tx_extra);
        if (FUSED) {
            bulk_load(st, a.z + off, bin, &bars[s]);
            bulk_load(st + EPC * N3, a.p + off, bin, &bars[s]);
        } else {
            bulk_load(st, a.u + off, bin, &bars[s]);
        }
        bulk_load(st + C::IN * EPC * N3, a.G + 6 * off, bG, &bars[s]);
    };

    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < NST; s++) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    for (int t = tid; t < LX * LX; t += blockDim.x) sD[(t / LX) * DP + (t % LX)] = a.D[t];
    __syncthreads();
    if (FUSED && !BATCH) tbeta = s_tbeta;
    // this thread's rows (r, s derivatives) and columns (transposed ones) of D
    T Dri[LX], Drj[LX], Dci[LX], Dcj[LX];
#pragma unroll
    for (int l = 0; l < LX; l++) {
        Dri[l] = sD[i * DP + l];
        Drj[l] = sD[j * DP + l];
        Dci[l] = sD[l * DP + i];
        Dcj[l] = sD[l * DP + j];
    }
    // A batched CG launch skips the groups of converged solves: their stages
    // are never filled, so no bytes move for them.  A solve's done flag cannot
    // change while any of its groups is still to come in this launch (only the
    // CTA that finishes its last group writes its state), so the producer's
    // decision at issue time and the consumers' at use time agree.  Each stage
    // keeps its own phase bit, flipped only by fills that were waited for.
    auto skipped = [&](int64_t g) -> bool { return BATCH && FUSED && a.st[a.solve[g]].done; };
    __shared__ unsigned inflight;  // stages with a fill in flight (thread 0's bookkeeping, for the drain)
    if (tid == 0) {
        inflight = 0u;
        for (int s = 0; s < NST; s++) {
            const int64_t g = blockIdx.x + (int64_t)s * gridDim.x;
            if (g < ngroups && !skipped(g)) {
                issue(s, g);
                inflight |= 1u << s;
            }
        }
    }

    double pap = 0.0;
    float paph = 0.f, papl = 0.f;  // FP32 kernels: <p, A p> as a float pair (no FP64 per group)
    int64_t it = 0;
    uint32_t phase = 0u;  // bit s: parity of the next completed fill of stage s
    __shared__ int s_skip;
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x, it++) {
        const int s = (int)(it % NST);
        if (BATCH && FUSED) {
            if (tid == 0) s_skip = skipped(g) ? 1 : 0;
            __syncthreads();
        }
        const bool skip = BATCH && FUSED && s_skip;
        if (!skip) {
            if (!mbar_wait_bounded(&bars[s], (phase >> s) & 1u, a.wait_budget))
                abort_flag = 1;  // the stage stays in flight: the drain waits for its phase again
            else
                phase ^= 1u << s;
        }
        __syncthreads();
        if (abort_flag) break;
        if (tid == 0 && !skip) inflight &= ~(1u << s);
        int sol = 0;
        if (skip) {  // converged solve: its stage was never filled; fill it with the group NST rounds ahead
            if (tid == 0) {
                const int64_t gn = g + (int64_t)NST * gridDim.x;
                if (gn < ngroups && !skipped(gn)) {
                    issue(s, gn);
                    inflight |= 1u << s;
                }
            }
            __syncthreads();  // s_skip is rewritten next round
            continue;
        }
        if (BATCH && FUSED) {
            sol = a.solve[g];
            const CGState* stg = a.st + sol;
            beta = cg_beta(stg);
            first = cg_first(stg);
            tbeta = (T)beta;
        }
        const T* st = stage0 + s * C::STAGE;
        const bool valid = active && el < group_cnt(g);
        const int64_t base = group_off(g) + (int64_t)(active ? el : 0) * N3 + ij;
        // phase 0: this thread's column of u (or z + beta p)
        T ucol[LX];
#pragma unroll
        for (int k = 0; k < LX; k++) {
            T v = st[so + k * N2 + ij];
            if (FUSED) {
                const T pp = first ? T(0) : st[EPC * N3 + so + k * N2 + ij];
                v = fma(tbeta, pp, v);
                if (valid) a.p[base + k * N2] = v;
            }
            ucol[k] = v;
            if (active) su[so + k * N2 + ij] = v;
        }
        __syncthreads();
        // phase 1: derivatives and weighting by the factors of the stage
        const T* Gs = st + C::IN * EPC * N3 + (active ? el : 0) * 6 * N3 + ij;
        T wt[LX];
#pragma unroll
        for (int k = 0; k < LX; k++) {
            T ur = T(0), us = T(0), ut = T(0);
            T row[LX];
            load_row<T, LX>(su + so + k * N2 + j * LX, row);
#pragma unroll
            for (int l = 0; l < LX; l++) {
                ur = fma(Dri[l], row[l], ur);
                us = fma(Drj[l], su[so + k * N2 + l * LX + i], us);
                ut = fma(bulk_d<T>(LX, k * LX + l), ucol[l], ut);
            }
            const T g11 = Gs[0 * N3 + k * N2], g12 = Gs[1 * N3 + k * N2], g13 = Gs[2 * N3 + k * N2];
            const T g22 = Gs[3 * N3 + k * N2], g23 = Gs[4 * N3 + k * N2], g33 = Gs[5 * N3 + k * N2];
            const T wr = fma(g11, ur, fma(g12, us, g13 * ut));
            const T ws = fma(g12, ur, fma(g22, us, g23 * ut));
            wt[k] = fma(g13, ur, fma(g23, us, g33 * ut));
            if (active) {
                sr[so + k * N2 + ij] = wr;
                ss[so + k * N2 + ij] = ws;
            }
        }
        __syncthreads();
        // the stage is consumed: refill it with the group NST rounds ahead
        if (tid == 0) {
            const int64_t gn = g + (int64_t)NST * gridDim.x;
            if (gn < ngroups && !skipped(gn)) {
                issue(s, gn);
                inflight |= 1u << s;
            }
        }
        // phase 2: transposed contractions
        T pw = T(0);
#pragma unroll
        for (int k = 0; k < LX; k++) {
            T acc = T(0);
            T row[LX];
            load_row<T, LX>(sr + so + k * N2 + j * LX, row);
            if constexpr (sizeof(T) == 4 && FUSED) {
                // the three chains of ax_group's FP32 CG form, in its order
                T ar = T(0), as = T(0), at = T(0);
#pragma unroll
                for (int l = 0; l < LX; l++) {
                    ar = fma(Dci[l], row[l], ar);
                    as = fma(Dcj[l], ss[so + k * N2 + l * LX + i], as);
                    at = fma(bulk_d<T>(LX, l * LX + k), wt[l], at);
                }
                acc = (ar + as) + at;
            } else {
#pragma unroll
                for (int l = 0; l < LX; l++) {
                    acc = fma(Dci[l], row[l], acc);
                    acc = fma(Dcj[l], ss[so + k * N2 + l * LX + i], acc);
                    acc = fma(bulk_d<T>(LX, l * LX + k), wt[l], acc);
                }
            }
            if (valid) {
                st_keep<FUSED>(a.w + base + k * N2, acc);
                if (FUSED) pw = fma(ucol[k], acc, pw);
            }
        }
        if (FUSED && BATCH) {
            double v[1] = {(double)pw};
            block_sum<1>(v, red);
            if (tid == 0) {
                a.gpart[a.goff + g] = v[0];
                __threadfence();
                is_last = (atomicAdd(&a.scount[sol], 1u) == (unsigned)a.sgcount[sol] - 1u) ? 1 : 0;
            }
            __syncthreads();
            if (is_last) {
                __threadfence();
                const int f = a.sgfirst[sol], c = a.sgcount[sol];
                double acc[1] = {0.0};
                for (int q = tid; q < c; q += blockDim.x) acc[0] += __ldcg(&a.gpart[f + q]);
                block_sum<1>(acc, red);
                if (tid == 0) {
                    cg_set_alpha(a.st + sol, acc[0]);
                    a.scount[sol] = 0u;
                }
            }
        } else if (FUSED) {
            if constexpr (sizeof(T) == 4)
                fpair_add(paph, papl, pw);
            else
                pap += (double)pw;
        }
        __syncthreads();
    }
    if (abort_flag) {
        // a copy never completed: report, let the other copies land, return.
        // No stage is issued after the failed wait (the loop breaks before its
        // refill).  The drain is bounded and best-effort: each stage still in
        // flight gets a quarter of the wait budget, after which the CTA exits
        // whether or not its copies have landed.
        if (tid == 0) {
            atomicExch(a.err, 1);
            for (int s = 0; s < NST; s++)
                if (inflight & (1u << s)) mbar_wait_bounded(&bars[s], (phase >> s) & 1u, a.wait_budget / 4);
        }
        return;
    }
    if (FUSED && !BATCH) {
        CGState* stt = a.st;
        if constexpr (sizeof(T) == 4) {
            float h[1] = {paph}, l[1] = {papl};
            grid_sum_finalize_pair<1>(h, l, a.partials, a.counter,
                                      [&](double (&acc)[1]) { cg_set_alpha(stt, acc[0]); });
        } else {
            double v[1] = {pap};
            grid_sum_finalize<1>(v, a.partials, a.counter, [&](double (&acc)[1]) { cg_set_alpha(stt, acc[0]); });
        }
    }
}

// Fill this translation unit's constant copy of D for order lx.
template <typename T>
inline int bulk_set_d(const T* D, int lx) {
    cudaError_t e;
    if constexpr (sizeof(T) == 4)
        e = cudaMemcpyToSymbol(c_bulkD32, D, sizeof(T) * lx * lx, sizeof(T) * (size_t)lx * kMaxLx * kMaxLx);
    else
        e = cudaMemcpyToSymbol(c_bulkD64, D, sizeof(T) * lx * lx, sizeof(T) * (size_t)lx * kMaxLx * kMaxLx);
    return e == cudaSuccess ? SEM_OK : cuda_fail(e, "cudaMemcpyToSymbol(D)");
}

template <typename T, int LX, int EPC, int NST, bool FUSED>
inline int launch_ax_bulk_t(sem_handle* h, const AxParams<T>& a, cudaStream_t s) {
    using C = BulkCfg<T, LX, EPC, NST, FUSED>;
    if constexpr (C::BYTES > 227 * 1024) {
        return fail(SEM_EINVAL, "bulk variant does not fit in shared memory");
    } else {
        static int per_sm = -1;
        if (per_sm < 0) {
            cudaFuncSetAttribute(ax_bulk_kernel<T, LX, EPC, NST, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)C::BYTES);
            int nb = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ax_bulk_kernel<T, LX, EPC, NST, FUSED>, C::THREADS,
                                                          C::BYTES);
            per_sm = nb;
        }
        if (per_sm <= 0) return fail(SEM_EINVAL, "bulk variant cannot be resident");
        if (a.dry) return SEM_OK;
        const int64_t ngroups = (a.E + EPC - 1) / EPC;
        int64_t grid = std::min<int64_t>(ngroups, (int64_t)h->sm_count * per_sm);
        grid = std::max<int64_t>(1, std::min<int64_t>(grid, kMaxPartials));
        ax_bulk_kernel<T, LX, EPC, NST, FUSED><<<(int)grid, C::THREADS, C::BYTES, s>>>(a);
        SEM_LAUNCH_CHECK("ax_bulk_kernel");
        h->launches++;
        return SEM_OK;
    }
}

// Batched form: one persistent launch over the element-group list of one order.
template <typename T, int LX, int EPC, int NST, bool FUSED>
inline int launch_ax_bulk_batch_t(sem_handle* h, const AxParams<T>& a, cudaStream_t s) {
    using C = BulkCfg<T, LX, EPC, NST, FUSED>;
    if constexpr (C::BYTES > 227 * 1024) {
        return fail(SEM_EINVAL, "bulk variant does not fit in shared memory");
    } else {
        static int per_sm = -1;
        if (per_sm < 0) {
            cudaFuncSetAttribute(ax_bulk_kernel<T, LX, EPC, NST, FUSED, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES);
            int nb = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ax_bulk_kernel<T, LX, EPC, NST, FUSED, true>,
                                                          C::THREADS, C::BYTES);
            per_sm = nb;
        }
        if (per_sm <= 0) return fail(SEM_EINVAL, "bulk variant cannot be resident");
        if (a.dry || a.ngroups == 0) return SEM_OK;
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(a.ngroups, (int64_t)h->sm_count * per_sm));
        ax_bulk_kernel<T, LX, EPC, NST, FUSED, true><<<(int)grid, C::THREADS, C::BYTES, s>>>(a);
        SEM_LAUNCH_CHECK("ax_bulk_kernel (batched)");
        h->launches++;
        return SEM_OK;
    }
}

template <typename T, int LX, bool FUSED>
inline int dispatch_bulk_batch_cfg(sem_handle* h, const AxParams<T>& a, cudaStream_t s) {
    switch (a.variant) {
        case 1: return launch_ax_bulk_batch_t<T, LX, kBulkCfg[0][0], kBulkCfg[0][1], FUSED>(h, a, s);
        case 2: return launch_ax_bulk_batch_t<T, LX, kBulkCfg[1][0], kBulkCfg[1][1], FUSED>(h, a, s);
        case 3: return launch_ax_bulk_batch_t<T, LX, kBulkCfg[2][0], kBulkCfg[2][1], FUSED>(h, a, s);
        case 4: return launch_ax_bulk_batch_t<T, LX, kBulkCfg[3][0], kBulkCfg[3][1], FUSED>(h, a, s);
        default: return fail(SEM_EINVAL, "unknown operator variant");
    }
}

template <typename T, bool FUSED>
inline int dispatch_ax_bulk_batch(sem_handle* h, int lx, const AxParams<T>& a, cudaStream_t s) {
    switch (lx) {
        case 4: return dispatch_bulk_batch_cfg<T, 4, FUSED>(h, a, s);
        case 6: return dispatch_bulk_batch_cfg<T, 6, FUSED>(h, a, s);
        case 8: return dispatch_bulk_batch_cfg<T, 8, FUSED>(h, a, s);
        case 10: return dispatch_bulk_batch_cfg<T, 10, FUSED>(h, a, s);
        case 12: return dispatch_bulk_batch_cfg<T, 12, FUSED>(h, a, s);
        default: return fail(SEM_EINVAL, "bulk staging needs lx in {4, 6, 8, 10, 12}");
    }
}

template <typename T, int LX, bool FUSED>
inline int dispatch_bulk_cfg(sem_handle* h, const AxParams<T>& a, cudaStream_t s) {
    switch (a.variant) {
        case 1: return launch_ax_bulk_t<T, LX, kBulkCfg[0][0], kBulkCfg[0][1], FUSED>(h, a, s);
        case 2: return launch_ax_bulk_t<T, LX, kBulkCfg[1][0], kBulkCfg[1][1], FUSED>(h, a, s);
        case 3: return launch_ax_bulk_t<T, LX, kBulkCfg[2][0], kBulkCfg[2][1], FUSED>(h, a, s);
        case 4: return launch_ax_bulk_t<T, LX, kBulkCfg[3][0], kBulkCfg[3][1], FUSED>(h, a, s);
        default: return fail(SEM_EINVAL, "unknown operator variant");
    }
}

template <typename T, bool FUSED>
inline int dispatch_ax_bulk(sem_handle* h, int lx, const AxParams<T>& a, cudaStream_t s) {
    switch (lx) {
        case 4: return dispatch_bulk_cfg<T, 4, FUSED>(h, a, s);
        case 6: return dispatch_bulk_cfg<T, 6, FUSED>(h, a, s);
        case 8: return dispatch_bulk_cfg<T, 8, FUSED>(h, a, s);
        case 10: return dispatch_bulk_cfg<T, 10, FUSED>(h, a, s);
        case 12: return dispatch_bulk_cfg<T, 12, FUSED>(h, a, s);
        default: return fail(SEM_EINVAL, "bulk staging needs lx in {4, 6, 8, 10, 12}");
    }
}

}  // namespace sem
