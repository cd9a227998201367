// Kernels of the batched solve over many independent meshes: the local
// operator over a list of element groups (one launch per order present, every
// unconverged solve of that order in the same persistent launch), with the
// per-solve CG scalars in device memory.  Each solve's <p, A p> is summed from
// its group partials in group order by the CTA that finishes the solve's last
// group, so every solve of a batch is bit-reproducible.
#pragma once

#include "sem_ax.cuh"

namespace sem {

template <typename T>
struct BatchAxParams {
    const T* u;            // plain variant input
    const T* z;            // fused variant
    T* p;
    T* w;
    const T* G;
    const T* D;
    const int64_t* loc;    // group lists of this order
    const int* cnt;
    const int* solve;
    int64_t ngroups;
    int64_t goff;
    CGState* st;           // per-solve states
    const int* sgfirst;
    const int* sgcount;
    double* gpart;
    unsigned int* scount;
    int dry;
    const T* mass;         // [n] Helmholtz term h2 B, null for Poisson
};

template <typename T, int LX, bool FUSED>
__global__ void __launch_bounds__(AxCfg<LX>::THREADS) ax_batch_kernel(BatchAxParams<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const AxSmem<T, LX> sm(smem_raw);
    __shared__ double red[32];
    __shared__ float redf[64];
    __shared__ int is_last;
    // the solve's scalars, read and converted once per group by thread 0 (an
    // FP64 division per thread would load GB300's slow FP64 pipe)
    __shared__ T s_tbeta;
    __shared__ int s_done, s_first;
    ax_load_d<T, LX>(sm.sD, a.D);
    const AxThread<LX> th;
    __syncthreads();
    for (int64_t g = blockIdx.x; g < a.ngroups; g += gridDim.x) {
        const int s = a.solve[g];
        CGState* st = a.st + s;
        T tbeta = T(0);
        bool first = false;
        if (FUSED) {
            if (threadIdx.x == 0) {
                // no write to this solve's state can happen before all its groups are done
                s_done = st->done;
                s_tbeta = s_done ? T(0) : (T)cg_beta(st);
                s_first = cg_first(st);
            }
            __syncthreads();
            if (s_done) {
                __syncthreads();  // thread 0 rewrites the scalars next round
                continue;
            }
            tbeta = s_tbeta;
            first = s_first != 0;
        }
        const int64_t loc = a.loc[g];
        const bool valid = th.active && th.el < a.cnt[g];
        const T pw = ax_group<T, LX, FUSED>(sm, th, th.el, valid, FUSED ? nullptr : a.u + loc,
                                            FUSED ? a.z + loc : nullptr, FUSED ? a.p + loc : nullptr,
                                            a.w + loc, a.G + 6 * loc, tbeta, first,
                                            a.mass ? a.mass + loc : nullptr);
        if (FUSED) {
            double v[1] = {0.0};
            if constexpr (sizeof(T) == 4) {  // float-pair block sum: FP64 only in thread 0
                float ph[1] = {(float)pw}, pl[1] = {0.f};
                block_sum_pair<1>(ph, pl, redf);
                v[0] = (double)ph[0] + (double)pl[0];
            } else {
                v[0] = (double)pw;
                block_sum<1>(v, red);
            }
            if (threadIdx.x == 0) {
                a.gpart[a.goff + g] = v[0];
                __threadfence();
                is_last = (atomicAdd(&a.scount[s], 1u) == (unsigned)a.sgcount[s] - 1u) ? 1 : 0;
            }
            __syncthreads();
            if (is_last) {
                __threadfence();
                const int f = a.sgfirst[s], c = a.sgcount[s];
                double acc[1] = {0.0};
                for (int q = threadIdx.x; q < c; q += blockDim.x) acc[0] += __ldcg(&a.gpart[f + q]);
                block_sum<1>(acc, red);
                if (threadIdx.x == 0) {
                    cg_set_alpha(st, acc[0]);
                    a.scount[s] = 0u;
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// One launch over the element groups of every order of a batch (orders up to
// kMultiMaxLx): each group carries its order, and the CTA takes the slab
// operator of that order for it (the same arithmetic, in the same order, as
// ax_batch_kernel<T, LX>, so results are bit-identical).  The D matrices of
// all orders present sit in shared memory for the whole launch; the element
// slots are sized for the largest order present.
// ---------------------------------------------------------------------------
constexpr int kMultiMaxLx = 10;
constexpr int kMultiThreads = 256;  // >= AxCfg<LX>::THREADS for every LX <= kMultiMaxLx

// offset of order lx's padded D (lx rows of lx + 1) in the shared D table
__host__ __device__ constexpr int multi_d_off(int lx) {
    int o = 0;
    for (int m = 2; m < lx; m++) o += m * (m + 1);
    return o;
}
constexpr int kMultiDTable = (multi_d_off(kMultiMaxLx + 1) + 1) / 2 * 2;  // even: slots stay 16-byte aligned

template <typename T>
struct MultiOrder {
    const T* D[kMultiMaxLx + 1];  // D of each order present (nullptr for the others)
    const uint8_t* lx;            // [ngroups] order of every group
};

template <typename T, int LX>
constexpr size_t multi_slot_elems() {
    return 3 * (size_t)AxCfg<LX>::EPC * AxCfg<LX>::N3;
}

template <typename T, int LX, bool FUSED>
__device__ __forceinline__ T multi_group(T* dtab, T* slots, const BatchAxParams<T>& a, int64_t g, T tbeta,
                                         bool first) {
    const AxSmem<T, LX> sm(dtab + multi_d_off(LX), slots);
    const AxThread<LX> th;
    const int64_t loc = a.loc[g];
    const bool valid = th.active && th.el < a.cnt[g];
    return ax_group<T, LX, FUSED>(sm, th, th.el, valid, FUSED ? nullptr : a.u + loc, FUSED ? a.z + loc : nullptr,
                                  FUSED ? a.p + loc : nullptr, a.w + loc, a.G + 6 * loc, tbeta, first,
                                  a.mass ? a.mass + loc : nullptr);
}

template <typename T, bool FUSED>
__global__ void __launch_bounds__(kMultiThreads, 2) ax_batch_multi_kernel(BatchAxParams<T> a, MultiOrder<T> mo) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* dtab = reinterpret_cast<T*>(smem_raw);
    T* slots = dtab + kMultiDTable;
    __shared__ double red[32];
    __shared__ float redf[64];
    __shared__ int is_last;
    __shared__ T s_tbeta;
    __shared__ int s_done, s_first;
#pragma unroll 1
    for (int lx = 2; lx <= kMultiMaxLx; lx++) {
        const T* D = mo.D[lx];
        if (!D) continue;
        for (int t = threadIdx.x; t < lx * lx; t += blockDim.x)
            dtab[multi_d_off(lx) + (t / lx) * (lx + 1) + (t % lx)] = D[t];
    }
    __syncthreads();
    for (int64_t g = blockIdx.x; g < a.ngroups; g += gridDim.x) {
        const int s = a.solve[g];
        CGState* st = a.st + s;
        T tbeta = T(0);
        bool first = false;
        if (FUSED) {
            if (threadIdx.x == 0) {
                s_done = st->done;
                s_tbeta = s_done ? T(0) : (T)cg_beta(st);
                s_first = cg_first(st);
            }
            __syncthreads();
            if (s_done) {
                __syncthreads();
                continue;
            }
            tbeta = s_tbeta;
            first = s_first != 0;
        }
        T pw = T(0);
        switch (mo.lx[g]) {  // uniform over the CTA: every thread takes the same order
            case 2: pw = multi_group<T, 2, FUSED>(dtab, slots, a, g, tbeta, first); break;
            case 3: pw = multi_group<T, 3, FUSED>(dtab, slots, a, g, tbeta, first); break;
            case 4: pw = multi_group<T, 4, FUSED>(dtab, slots, a, g, tbeta, first); break;
            case 5: pw = multi_group<T, 5, FUSED>(dtab, slots, a, g, tbeta, first); break;
            case 6: pw = multi_group<T, 6, FUSED>(dtab, slots, a, g, tbeta, first); break;
            case 7: pw = multi_group<T, 7, FUSED>(dtab, slots, a, g, tbeta, first); break;
            case 8: pw = multi_group<T, 8, FUSED>(dtab, slots, a, g, tbeta, first); break;
            case 9: pw = multi_group<T, 9, FUSED>(dtab, slots, a, g, tbeta, first); break;
            default: pw = multi_group<T, 10, FUSED>(dtab, slots, a, g, tbeta, first); break;
        }
        if (FUSED) {
            double v[1] = {0.0};
            if constexpr (sizeof(T) == 4) {
                float ph[1] = {(float)pw}, pl[1] = {0.f};
                block_sum_pair<1>(ph, pl, redf);
                v[0] = (double)ph[0] + (double)pl[0];
            } else {
                v[0] = (double)pw;
                block_sum<1>(v, red);
            }
            if (threadIdx.x == 0) {
                a.gpart[g] = v[0];
                __threadfence();
                is_last = (atomicAdd(&a.scount[s], 1u) == (unsigned)a.sgcount[s] - 1u) ? 1 : 0;
            }
            __syncthreads();
            if (is_last) {
                __threadfence();
                const int f = a.sgfirst[s], c = a.sgcount[s];
                double acc[1] = {0.0};
                for (int q = threadIdx.x; q < c; q += blockDim.x) acc[0] += __ldcg(&a.gpart[f + q]);
                block_sum<1>(acc, red);
                if (threadIdx.x == 0) {
                    cg_set_alpha(st, acc[0]);
                    a.scount[s] = 0u;
                }
            }
        }
        __syncthreads();
    }
}

// bytes of shared memory the multi-order kernel needs for the orders present
template <typename T>
inline size_t multi_smem_bytes(const bool (&present)[kMaxLx + 1]) {
    size_t slots = 0;
    auto take = [&](int lx, size_t n) {
        if (present[lx] && n > slots) slots = n;
    };
    take(2, multi_slot_elems<T, 2>()); take(3, multi_slot_elems<T, 3>()); take(4, multi_slot_elems<T, 4>());
    take(5, multi_slot_elems<T, 5>()); take(6, multi_slot_elems<T, 6>()); take(7, multi_slot_elems<T, 7>());
    take(8, multi_slot_elems<T, 8>()); take(9, multi_slot_elems<T, 9>()); take(10, multi_slot_elems<T, 10>());
    return sizeof(T) * (kMultiDTable + slots);
}

int launch_ax_batch_multi_f64(sem_handle* h, const BatchAxParams<double>& a, const MultiOrder<double>& mo,
                              size_t smem, bool fused, cudaStream_t s);
int launch_ax_batch_multi_f32(sem_handle* h, const BatchAxParams<float>& a, const MultiOrder<float>& mo,
                              size_t smem, bool fused, cudaStream_t s);

template <typename T, int LX, bool FUSED>
inline int launch_ax_batch_t(sem_handle* h, const BatchAxParams<T>& a, cudaStream_t s) {
    using C = AxCfg<LX>;
    constexpr size_t smem = ax_smem_bytes<T, LX>();
    static int per_sm = -1;
    if (per_sm < 0) {
        cudaFuncSetAttribute(ax_batch_kernel<T, LX, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ax_batch_kernel<T, LX, FUSED>, C::THREADS, smem);
        per_sm = nb > 0 ? nb : 1;
    }
    if (a.dry || a.ngroups == 0) return SEM_OK;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(a.ngroups, (int64_t)h->sm_count * per_sm));
    ax_batch_kernel<T, LX, FUSED><<<(int)grid, C::THREADS, smem, s>>>(a);
    SEM_LAUNCH_CHECK("ax_batch_kernel");
    h->launches++;
    return SEM_OK;
}

template <typename T, bool FUSED>
inline int dispatch_ax_batch(sem_handle* h, int lx, const BatchAxParams<T>& a, cudaStream_t s) {
    switch (lx) {
        case 2: return launch_ax_batch_t<T, 2, FUSED>(h, a, s);
        case 3: return launch_ax_batch_t<T, 3, FUSED>(h, a, s);
        case 4: return launch_ax_batch_t<T, 4, FUSED>(h, a, s);
        case 5: return launch_ax_batch_t<T, 5, FUSED>(h, a, s);
        case 6: return launch_ax_batch_t<T, 6, FUSED>(h, a, s);
        case 7: return launch_ax_batch_t<T, 7, FUSED>(h, a, s);
        case 8: return launch_ax_batch_t<T, 8, FUSED>(h, a, s);
        case 9: return launch_ax_batch_t<T, 9, FUSED>(h, a, s);
        case 10: return launch_ax_batch_t<T, 10, FUSED>(h, a, s);
        case 11: return launch_ax_batch_t<T, 11, FUSED>(h, a, s);
        case 12: return launch_ax_batch_t<T, 12, FUSED>(h, a, s);
        case 13: return launch_ax_batch_t<T, 13, FUSED>(h, a, s);
        case 14: return launch_ax_batch_t<T, 14, FUSED>(h, a, s);
        case 15: return launch_ax_batch_t<T, 15, FUSED>(h, a, s);
        case 16: return launch_ax_batch_t<T, 16, FUSED>(h, a, s);
        default: return fail(SEM_EINVAL, "lx out of range");
    }
}

int dispatch_ax_batch_f64(sem_handle* h, int lx, const BatchAxParams<double>& a, bool fused, cudaStream_t s);
int dispatch_ax_batch_f32(sem_handle* h, int lx, const BatchAxParams<float>& a, bool fused, cudaStream_t s);

}  // namespace sem
