// Device helpers shared by the kernels of libsem: deterministic block and grid
// reductions, streaming loads, and the CG scalar updates.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sem_internal.h"

namespace sem {

template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) { return __ldcs(p); }
template <typename T>
__device__ __forceinline__ void st_stream(T* p, T v) { __stcs(p, v); }
// Output of an operator launch: inside the CG loop (KEEP) the next launch
// reads it at once, so it is stored with the default policy and can stay in
// L2; a plain operator application streams it out (evict-first).
template <bool KEEP, typename T>
__device__ __forceinline__ void st_keep(T* p, T v) {
    if (KEEP)
        *p = v;
    else
        __stcs(p, v);
}

// Sum of NV values over the block (blockDim.x a multiple of 32, <= 1024).
// Fixed shuffle/tree order: bit-reproducible for a fixed block size.  The
// result is valid in thread 0.  `red` holds NV*32 doubles of shared memory.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red) {
#pragma unroll
    for (int q = 0; q < NV; q++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; q++) red[q * 32 + wid] = v[q];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < NV; q++) {
            v[q] = lane < nw ? red[q * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
        }
    }
}

// Grid-wide deterministic sum: every block writes its block sum to
// partials[q * kMaxPartials + blockIdx.x]; the last block to arrive (a ticket
// counter decides who, not what is summed) adds the partials in block order
// and calls fin(sums) in thread 0, then resets the counter for the next
// launch.  Returns nothing; fin runs exactly once per launch.
template <int NV, typename Fin>
__device__ __forceinline__ void grid_sum_finalize(double (&v)[NV], double* partials,
                                                  unsigned int* counter, Fin fin) {
    __shared__ double red[NV * 32];
    __shared__ int is_last;
    block_sum<NV>(v, red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; q++) partials[q * kMaxPartials + blockIdx.x] = v[q];
        __threadfence();
        const unsigned int t = atomicAdd(counter, 1u);
        is_last = (t == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        double acc[NV];
#pragma unroll
        for (int q = 0; q < NV; q++) acc[q] = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
            for (int q = 0; q < NV; q++) acc[q] += __ldcg(&partials[q * kMaxPartials + b]);
        block_sum<NV>(acc, red);
        if (threadIdx.x == 0) {
            fin(acc);
            *counter = 0u;
        }
    }
}

// Float-pair accumulation for the block and grid reductions of FP32 kernels:
// the FP64 pipe of this GPU runs at 1/64 of the FP32 rate, so per-thread sums
// stay in (hi, lo) float pairs (TwoSum of the high parts, low parts in FP32,
// ~2^-48 relative) and only thread 0 of each block and the last block go to
// FP64.
__device__ __forceinline__ void fpair_add(float& h, float& l, float v) {
    const float s = h + v;
    const float bb = s - h;
    l += (h - (s - bb)) + (v - bb);
    h = s;
}
__device__ __forceinline__ void fpair_add2(float& h, float& l, float bh, float bl) {
    const float s = h + bh;
    const float bb = s - h;
    l += ((h - (s - bb)) + (bh - bb)) + bl;
    h = s;
}

// Sum of NV float pairs over the block (fixed shuffle/tree order); valid in
// thread 0.  `red` holds 2 * NV * 32 floats of shared memory.
template <int NV>
__device__ __forceinline__ void block_sum_pair(float (&h)[NV], float (&l)[NV], float* red) {
#pragma unroll
    for (int q = 0; q < NV; q++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_down_sync(0xffffffffu, h[q], o);
            const float ol = __shfl_down_sync(0xffffffffu, l[q], o);
            fpair_add2(h[q], l[q], oh, ol);
        }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; q++) {
            red[q * 32 + wid] = h[q];
            red[(NV + q) * 32 + wid] = l[q];
        }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < NV; q++) {
            h[q] = lane < nw ? red[q * 32 + lane] : 0.f;
            l[q] = lane < nw ? red[(NV + q) * 32 + lane] : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float oh = __shfl_down_sync(0xffffffffu, h[q], o);
                const float ol = __shfl_down_sync(0xffffffffu, l[q], o);
                fpair_add2(h[q], l[q], oh, ol);
            }
        }
    }
}

// grid_sum_finalize for per-thread float pairs: the block sums become FP64
// partials in thread 0; the last block adds them in FP64 in block order.
template <int NV, typename Fin>
__device__ __forceinline__ void grid_sum_finalize_pair(float (&h)[NV], float (&l)[NV], double* partials,
                                                       unsigned int* counter, Fin fin) {
    __shared__ float redf[2 * NV * 32];
    __shared__ double red[NV * 32];
    __shared__ int is_last;
    block_sum_pair<NV>(h, l, redf);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; q++) partials[q * kMaxPartials + blockIdx.x] = (double)h[q] + (double)l[q];
        __threadfence();
        const unsigned int t = atomicAdd(counter, 1u);
        is_last = (t == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        double acc[NV];
#pragma unroll
        for (int q = 0; q < NV; q++) acc[q] = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
            for (int q = 0; q < NV; q++) acc[q] += __ldcg(&partials[q * kMaxPartials + b]);
        block_sum<NV>(acc, red);
        if (threadIdx.x == 0) {
            fin(acc);
            *counter = 0u;
        }
    }
}

// CG scalar step after <p, A p> is known (Sec. II-B, P-CG).
__device__ __forceinline__ void cg_set_alpha(CGState* st, double pap) {
    st->pap = pap;
    if (!(pap > 0.0) || !isfinite(pap)) {
        st->alpha = 0.0;
        st->done = 1;
        st->status = SEM_EBREAKDOWN;
    } else {
        st->alpha = st->rho / pap;
    }
}

// CG scalar step after <r, z> and <r, r> of the new residual are known.
__device__ __forceinline__ void cg_set_rho(CGState* st, double rz, double rr) {
    st->rho_old = st->rho;
    st->rho = rz;
    st->rr = rr;
    st->iter += 1;
    if (!isfinite(rr) || !isfinite(rz)) {
        st->done = 1;
        st->status = SEM_EBREAKDOWN;
    } else if (rr <= st->tol2) {
        st->done = 1;
        st->status = SEM_OK;
    } else if (st->iter >= st->max_iter) {
        st->done = 1;
        st->status = SEM_ENOTCONV;
    }
}

// p = z (no earlier direction) in this iteration
__device__ __forceinline__ bool cg_first(const CGState* st) { return st->iter == 0 && !st->carry; }

__device__ __forceinline__ double cg_beta(const CGState* st) {
    return cg_first(st) ? 0.0 : st->rho / st->rho_old;
}

// Bounded grid barrier of a cooperative launch: returns false (error word
// set) when the other CTAs did not arrive within the budget.
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, int* err, long long budget, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* gen = bar + 1;
        const unsigned int g0 = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g0) {
                if (clock64() - t0 > budget) {
                    ok = 0;
                    atomicExch(err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

}  // namespace sem
