// Bandwidth-bound Krylov-basis kernels shared by the GMRES solver and the
// projection onto previous solutions: one Gram-Schmidt pass (subtract a
// combination of basis vectors, dot products with up to 16 of them, the norm)
// and x += Z y, on 16-byte packs of points with the basis loads of a chunk in
// flight together, and a deterministic grid sum.
#pragma once

#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

constexpr int kGmNV = 16;           // dot products per Gram-Schmidt launch
constexpr int kGmMaxRestart = 200;  // largest basis a pass combines

// 16-byte packs of consecutive points: 4 floats or 2 doubles per load
template <typename T>
struct alignas(16) Pk {
    T v[16 / sizeof(T)];
};
template <typename T>
__device__ __forceinline__ Pk<T> ld_pk(const T* p) {
    return *reinterpret_cast<const Pk<T>*>(p);
}
template <int P>
__device__ __forceinline__ void ld_mult(const uint8_t* m, uint8_t (&o)[P]) {
    if constexpr (P == 4) {
        const uint32_t u = *reinterpret_cast<const uint32_t*>(m);
        o[0] = u & 255u;
        o[1] = (u >> 8) & 255u;
        o[2] = (u >> 16) & 255u;
        o[3] = u >> 24;
    } else {
        const uint32_t u = *reinterpret_cast<const uint16_t*>(m);
        o[0] = u & 255u;
        o[1] = u >> 8;
    }
}

// Deterministic grid sum of K per-thread values of type T: warp sums in T,
// block and grid sums in FP64 in a fixed order (the last block to arrive adds
// the block partials, a warp per value); fin receives the K sums in thread 0
// of that block.
template <typename T, int K, typename Fin>
__device__ __forceinline__ void gm_grid_sum(T (&d)[K], double* partials, unsigned int* counter, Fin fin) {
    __shared__ double red[K][8];
    __shared__ double tot[K];
    __shared__ int is_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < K; q++) {
        T v = d[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][wid] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double sum = 0.0;
        for (int q = 0; q < nw; q++) sum += red[threadIdx.x][q];
        partials[threadIdx.x * kMaxPartials + blockIdx.x] = sum;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1) ? 1 : 0;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // the last block: warp w sums the partials of values w, w + nw, ..., each
    // lane a fixed stride of blocks, then a fixed shuffle tree
    for (int q = wid; q < K; q += nw) {
        const double* pq = partials + q * kMaxPartials;
        double acc = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) acc += __ldcg(pq + b);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) tot[q] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        fin(tot);
        *counter = 0u;
    }
}

// One Gram-Schmidt pass over the basis V (vector i at V + i ld):
//   sub_cnt > 0:  w -= sum_{i < sub_cnt} c_i V_i   (c from the device)
//   dot_cnt > 0:  dot_out[i] = <V_{dot_lo + i}, w>  for i < dot_cnt <= NV
//   want_norm:    *norm_out = <w, w>
// in the unique-node inner product (1 / mult weights).  A thread handles one
// 16-byte pack of points per step and loads the basis vectors in chunks of
// eight (all loads of a chunk in flight together); points past the last full
// pack are done one by one in block 0.  Per-thread sums in T.
template <typename T, int NV>
__global__ void __launch_bounds__(256) gm_pass_kernel(T* __restrict__ w, const T* __restrict__ V, int64_t ld,
                                                      int64_t n, int sub_cnt, const double* __restrict__ sub_coef,
                                                      int dot_lo, int dot_cnt, int want_norm,
                                                      const uint8_t* __restrict__ mult, double* __restrict__ dot_out,
                                                      double* __restrict__ norm_out, double* partials,
                                                      unsigned int* counter) {
    constexpr int P = 16 / sizeof(T), CH = 8;
    __shared__ T inv[256];
    __shared__ T cs[kGmMaxRestart + 1];
    for (int q = threadIdx.x; q < 256; q += blockDim.x) inv[q] = q ? (T)1 / (T)q : (T)0;
    for (int q = threadIdx.x; q < sub_cnt; q += blockDim.x) cs[q] = (T)sub_coef[q];
    __syncthreads();
    T d[NV + 1];
#pragma unroll
    for (int q = 0; q <= NV; q++) d[q] = (T)0;
    const T* Vd = V + (int64_t)dot_lo * ld;
    const int64_t np = n / P;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t L0 = q * P;
        Pk<T> wv = ld_pk(w + L0);
        if (sub_cnt > 0) {
            T acc[P];
#pragma unroll
            for (int k = 0; k < P; k++) acc[k] = (T)0;
            for (int i0 = 0; i0 < sub_cnt; i0 += CH) {
                Pk<T> vv[CH];
#pragma unroll
                for (int c = 0; c < CH; c++)
                    if (i0 + c < sub_cnt) vv[c] = ld_pk(V + (int64_t)(i0 + c) * ld + L0);
#pragma unroll
                for (int c = 0; c < CH; c++)
                    if (i0 + c < sub_cnt)
#pragma unroll
                        for (int k = 0; k < P; k++) acc[k] = fma(cs[i0 + c], vv[c].v[k], acc[k]);
            }
#pragma unroll
            for (int k = 0; k < P; k++) wv.v[k] -= acc[k];
            *reinterpret_cast<Pk<T>*>(w + L0) = wv;
        }
        uint8_t mu[P];
        ld_mult<P>(mult + L0, mu);
        T wi[P];
#pragma unroll
        for (int k = 0; k < P; k++) wi[k] = wv.v[k] * inv[mu[k]];
#pragma unroll
        for (int c0 = 0; c0 < NV; c0 += CH) {
            if (c0 < dot_cnt) {
                Pk<T> vv[CH];
#pragma unroll
                for (int c = 0; c < CH; c++)
                    if (c0 + c < dot_cnt) vv[c] = ld_pk(Vd + (int64_t)(c0 + c) * ld + L0);
#pragma unroll
                for (int c = 0; c < CH; c++)
                    if (c0 + c < dot_cnt)
#pragma unroll
                        for (int k = 0; k < P; k++) d[c0 + c] = fma(vv[c].v[k], wi[k], d[c0 + c]);
            }
        }
        if (want_norm)
#pragma unroll
            for (int k = 0; k < P; k++) d[NV] = fma(wv.v[k], wi[k], d[NV]);
    }
    if (blockIdx.x == 0 && threadIdx.x < n - np * P) {  // the last n mod P points
        const int64_t L = np * P + threadIdx.x;
        T wv = w[L];
        if (sub_cnt > 0) {
            T acc = (T)0;
            for (int i = 0; i < sub_cnt; i++) acc = fma(cs[i], V[(int64_t)i * ld + L], acc);
            wv -= acc;
            w[L] = wv;
        }
        const T wi = wv * inv[mult[L]];
#pragma unroll
        for (int i = 0; i < NV; i++)
            if (i < dot_cnt) d[i] = fma(Vd[(int64_t)i * ld + L], wi, d[i]);
        if (want_norm) d[NV] = fma(wv, wi, d[NV]);
    }
    gm_grid_sum<T, NV + 1>(d, partials, counter, [&](const double* a) {
        for (int i = 0; i < dot_cnt; i++) dot_out[i] = a[i];
        if (want_norm) *norm_out = a[NV];
    });
}

// x += sum_{i < k} y_i Z_i  (Z_i at Z + i ld; the combination in T, chunks of
// eight basis loads in flight, the addition in FP64)
template <typename T>
__global__ void __launch_bounds__(256) gm_update_kernel(double* __restrict__ x, const T* __restrict__ Z, int64_t ld,
                                                        const double* __restrict__ y, int k, int64_t n) {
    constexpr int P = 16 / sizeof(T), CH = 8;
    __shared__ T ys[kGmMaxRestart];
    for (int q = threadIdx.x; q < k; q += blockDim.x) ys[q] = (T)y[q];
    __syncthreads();
    const int64_t np = n / P;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t L0 = q * P;
        T acc[P];
#pragma unroll
        for (int j = 0; j < P; j++) acc[j] = (T)0;
        for (int i0 = 0; i0 < k; i0 += CH) {
            Pk<T> vv[CH];
#pragma unroll
            for (int c = 0; c < CH; c++)
                if (i0 + c < k) vv[c] = ld_pk(Z + (int64_t)(i0 + c) * ld + L0);
#pragma unroll
            for (int c = 0; c < CH; c++)
                if (i0 + c < k)
#pragma unroll
                    for (int j = 0; j < P; j++) acc[j] = fma(ys[i0 + c], vv[c].v[j], acc[j]);
        }
#pragma unroll
        for (int j = 0; j < P; j++) x[L0 + j] += (double)acc[j];
    }
    if (blockIdx.x == 0 && threadIdx.x < n - np * P) {
        const int64_t L = np * P + threadIdx.x;
        T acc = (T)0;
        for (int i = 0; i < k; i++) acc = fma(ys[i], Z[(int64_t)i * ld + L], acc);
        x[L] += (double)acc;
    }
}

// One Gram-Schmidt pass (see gm_pass_kernel) over the basis V (vector i at
// V + i ld, ld a multiple of 16 bytes), dots split into launches of kGmNV;
// partials: (kGmNV + 1) kMaxPartials doubles, counter zero between launches.
template <typename T>
inline int krylov_pass(sem_handle* h, T* w, const T* V, int64_t ld, int sub_cnt, const double* sub_coef, int dot_cnt,
                       double* dot_out, double* norm_out, double* partials, unsigned int* counter, cudaStream_t s) {
    const int64_t n = h->n_local;
    static int per_sm = 0;  // resident CTAs per SM: the grid is one full wave
    if (per_sm == 0) {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, gm_pass_kernel<T, kGmNV>, 256, 0);
        per_sm = nb > 0 ? nb : 1;
    }
    const int64_t packs = n / (16 / (int64_t)sizeof(T));
    int64_t grid = (packs + 255) / 256;
    grid = grid < (int64_t)h->sm_count * per_sm ? grid : (int64_t)h->sm_count * per_sm;
    grid = grid < kMaxPartials ? (grid > 0 ? grid : 1) : kMaxPartials;
    int lo = 0;
    do {
        const int cnt = dot_cnt - lo < kGmNV ? dot_cnt - lo : kGmNV;
        const bool last = lo + kGmNV >= dot_cnt;
        gm_pass_kernel<T, kGmNV><<<(int)grid, 256, 0, s>>>(w, V, ld, n, lo == 0 ? sub_cnt : 0, sub_coef, lo,
                                                           cnt > 0 ? cnt : 0, (last && norm_out) ? 1 : 0, h->mult,
                                                           dot_out ? dot_out + lo : nullptr, norm_out, partials,
                                                           counter);
        SEM_LAUNCH_CHECK("gm_pass_kernel");
        h->launches++;
        lo += kGmNV;
    } while (lo < dot_cnt);
    return SEM_OK;
}

// x += sum_{i < k} y_i Z_i  (y on the device)
template <typename T>
inline int krylov_update(sem_handle* h, double* x, const T* Z, int64_t ld, const double* y, int k, cudaStream_t s) {
    if (k <= 0) return SEM_OK;
    gm_update_kernel<T><<<grid_for(h, h->n_local, 256, 8), 256, 0, s>>>(x, Z, ld, y, k, h->n_local);
    SEM_LAUNCH_CHECK("gm_update_kernel");
    h->launches++;
    return SEM_OK;
}

}  // namespace sem
