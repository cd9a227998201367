// The paper's pressure solver (Sec. II-B): restarted GMRES with a
// preconditioner built from an overlapping additive Schwarz method and a
// coarse-grid solve of 10 P-CG iterations (after Lottes and Fischer 2005).
// The paper gives no further detail; this is the reading implemented:
//
//   M^-1 r = mask (Minv r  on every node (point Jacobi),
//                  replaced on each element's interior nodes by the fast-
//                  diagonalisation solve of the element approximated by a box
//                  (mean edge lengths L_r, L_s, L_t, mean h1), homogeneous
//                  Dirichlet on the element boundary:
//                    (S_t x S_s x S_r) diag(1 / (lam_i + lam_j + lam_k)) (S_t x S_s x S_r)^T
//                  with K S = W S Lambda, S^T W S = I of the reference interior
//                  stiffness and mass, scaled by sqrt(2 / L) and 4 / L^2,
//                + P A_c^-1 R r  (the same elements with N = 1 on their corners:
//                  R r = QQ_c^T sum_L P^T r / mult, P the trilinear weights,
//                  A_c^-1 by 10 Jacobi-PCG iterations from zero))
//
// and flexible GMRES (the coarse CG makes the preconditioner change with its
// argument): Arnoldi in the unique-node inner product with classical
// Gram-Schmidt run twice, Givens rotations on the host, x = x0 + Z y at the end
// of every restart cycle, the true FP64 residual checked at every restart.
//
// Two forms share the code, templated on the type T of the Krylov vectors:
//  * FP64 (T = double): operator SEM_FP64 (native) or SEM_FP64_PAIR, Schwarz
//    arithmetic in FP64 or, with precond_precision = SEM_FP32, in FP32 (the
//    preconditioner of a flexible method may be any map: only its output z_j
//    enters the Arnoldi relation A Z = V H, through the FP64 operator).
//  * mixed (T = float, precision = SEM_FP32): every restart cycle is an FP32
//    FGMRES solve of A d = r for the true FP64 residual r, and x += d in FP64:
//    restarted GMRES as iterative refinement (the GMRES-IR scheme of Carson and
//    Higham 2017, with a flexible preconditioner), as the CG refinement of this
//    library does around its FP32 inner CG.
//
// GB300 has 1/64 of the FP32 rate in FP64, so the FP64 form is bound by FP64
// arithmetic in the operator, the preconditioner and the Gram-Schmidt sums;
// the mixed form moves all of that to the FP32 pipe and halves the bytes.
//
// Per Arnoldi step: one fused Schwarz kernel (Jacobi, restriction, interior
// solves), the coarse gather-scatter and CG, one prolongation kernel, the
// operator and its gather-scatter, three Gram-Schmidt passes (dots; subtract
// and dots; subtract and norm), one scaling kernel, and ONE host read of the
// coefficients for the Givens rotations.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

constexpr int kGmNV = 16;           // dot products per Gram-Schmidt launch
constexpr int kGmMaxRestart = 200;  // largest restart length
constexpr int kCoefStride = kGmMaxRestart + 2;

// v0 = T(r * f)
template <typename T>
__global__ void gm_start_kernel(T* __restrict__ v0, const double* __restrict__ r, double f, int64_t n) {
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x)
        v0[L] = (T)(r[L] * f);
}

// out = in / sqrt(*norm2)  (zero when the norm vanished: the host then stops)
template <typename T>
__global__ void gm_scale_kernel(T* __restrict__ out, const T* __restrict__ in, const double* __restrict__ norm2,
                                int64_t n) {
    __shared__ T f;
    if (threadIdx.x == 0) {
        const double q = *norm2;
        f = q > 0.0 ? (T)(1.0 / sqrt(q)) : (T)0;
    }
    __syncthreads();
    const T fs = f;
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x)
        out[L] = in[L] * fs;
}

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
// block and grid sums in FP64 in a fixed order (last block to arrive); fin
// receives the K sums in thread 0 of that block.
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
    if (threadIdx.x < K) {
        const double* pq = partials + threadIdx.x * kMaxPartials;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int q = 0;
        for (; q + 4 <= (int)gridDim.x; q += 4) {
            s0 += __ldcg(pq + q);
            s1 += __ldcg(pq + q + 1);
            s2 += __ldcg(pq + q + 2);
            s3 += __ldcg(pq + q + 3);
        }
        for (; q < (int)gridDim.x; q++) s0 += __ldcg(pq + q);
        tot[threadIdx.x] = (s0 + s1) + (s2 + s3);
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

// The local part of the Schwarz preconditioner, one CTA per element at a time:
// z = Minv r on the element's boundary nodes, the coarse right-hand side
// rc[e][c] = sum_q Pw[q][c] r_q / mult_q, and the fast-diagonalisation solve on
// the (lx-2)^3 interior nodes (three contractions with S^T, the diagonal,
// three with S, in shared memory).  Data of type TI, arithmetic in TC.
template <int LX, typename TI, typename TC>
__global__ void __launch_bounds__(256) schwarz_local_kernel(const TI* __restrict__ r, TI* __restrict__ z,
                                                            const TI* __restrict__ minv,
                                                            const uint8_t* __restrict__ mult,
                                                            const TC* __restrict__ Pw, const TC* __restrict__ Sg,
                                                            const TC* __restrict__ lamg, const TC* __restrict__ fac,
                                                            double* __restrict__ rc, int64_t E) {
    constexpr int NI = LX - 2, N3 = LX * LX * LX;
    constexpr int M3 = NI > 0 ? NI * NI * NI : 1, S2 = NI > 0 ? NI * NI : 1, S1 = NI > 0 ? NI : 1;
    __shared__ TC a[M3], b[M3], S[S2], lam[S1], inv[256];
    __shared__ TC red[8][8];
    __shared__ TC F[2][LX];  // 1-D corner weights (1 -/+ xi) / 2: Pw[q][c] = F[c&1][i] F[c>>1&1][j] F[c>>2][k]
    for (int t = threadIdx.x; t < 256; t += blockDim.x) inv[t] = t ? (TC)1 / (TC)t : (TC)0;
    for (int t = threadIdx.x; t < 2 * LX; t += blockDim.x) F[t / LX][t % LX] = Pw[(t % LX) * 8 + t / LX];
    if constexpr (NI > 0) {
        for (int t = threadIdx.x; t < NI * NI; t += blockDim.x) S[t] = Sg[t];
        for (int t = threadIdx.x; t < NI; t += blockDim.x) lam[t] = lamg[t];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        const TI* re = r + e * N3;
        TI* ze = z + e * N3;
        TC acc[8];
#pragma unroll
        for (int c = 0; c < 8; c++) acc[c] = (TC)0;
        for (int t = threadIdx.x; t < N3; t += blockDim.x) {
            const TC v = (TC)re[t];
            const int i = t % LX, j = (t / LX) % LX, k = t / (LX * LX);
            const bool interior = i > 0 && i < LX - 1 && j > 0 && j < LX - 1 && k > 0 && k < LX - 1;
            if (interior) {
                if constexpr (NI > 0) a[((k - 1) * NI + (j - 1)) * NI + (i - 1)] = v;
            } else {
                ze[t] = (TI)((TC)minv[e * N3 + t] * v);
            }
            const TC vm = v * inv[mult[e * N3 + t]];
            const TC a0 = F[0][i] * vm, a1 = F[1][i] * vm;
            const TC bj[4] = {a0 * F[0][j], a1 * F[0][j], a0 * F[1][j], a1 * F[1][j]};
#pragma unroll
            for (int c = 0; c < 4; c++) {
                acc[c] = fma(bj[c], F[0][k], acc[c]);
                acc[c + 4] = fma(bj[c], F[1][k], acc[c + 4]);
            }
        }
#pragma unroll
        for (int c = 0; c < 8; c++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], o);
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < 8; c++) red[wid][c] = acc[c];
        __syncthreads();
        if (threadIdx.x < 8) {
            double sum = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); q++) sum += (double)red[q][threadIdx.x];
            rc[e * 8 + threadIdx.x] = sum;
        }
        if constexpr (NI > 0) {
            // sqrt(2 / L_d) and h1m 4 / L_d^2, precomputed per element at set-up
            const TC* fe = fac + e * 6;
            const TC sr = fe[0], ss = fe[1], st = fe[2], cr = fe[3], cs = fe[4], ct = fe[5];
            auto ijk = [](int t, int& i, int& j, int& k) {
                i = t % NI;
                j = (t / NI) % NI;
                k = t / (NI * NI);
            };
            for (int t = threadIdx.x; t < M3; t += blockDim.x) {  // along i: b[k][j][m] = sr sum_i S[i][m] a[k][j][i]
                int m, j, k;
                ijk(t, m, j, k);
                TC s = (TC)0;
#pragma unroll
                for (int i = 0; i < NI; i++) s = fma(S[i * NI + m], a[(k * NI + j) * NI + i], s);
                b[t] = sr * s;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < M3; t += blockDim.x) {  // along j
                int i, m, k;
                ijk(t, i, m, k);
                TC s = (TC)0;
#pragma unroll
                for (int j = 0; j < NI; j++) s = fma(S[j * NI + m], b[(k * NI + j) * NI + i], s);
                a[t] = ss * s;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < M3; t += blockDim.x) {  // along k, then the diagonal
                int i, j, m;
                ijk(t, i, j, m);
                TC s = (TC)0;
#pragma unroll
                for (int k = 0; k < NI; k++) s = fma(S[k * NI + m], a[(k * NI + j) * NI + i], s);
                b[t] = st * s / (lam[i] * cr + lam[j] * cs + lam[m] * ct);
            }
            __syncthreads();
            for (int t = threadIdx.x; t < M3; t += blockDim.x) {  // back along k
                int i, j, k;
                ijk(t, i, j, k);
                TC s = (TC)0;
#pragma unroll
                for (int m = 0; m < NI; m++) s = fma(S[k * NI + m], b[(m * NI + j) * NI + i], s);
                a[t] = st * s;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < M3; t += blockDim.x) {  // back along j
                int i, j, k;
                ijk(t, i, j, k);
                TC s = (TC)0;
#pragma unroll
                for (int m = 0; m < NI; m++) s = fma(S[j * NI + m], a[(k * NI + m) * NI + i], s);
                b[t] = ss * s;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < M3; t += blockDim.x) {  // back along i, out
                int i, j, k;
                ijk(t, i, j, k);
                TC s = (TC)0;
#pragma unroll
                for (int m = 0; m < NI; m++) s = fma(S[i * NI + m], b[(k * NI + j) * NI + m], s);
                ze[((k + 1) * LX + (j + 1)) * LX + (i + 1)] = (TI)(sr * s);
            }
        }
        __syncthreads();  // a, b and red are reused by the next element
    }
}

// z = mask (z + sum_c Pw[q][c] xc[e][c]), one CTA per element at a time
template <int LX, typename TI, typename TC>
__global__ void __launch_bounds__(256) prolong_kernel(TI* __restrict__ z, const double* __restrict__ xc,
                                                      const TC* __restrict__ Pw, const uint8_t* __restrict__ mask,
                                                      int64_t E) {
    constexpr int N3 = LX * LX * LX;
    __shared__ TC xs[8];
    __shared__ TC F[2][LX];  // 1-D corner weights, as in schwarz_local_kernel
    for (int t = threadIdx.x; t < 2 * LX; t += blockDim.x) F[t / LX][t % LX] = Pw[(t % LX) * 8 + t / LX];
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        if (threadIdx.x < 8) xs[threadIdx.x] = (TC)xc[e * 8 + threadIdx.x];  // 8 conversions per element
        __syncthreads();
        TC c8[8];
#pragma unroll
        for (int c = 0; c < 8; c++) c8[c] = xs[c];
        for (int t = threadIdx.x; t < N3; t += blockDim.x) {
            const int i = t % LX, j = (t / LX) % LX, k = t / (LX * LX);
            TC y[4];  // along k, then j, then i: corr = sum_c F[c&1][i] F[c>>1&1][j] F[c>>2][k] x_c
#pragma unroll
            for (int c = 0; c < 4; c++) y[c] = fma(F[0][k], c8[c], F[1][k] * c8[c + 4]);
            const TC y0 = fma(F[0][j], y[0], F[1][j] * y[2]), y1 = fma(F[0][j], y[1], F[1][j] * y[3]);
            const TC corr = fma(F[0][i], y0, F[1][i] * y1);
            const int64_t L = e * N3 + t;
            z[L] = mask[L] ? (TI)(z[L] + (TI)corr) : (TI)0;
        }
        __syncthreads();  // xs is rewritten for the next element
    }
}

template <typename TC>
static const TC* sch_table(const SchwarzData& sc, int which) {  // 0 Pw, 1 S, 2 lam, 3 fac
    if constexpr (std::is_same<TC, double>::value)
        return which == 0 ? sc.Pw : which == 1 ? sc.S : which == 2 ? sc.lam : sc.fac;
    else
        return which == 0 ? sc.Pw32 : which == 1 ? sc.S32 : which == 2 ? sc.lam32 : sc.fac32;
}

template <int LX, typename TI, typename TC>
static int launch_local_t(sem_handle* h, const TI* r, TI* z, const TI* minv, cudaStream_t s) {
    const SchwarzData& sc = h->sch;
    const int64_t E = h->parts[0].E;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(E, (int64_t)h->sm_count * 8));
    schwarz_local_kernel<LX, TI, TC><<<grid, 256, 0, s>>>(r, z, minv, h->mult, sch_table<TC>(sc, 0),
                                                          sch_table<TC>(sc, 1), sch_table<TC>(sc, 2),
                                                          sch_table<TC>(sc, 3), sc.coarse->ws.b, E);
    SEM_LAUNCH_CHECK("schwarz_local_kernel");
    h->launches++;
    return SEM_OK;
}

template <int LX, typename TI, typename TC>
static int launch_prolong_t(sem_handle* h, TI* z, cudaStream_t s) {
    const SchwarzData& sc = h->sch;
    const int64_t E = h->parts[0].E;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(E, (int64_t)h->sm_count * 8));
    prolong_kernel<LX, TI, TC><<<grid, 256, 0, s>>>(z, sc.coarse->ws.x, sch_table<TC>(sc, 0), h->mask, E);
    SEM_LAUNCH_CHECK("prolong_kernel");
    h->launches++;
    return SEM_OK;
}

// phase 0: local part (and the coarse right-hand side), phase 1: prolongation
template <typename TI, typename TC>
static int launch_schwarz_phase(sem_handle* h, int phase, const TI* r, TI* z, const TI* minv, cudaStream_t s) {
#define SEM_SCH_CASE(LXV)                                                                   \
    case LXV:                                                                                \
        return phase == 0 ? launch_local_t<LXV, TI, TC>(h, r, z, minv, s)                  \
                          : launch_prolong_t<LXV, TI, TC>(h, z, s);
    switch (h->parts[0].lx) {
        SEM_SCH_CASE(2)
        SEM_SCH_CASE(3)
        SEM_SCH_CASE(4)
        SEM_SCH_CASE(5)
        SEM_SCH_CASE(6)
        SEM_SCH_CASE(7)
        SEM_SCH_CASE(8)
        SEM_SCH_CASE(9)
        SEM_SCH_CASE(10)
        SEM_SCH_CASE(11)
        SEM_SCH_CASE(12)
        default: return fail(SEM_EINVAL, "the Schwarz preconditioner covers lx <= 12");
    }
#undef SEM_SCH_CASE
}

// z = M^-1 r (two-level additive Schwarz; see the top of this file); data TI,
// local arithmetic TC, the coarse CG in FP64
template <typename TI, typename TC>
static int apply_schwarz(sem_handle* h, const TI* r, TI* z, bool persist, cudaStream_t s) {
    sem_handle* hc = h->sch.coarse;
    const TI* minv;
    if constexpr (std::is_same<TI, double>::value)
        minv = h->minv64;
    else
        minv = h->minv32;
    int rc = launch_schwarz_phase<TI, TC>(h, 0, r, z, minv, s);
    if (!rc) rc = launch_gs(hc, hc->ws.b, false, true, s);
    if (!rc) rc = coarse_pcg(hc, 10, persist, s);
    if (!rc) rc = launch_schwarz_phase<TI, TC>(h, 1, r, z, minv, s);
    return rc;
}

void free_schwarz(sem_handle* h) {
    SchwarzData& sc = h->sch;
    if (sc.coarse) sem_destroy(sc.coarse);
    cudaFree(sc.fac);
    cudaFree(sc.fac32);
    cudaFree(sc.S);
    cudaFree(sc.lam);
    cudaFree(sc.Pw);
    cudaFree(sc.S32);
    cudaFree(sc.lam32);
    cudaFree(sc.Pw32);
    cudaFree(sc.V);
    cudaFree(sc.Z);
    cudaFree(sc.coef);
    cudaFree(sc.gpart);
    cudaFree(sc.gcount);
    sc = SchwarzData{};
}

// Krylov storage for restart length m and vectors of `elem` bytes: V (m + 1
// vectors), Z (m vectors), the coefficients and the Gram-Schmidt partials
static int ensure_krylov(sem_handle* h, int m, int elem) {
    SchwarzData& sc = h->sch;
    if (!sc.coef) {
        int rc = dalloc(h, &sc.coef, (size_t)kCoefStride * 4);
        if (!rc) rc = dalloc(h, &sc.gpart, (size_t)(kGmNV + 1) * kMaxPartials);
        if (rc) return rc;
        SEM_CUDA_TRY(cudaMalloc(&sc.gcount, sizeof(unsigned int)));
        SEM_CUDA_TRY(cudaMemset(sc.gcount, 0, sizeof(unsigned int)));
    }
    if (sc.m == m && sc.elem == elem && sc.V) return SEM_OK;
    // leading dimension: a multiple of 4 points, so every vector starts on 16 bytes
    const size_t n = (size_t)((h->n_local + 3) & ~(int64_t)3);
    if (sc.V) {
        h->device_bytes -= (size_t)sc.elem * (size_t)(2 * sc.m + 1) * n;
        cudaFree(sc.V);
        cudaFree(sc.Z);
        sc.V = sc.Z = nullptr;
        sc.m = 0;
    }
    const size_t bv = (size_t)elem * (size_t)(m + 1) * n, bz = (size_t)elem * (size_t)m * n;
    if (cudaMalloc(&sc.V, bv) != cudaSuccess || cudaMalloc(&sc.Z, bz) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(sc.V);
        cudaFree(sc.Z);
        sc.V = sc.Z = nullptr;
        return fail(SEM_ENOMEM, "cudaMalloc of the GMRES Krylov basis failed");
    }
    h->device_bytes += bv + bz;
    sc.m = m;
    sc.elem = elem;
    sc.ld = (int64_t)n;
    return SEM_OK;
}

static int read_scalars(double* dst, const double* src, int count, cudaStream_t s) {
    SEM_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
    SEM_CUDA_TRY(cudaStreamSynchronize(s));
    return SEM_OK;
}

// One Gram-Schmidt pass, dots split into launches of kGmNV
template <typename T>
static int gs_pass(sem_handle* h, T* w, int sub_cnt, const double* sub_coef, int dot_cnt, double* dot_out,
                   double* norm_out, cudaStream_t s) {
    SchwarzData& sc = h->sch;
    const T* V = static_cast<const T*>(sc.V);
    const int64_t n = h->n_local;
    static int per_sm = 0;  // resident CTAs per SM: the grid is one full wave
    if (per_sm == 0) {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, gm_pass_kernel<T, kGmNV>, 256, 0);
        per_sm = std::max(nb, 1);
    }
    const int64_t packs = n / (16 / (int64_t)sizeof(T));
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>({(packs + 255) / 256, (int64_t)h->sm_count * per_sm, (int64_t)kMaxPartials}));
    int lo = 0;
    do {
        const int cnt = std::min(kGmNV, dot_cnt - lo);
        const bool last = lo + kGmNV >= dot_cnt;
        gm_pass_kernel<T, kGmNV><<<grid, 256, 0, s>>>(w, V, sc.ld, n, lo == 0 ? sub_cnt : 0, sub_coef, lo,
                                                      std::max(cnt, 0),
                                                      (last && norm_out) ? 1 : 0, h->mult, dot_out + lo, norm_out,
                                                      sc.gpart, sc.gcount);
        SEM_LAUNCH_CHECK("gm_pass_kernel");
        h->launches++;
        lo += kGmNV;
    } while (lo < dot_cnt);
    return SEM_OK;
}

// w = mask QQ^T A_L z with the operator of the solve's precision
template <typename T>
static int apply_operator(sem_handle* h, const T* z, T* w, int op_prec, cudaStream_t s) {
    int rc = launch_ax_local(h, z, w, std::is_same<T, float>::value ? SEM_FP32 : op_prec, s);
    return rc ? rc : launch_gs(h, w, std::is_same<T, float>::value, true, s);
}

// A staged operator kernel (fine handle) or the persistent coarse CG (coarse
// handle) that gave up a bounded wait set its handle's error word and returned:
// the solve ends with SEM_ETIMEOUT, the context intact.
static int check_error_words(sem_handle* h, cudaStream_t s) {
    for (sem_handle* q : {h, h->sch.coarse}) {
        int word = 0;
        SEM_CUDA_TRY(cudaMemcpyAsync(&word, device_error_word(q), sizeof(int), cudaMemcpyDeviceToHost, s));
        SEM_CUDA_TRY(cudaStreamSynchronize(s));
        if (word) {
            cudaMemset(device_error_word(q), 0, sizeof(int));
            cudaMemset(q->counters, 0, 16 * sizeof(unsigned));
            return fail(SEM_ETIMEOUT, "a bounded device-side wait of the GMRES solve expired");
        }
    }
    return SEM_OK;
}

template <typename T>
static int solve_gmres_t(sem_handle* h, const sem_solve_opts& o, sem_solve_stats* st, cudaStream_t s) {
    constexpr bool kMixed = std::is_same<T, float>::value;
    SchwarzData& sc = h->sch;
    const int m = o.gmres_restart;
    const int64_t n = h->n_local;
    const int grid = grid_for(h, n, 256, 8);
    const bool pc32 = kMixed || o.precond_precision == SEM_FP32;
    const int op_prec = o.precision;  // FP64 form: SEM_FP64, SEM_FP64_NATIVE or SEM_FP64_PAIR
    const bool persist = o.persistent != 0;  // the coarse CG as one cooperative launch
    T* w;
    if constexpr (kMixed)
        w = h->ws.w32;
    else
        w = h->ws.w;
    T* Vb = static_cast<T*>(sc.V);
    T* Zb = static_cast<T*>(sc.Z);
    double* c1 = sc.coef;
    double* c2 = sc.coef + kCoefStride;
    double* nrm = sc.coef + 2 * kCoefStride;
    double* yd = sc.coef + 3 * kCoefStride;
    double* rrbb = h->scratch;
    std::vector<double> H((size_t)(m + 1) * m), g(m + 1), cs(m), sn(m), hcol(m + 2), y(m),
        hc(2 * kCoefStride + 1);
    double hb[2] = {0.0, 0.0};
    double rel_prev = INFINITY;
    int status = SEM_ENOTCONV, it = 0, cycles = 0, rc;
    for (;;) {
        if ((rc = true_residual(h, h->ws.x, h->ws.b, rrbb, s)) || (rc = read_scalars(hb, rrbb, 2, s)) ||
            (rc = check_error_words(h, s)))
            return rc;
        const double rel = relative_residual(hb[0], hb[1]);
        if (cycles == 0) st->relres_start = rel;
        if (!std::isfinite(rel)) {
            status = SEM_EBREAKDOWN;
            break;
        }
        if (hb[1] == 0.0 || rel <= o.tol) {
            status = SEM_OK;
            break;
        }
        if (it >= o.max_iter) break;
        if (kMixed && cycles >= o.max_outer) break;
        if (kMixed && cycles > 0 && !(rel < rel_prev)) {  // a refinement cycle that gained nothing
            status = SEM_ESTAGNATE;
            break;
        }
        rel_prev = rel;
        const double bn = std::sqrt(hb[1]), beta = std::sqrt(hb[0]);
        // stop the cycle at the target (FP64), or at inner_tol of its start (mixed)
        const double stop = kMixed ? std::max(o.inner_tol * beta, 0.3 * o.tol * bn) : o.tol * bn;
        gm_start_kernel<T><<<grid, 256, 0, s>>>(Vb, h->ws.r, 1.0 / beta, n);
        SEM_LAUNCH_CHECK("gm_start_kernel");
        h->launches++;
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m; j++) {
            T* vj = Vb + (int64_t)j * sc.ld;
            T* zj = Zb + (int64_t)j * sc.ld;
            if constexpr (kMixed)
                rc = apply_schwarz<float, float>(h, vj, zj, persist, s);
            else
                rc = pc32 ? apply_schwarz<double, float>(h, vj, zj, persist, s)
                          : apply_schwarz<double, double>(h, vj, zj, persist, s);
            if (rc || (rc = apply_operator<T>(h, zj, w, op_prec, s))) return rc;
            const int c = j + 1;
            // classical Gram-Schmidt twice: c1 = V^T w; w -= V c1, c2 = V^T w; w -= V c2, ||w||^2
            if ((rc = gs_pass<T>(h, w, 0, nullptr, c, c1, nullptr, s)) ||
                (rc = gs_pass<T>(h, w, c, c1, c, c2, nullptr, s)) ||
                (rc = gs_pass<T>(h, w, c, c2, 0, nullptr, nrm, s)))
                return rc;
            gm_scale_kernel<T><<<grid, 256, 0, s>>>(Vb + (int64_t)c * sc.ld, w, nrm, n);
            SEM_LAUNCH_CHECK("gm_scale_kernel");
            h->launches++;
            if ((rc = read_scalars(hc.data(), sc.coef, 2 * kCoefStride + 1, s))) return rc;
            for (int i = 0; i < c; i++) hcol[i] = hc[i] + hc[kCoefStride + i];
            const double ww = hc[2 * kCoefStride];
            hcol[c] = std::sqrt(std::max(ww, 0.0));
            for (int i = 0; i < j; i++) {  // earlier rotations
                const double t = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
                hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
                hcol[i] = t;
            }
            const double den = std::hypot(hcol[j], hcol[c]);
            if (!(den > 0.0) || !std::isfinite(den)) {
                status = SEM_EBREAKDOWN;
                break;
            }
            cs[j] = hcol[j] / den;
            sn[j] = hcol[c] / den;
            hcol[j] = den;
            g[c] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            for (int i = 0; i <= j; i++) H[(size_t)i * m + j] = hcol[i];
            it++;
            k = c;
            if (std::fabs(g[c]) <= stop || it >= o.max_iter || !(ww > 0.0)) break;
        }
        if (status == SEM_EBREAKDOWN) break;
        for (int i = k - 1; i >= 0; i--) {  // H y = g, upper triangular
            double t = g[i];
            for (int q = i + 1; q < k; q++) t -= H[(size_t)i * m + q] * y[q];
            y[i] = t / H[(size_t)i * m + i];
        }
        SEM_CUDA_TRY(cudaMemcpyAsync(yd, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
        gm_update_kernel<T><<<grid, 256, 0, s>>>(h->ws.x, Zb, sc.ld, yd, k, n);
        SEM_LAUNCH_CHECK("gm_update_kernel");
        h->launches++;
        cycles++;
    }
    st->status = status;
    st->iterations = it;
    st->outer_iterations = cycles;
    st->relres = relative_residual(hb[0], hb[1]);
    st->relres_recursive = st->relres;
    return SEM_OK;
}

int solve_gmres(sem_handle* h, double* x_user, const double* b_user, const sem_solve_opts& o,
                sem_solve_stats* stats, cudaStream_t s) {
    if (h->nsolve != 1 || !h->sch.coarse)
        return fail(SEM_EINVAL, "SEM_MODE_GMRES needs a single-mesh handle set up with SEM_FLAG_SCHWARZ");
    const int m = o.gmres_restart;
    if (m < 1 || m > kGmMaxRestart) return fail(SEM_EINVAL, "gmres_restart must be in [1, 200]");
    const bool mixed = o.precision == SEM_FP32;
    if (!mixed && o.precision != SEM_FP64 && o.precision != SEM_FP64_NATIVE && o.precision != SEM_FP64_PAIR)
        return fail(SEM_EINVAL, "GMRES mode takes SEM_FP64, SEM_FP64_NATIVE, SEM_FP64_PAIR or SEM_FP32");
    if (o.precond_precision != SEM_FP64 && o.precond_precision != SEM_FP32)
        return fail(SEM_EINVAL, "precond_precision must be SEM_FP64 or SEM_FP32");
    if (mixed && !(o.inner_tol > 0.0 && o.inner_tol < 1.0)) return fail(SEM_EINVAL, "inner_tol must be in (0, 1)");
    int rc = ensure_workspace(h, mixed);
    if (!rc) rc = ensure_workspace(h->sch.coarse, false);
    if (!rc) rc = ensure_krylov(h, m, mixed ? (int)sizeof(float) : (int)sizeof(double));
    if (!rc && o.autotune) {
        rc = autotune_ax(h, false, s);
        if (!rc && mixed) rc = autotune_ax(h, true, s);
    }
    if (rc) return rc;
    SchwarzData& sc = h->sch;
    const size_t bytes = sizeof(double) * h->n_local;
    const bool xh = host_resident(x_user), bh = host_resident(b_user);
    const int64_t launches0 = h->launches + sc.coarse->launches;
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, s);
    SEM_CUDA_TRY(cudaMemcpyAsync(h->ws.x, x_user, bytes, xh ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    SEM_CUDA_TRY(cudaMemcpyAsync(h->ws.b, b_user, bytes, bh ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    sem_solve_stats st = {};
    rc = mixed ? solve_gmres_t<float>(h, o, &st, s) : solve_gmres_t<double>(h, o, &st, s);
    if (rc) {
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        return rc;
    }
    SEM_CUDA_TRY(cudaMemcpyAsync(x_user, h->ws.x, bytes, xh ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    cudaEventRecord(ev1, s);
    SEM_CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    st.time_ms = ms;
    st.kernel_launches = h->launches + sc.coarse->launches - launches0;
    st.ax_variant = mixed ? ax_variant_for(h, h->parts[0].lx, kClsF32)
                          : ax_variant_of_precision(h, h->parts[0].lx, o.precision);
    st.launches_per_iteration = -1;  // varies with the Arnoldi step
    if (stats) *stats = st;
    const int status = st.status;
    if (status != SEM_OK)
        set_error(status == SEM_ENOTCONV     ? "GMRES did not converge within max_iter / max_outer"
                  : status == SEM_ESTAGNATE ? "a GMRES refinement cycle did not reduce the FP64 residual"
                                             : "GMRES breakdown");
    return status;
}

}  // namespace sem

using namespace sem;

extern "C" {

SEM_API int sem_schwarz_apply(sem_handle* h, const double* r, double* z, cudaStream_t s) {
    if (!h || !r || !z) return fail(SEM_EINVAL, "null argument");
    if (r == z) return fail(SEM_EINVAL, "z must not alias r");
    if (h->nsolve != 1 || !h->sch.coarse) return fail(SEM_EINVAL, "the handle has no Schwarz preconditioner");
    int rc = ensure_workspace(h->sch.coarse, false);
    return rc ? rc : apply_schwarz<double, double>(h, r, z, false, s);
}

SEM_API int sem_schwarz_apply32(sem_handle* h, const float* r, float* z, cudaStream_t s) {
    if (!h || !r || !z) return fail(SEM_EINVAL, "null argument");
    if (r == z) return fail(SEM_EINVAL, "z must not alias r");
    if (h->nsolve != 1 || !h->sch.coarse) return fail(SEM_EINVAL, "the handle has no Schwarz preconditioner");
    int rc = ensure_workspace(h->sch.coarse, false);
    return rc ? rc : apply_schwarz<float, float>(h, r, z, false, s);
}

}  // extern "C"
