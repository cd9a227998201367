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
// Gram-Schmidt twice, the second pass lagged one step (or both in the step, or
// once: opts.gmres_orth), Givens rotations on the host, x = x0 + Z y at the end
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
// Per Arnoldi step (default form): the restriction, the coarse CG on the
// assembled coarse matrix (a second stream, in the precision of the data)
// beside the local solves (Jacobi and interior solves; one warp per element),
// one prolongation kernel, the operator and its gather-scatter, two passes
// over the basis (dots; one combined update), and ONE host read of the
// coefficients for the Givens rotations.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "sem_krylov.cuh"

namespace sem {

constexpr int kCoefStride = kGmMaxRestart + 2;
// device scalars of a cycle: regions of kCoefStride doubles in SchwarzData::coef
enum GmRegion { kRegA = 0, kRegB = 1, kRegNorm = 2, kRegY = 3, kRegSc = 4, kRegTc = 5, kRegions = 6 };

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

// Dot products of basis vectors X_lo .. X_{lo+cnt-1} (cnt <= NV) with two
// vectors u and w in one sweep: a_i = <X_{lo+i}, u>, b_i = <X_{lo+i}, w>
// (unique-node inner product; 16-byte packs, four basis loads in flight per
// chunk)
template <typename T, int NV>
__global__ void __launch_bounds__(256) gm_dots2_kernel(const T* __restrict__ X, int64_t ld, int64_t n, int lo,
                                                       int cnt, const T* __restrict__ u, const T* __restrict__ w,
                                                       const uint8_t* __restrict__ mult, double* __restrict__ a_out,
                                                       double* __restrict__ b_out, double* partials,
                                                       unsigned int* counter) {
    constexpr int P = 16 / sizeof(T), CH = 4;
    __shared__ T inv[256];
    for (int q = threadIdx.x; q < 256; q += blockDim.x) inv[q] = q ? (T)1 / (T)q : (T)0;
    __syncthreads();
    T d[2 * NV];
#pragma unroll
    for (int q = 0; q < 2 * NV; q++) d[q] = (T)0;
    const T* Xl = X + (int64_t)lo * ld;
    const int64_t np = n / P;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t L0 = q * P;
        const Pk<T> uv = ld_pk(u + L0), wv = ld_pk(w + L0);
        uint8_t mu[P];
        ld_mult<P>(mult + L0, mu);
        T ui[P], wi[P];
#pragma unroll
        for (int k = 0; k < P; k++) {
            ui[k] = uv.v[k] * inv[mu[k]];
            wi[k] = wv.v[k] * inv[mu[k]];
        }
#pragma unroll
        for (int c0 = 0; c0 < NV; c0 += CH) {
            if (c0 < cnt) {
                Pk<T> vv[CH];
#pragma unroll
                for (int c = 0; c < CH; c++)
                    if (c0 + c < cnt) vv[c] = ld_pk(Xl + (int64_t)(c0 + c) * ld + L0);
#pragma unroll
                for (int c = 0; c < CH; c++)
                    if (c0 + c < cnt)
#pragma unroll
                        for (int k = 0; k < P; k++) {
                            d[c0 + c] = fma(vv[c].v[k], ui[k], d[c0 + c]);
                            d[NV + c0 + c] = fma(vv[c].v[k], wi[k], d[NV + c0 + c]);
                        }
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < n - np * P) {  // the last n mod P points
        const int64_t L = np * P + threadIdx.x;
        const T ui = u[L] * inv[mult[L]], wi = w[L] * inv[mult[L]];
#pragma unroll
        for (int i = 0; i < NV; i++)
            if (i < cnt) {
                const T xv = Xl[(int64_t)i * ld + L];
                d[i] = fma(xv, ui, d[i]);
                d[NV + i] = fma(xv, wi, d[NV + i]);
            }
    }
    gm_grid_sum<T, 2 * NV>(d, partials, counter, [&](const double* t) {
        for (int i = 0; i < cnt; i++) {
            a_out[i] = t[i];
            b_out[i] = t[NV + i];
        }
    });
}

// The one update pass of an Arnoldi step with lagged reorthogonalisation
// (vectors X_i = X + i ld, u = X_j the newest basis vector, orthogonalised
// once and not normalised; coefficients from the host):
//   X_j     <- cu u - sum_{i<j} sc_i X_i      (u reorthogonalised and normalised; when rewrite_u)
//   X_{j+1} <- w - cw u - sum_{i<j} tc_i X_i  (w orthogonalised once against X_0..X_j)
//   *norm_out = <X_{j+1}, X_{j+1}>
// with cu = sc[j], cw = tc[j]; each X_i is loaded once for both sums.
template <typename T>
__global__ void __launch_bounds__(256) gm_lagged_update_kernel(T* __restrict__ X, int64_t ld, int64_t n, int j,
                                                               const double* __restrict__ sc,
                                                               const double* __restrict__ tc, int rewrite_u,
                                                               const T* __restrict__ w,
                                                               const uint8_t* __restrict__ mult,
                                                               double* __restrict__ norm_out, double* partials,
                                                               unsigned int* counter) {
    constexpr int P = 16 / sizeof(T), CH = 8;
    __shared__ T inv[256];
    __shared__ T scs[kGmMaxRestart + 1], tcs[kGmMaxRestart + 1];
    for (int q = threadIdx.x; q < 256; q += blockDim.x) inv[q] = q ? (T)1 / (T)q : (T)0;
    for (int q = threadIdx.x; q <= j; q += blockDim.x) {
        scs[q] = (T)sc[q];
        tcs[q] = (T)tc[q];
    }
    __syncthreads();
    const T cu = scs[j], cw = tcs[j];
    T* u = X + (int64_t)j * ld;
    T* out = X + (int64_t)(j + 1) * ld;
    T d[1] = {(T)0};
    const int64_t np = n / P;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t L0 = q * P;
        const Pk<T> uv = ld_pk(u + L0), wv = ld_pk(w + L0);
        T as[P], at[P];
#pragma unroll
        for (int k = 0; k < P; k++) as[k] = at[k] = (T)0;
        for (int i0 = 0; i0 < j; i0 += CH) {
            Pk<T> vv[CH];
#pragma unroll
            for (int c = 0; c < CH; c++)
                if (i0 + c < j) vv[c] = ld_pk(X + (int64_t)(i0 + c) * ld + L0);
#pragma unroll
            for (int c = 0; c < CH; c++)
                if (i0 + c < j)
#pragma unroll
                    for (int k = 0; k < P; k++) {
                        as[k] = fma(scs[i0 + c], vv[c].v[k], as[k]);
                        at[k] = fma(tcs[i0 + c], vv[c].v[k], at[k]);
                    }
        }
        Pk<T> nu, ov;
        uint8_t mu[P];
        ld_mult<P>(mult + L0, mu);
#pragma unroll
        for (int k = 0; k < P; k++) {
            nu.v[k] = fma(cu, uv.v[k], -as[k]);
            ov.v[k] = wv.v[k] - fma(cw, uv.v[k], at[k]);
            d[0] = fma(ov.v[k] * inv[mu[k]], ov.v[k], d[0]);
        }
        if (rewrite_u) *reinterpret_cast<Pk<T>*>(u + L0) = nu;
        *reinterpret_cast<Pk<T>*>(out + L0) = ov;
    }
    if (blockIdx.x == 0 && threadIdx.x < n - np * P) {
        const int64_t L = np * P + threadIdx.x;
        T as = (T)0, at = (T)0;
        for (int i = 0; i < j; i++) {
            const T xv = X[(int64_t)i * ld + L];
            as = fma(scs[i], xv, as);
            at = fma(tcs[i], xv, at);
        }
        const T uv = u[L];
        const T ov = w[L] - fma(cw, uv, at);
        if (rewrite_u) u[L] = fma(cu, uv, -as);
        out[L] = ov;
        d[0] = fma(ov * inv[mult[L]], ov, d[0]);
    }
    gm_grid_sum<T, 1>(d, partials, counter, [&](const double* t) { *norm_out = t[0]; });
}

// What one launch of schwarz_local_kernel does: all of the local part, only
// the coarse restriction, or all but the restriction (the coarse CG then runs
// on a second stream beside the local solves)
enum SchMode { kSchAll = 0, kSchRestrict = 1, kSchLocal = 2 };

// Warps (elements) per CTA of the Schwarz kernels: up to eight, fewer where
// the two interior work arrays of an element would not fit 40 KB per CTA
template <int LX, typename TC>
__host__ __device__ constexpr int sch_warps() {
    constexpr int NI = LX - 2, M3 = NI > 0 ? NI * NI * NI : 1;
    constexpr int w = 40000 / (2 * M3 * (int)sizeof(TC));
    return w < 1 ? 1 : (w > 8 ? 8 : w);
}

// The local part of the Schwarz preconditioner, one WARP per element (its
// contraction passes separated by __syncwarp only): z = Minv r on the
// element's boundary nodes, the coarse right-hand side
// rc[e][c] = sum_q Pw[q][c] r_q / mult_q with the trilinear weights taken as
// products of 1-D factors, and the fast-diagonalisation solve on the (lx-2)^3
// interior nodes (three contractions with S^T, the diagonal, three with S, in
// shared memory).  The input is r / sqrt(*r_norm2) when r_norm2 is given.
// Data of type TI, arithmetic in TC; MODE selects the parts (SchMode).
template <int LX, typename TI, typename TC, int MODE>
__global__ void __launch_bounds__(sch_warps<LX, TC>() * 32)
    schwarz_local_kernel(const TI* __restrict__ r, const double* __restrict__ r_norm2, TI* __restrict__ z,
                         const TI* __restrict__ minv, const uint8_t* __restrict__ mult, const TC* __restrict__ Pw,
                         const TC* __restrict__ Sg, const TC* __restrict__ lamg, const TC* __restrict__ fac,
                         TI* __restrict__ rc, int64_t E) {
    constexpr int NI = LX - 2, N3 = LX * LX * LX, W = sch_warps<LX, TC>();
    constexpr int M3 = NI > 0 ? NI * NI * NI : 1, S2 = NI > 0 ? NI * NI : 1, S1 = NI > 0 ? NI : 1;
    __shared__ TC ab[W][2][M3];
    __shared__ TC S[S2], lam[S1], inv[256];
    __shared__ TC F[2][LX];  // 1-D corner weights (1 -/+ xi) / 2: Pw[q][c] = F[c&1][i] F[c>>1&1][j] F[c>>2][k]
    __shared__ TC rs;
    for (int t = threadIdx.x; t < 256; t += blockDim.x) inv[t] = t ? (TC)1 / (TC)t : (TC)0;
    for (int t = threadIdx.x; t < 2 * LX; t += blockDim.x) F[t / LX][t % LX] = Pw[(t % LX) * 8 + t / LX];
    if (threadIdx.x == 0) {
        const double q = r_norm2 ? *r_norm2 : 1.0;
        rs = q > 0.0 ? (TC)(1.0 / sqrt(q)) : (TC)0;
    }
    if constexpr (NI > 0) {
        for (int t = threadIdx.x; t < NI * NI; t += blockDim.x) S[t] = Sg[t];
        for (int t = threadIdx.x; t < NI; t += blockDim.x) lam[t] = lamg[t];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    TC* a = ab[wid][0];
    TC* b = ab[wid][1];
    const TC rsc = rs;
    for (int64_t e = (int64_t)blockIdx.x * W + wid; e < E; e += (int64_t)gridDim.x * W) {
        const TI* re = r + e * N3;
        TI* ze = z + e * N3;
        TC acc[8];
#pragma unroll
        for (int c = 0; c < 8; c++) acc[c] = (TC)0;
        for (int t = lane; t < N3; t += 32) {
            const TC v = (TC)re[t] * rsc;
            const int i = t % LX, j = (t / LX) % LX, k = t / (LX * LX);
            if constexpr (MODE != kSchRestrict) {
                const bool interior = i > 0 && i < LX - 1 && j > 0 && j < LX - 1 && k > 0 && k < LX - 1;
                if (interior) {
                    if constexpr (NI > 0) a[((k - 1) * NI + (j - 1)) * NI + (i - 1)] = v;
                } else {
                    ze[t] = (TI)((TC)minv[e * N3 + t] * v);
                }
            }
            if constexpr (MODE != kSchLocal) {
                const TC vm = v * inv[mult[e * N3 + t]];
                const TC a0 = F[0][i] * vm, a1 = F[1][i] * vm;
                const TC bj[4] = {a0 * F[0][j], a1 * F[0][j], a0 * F[1][j], a1 * F[1][j]};
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    acc[c] = fma(bj[c], F[0][k], acc[c]);
                    acc[c + 4] = fma(bj[c], F[1][k], acc[c + 4]);
                }
            }
        }
        if constexpr (MODE != kSchLocal) {
#pragma unroll
            for (int c = 0; c < 8; c++)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], o);
            if (lane == 0)
#pragma unroll
                for (int c = 0; c < 8; c++) rc[e * 8 + c] = (TI)acc[c];
        }
        if constexpr (NI > 0 && MODE != kSchRestrict) {
            // sqrt(2 / L_d) and h1m 4 / L_d^2, precomputed per element at set-up
            const TC* fe = fac + e * 6;
            const TC sr = fe[0], ss = fe[1], st = fe[2], cr = fe[3], cs = fe[4], ct = fe[5];
            __syncwarp();
            for (int t = lane; t < M3; t += 32) {  // along i: b[k][j][m] = sr sum_i S[i][m] a[k][j][i]
                const int m = t % NI, j = (t / NI) % NI, k = t / (NI * NI);
                TC s = (TC)0;
#pragma unroll
                for (int i = 0; i < NI; i++) s = fma(S[i * NI + m], a[(k * NI + j) * NI + i], s);
                b[t] = sr * s;
            }
            __syncwarp();
            for (int t = lane; t < M3; t += 32) {  // along j
                const int i = t % NI, m = (t / NI) % NI, k = t / (NI * NI);
                TC s = (TC)0;
#pragma unroll
                for (int j = 0; j < NI; j++) s = fma(S[j * NI + m], b[(k * NI + j) * NI + i], s);
                a[t] = ss * s;
            }
            __syncwarp();
            for (int t = lane; t < M3; t += 32) {  // along k, then the diagonal
                const int i = t % NI, j = (t / NI) % NI, m = t / (NI * NI);
                TC s = (TC)0;
#pragma unroll
                for (int k = 0; k < NI; k++) s = fma(S[k * NI + m], a[(k * NI + j) * NI + i], s);
                b[t] = st * s / (lam[i] * cr + lam[j] * cs + lam[m] * ct);
            }
            __syncwarp();
            for (int t = lane; t < M3; t += 32) {  // back along k
                const int i = t % NI, j = (t / NI) % NI, k = t / (NI * NI);
                TC s = (TC)0;
#pragma unroll
                for (int m = 0; m < NI; m++) s = fma(S[k * NI + m], b[(m * NI + j) * NI + i], s);
                a[t] = st * s;
            }
            __syncwarp();
            for (int t = lane; t < M3; t += 32) {  // back along j
                const int i = t % NI, j = (t / NI) % NI, k = t / (NI * NI);
                TC s = (TC)0;
#pragma unroll
                for (int m = 0; m < NI; m++) s = fma(S[j * NI + m], a[(k * NI + m) * NI + i], s);
                b[t] = ss * s;
            }
            __syncwarp();
            for (int t = lane; t < M3; t += 32) {  // back along i, out
                const int i = t % NI, j = (t / NI) % NI, k = t / (NI * NI);
                TC s = (TC)0;
#pragma unroll
                for (int m = 0; m < NI; m++) s = fma(S[i * NI + m], b[(k * NI + j) * NI + m], s);
                ze[((k + 1) * LX + (j + 1)) * LX + (i + 1)] = (TI)(sr * s);
            }
        }
        __syncwarp();  // a and b are rewritten by this warp's next element
    }
}

// z = mask (z + sum_c Pw[q][c] xc[e][c]), one warp per element: trilinear
// interpolation of the element's corner values through the 1-D factors
template <int LX, typename TI, typename TC>
__global__ void __launch_bounds__(256) prolong_kernel(TI* __restrict__ z, const TI* __restrict__ xc,
                                                      const TC* __restrict__ Pw, const uint8_t* __restrict__ mask,
                                                      int64_t E) {
    constexpr int N3 = LX * LX * LX;
    __shared__ TC F[2][LX];
    for (int t = threadIdx.x; t < 2 * LX; t += blockDim.x) F[t / LX][t % LX] = Pw[(t % LX) * 8 + t / LX];
    __syncthreads();
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int64_t e = (int64_t)blockIdx.x * nw + (threadIdx.x >> 5); e < E; e += (int64_t)gridDim.x * nw) {
        const TC xv = lane < 8 ? (TC)xc[e * 8 + lane] : (TC)0;  // 8 conversions per element
        TC c8[8];
#pragma unroll
        for (int c = 0; c < 8; c++) c8[c] = __shfl_sync(0xffffffffu, xv, c);
        for (int t = lane; t < N3; t += 32) {
            const int i = t % LX, j = (t / LX) % LX, k = t / (LX * LX);
            TC y[4];  // along k, then j, then i: corr = sum_c F[c&1][i] F[c>>1&1][j] F[c>>2][k] x_c
#pragma unroll
            for (int c = 0; c < 4; c++) y[c] = fma(F[0][k], c8[c], F[1][k] * c8[c + 4]);
            const TC y0 = fma(F[0][j], y[0], F[1][j] * y[2]), y1 = fma(F[0][j], y[1], F[1][j] * y[3]);
            const TC corr = fma(F[0][i], y0, F[1][i] * y1);
            const int64_t L = e * N3 + t;
            z[L] = mask[L] ? (TI)(z[L] + (TI)corr) : (TI)0;
        }
    }
}

template <typename TC>
static const TC* sch_table(const SchwarzData& sc, int which) {  // 0 Pw, 1 S, 2 lam, 3 fac
    if constexpr (std::is_same<TC, double>::value)
        return which == 0 ? sc.Pw : which == 1 ? sc.S : which == 2 ? sc.lam : sc.fac;
    else
        return which == 0 ? sc.Pw32 : which == 1 ? sc.S32 : which == 2 ? sc.lam32 : sc.fac32;
}

// the element-corner restriction (E x 8 values, in the coarse handle's work
// vector) in the precision of the fine data
template <typename TI>
static TI* coarse_rhs(sem_handle* hc) {
    if constexpr (std::is_same<TI, double>::value)
        return hc->ws.b;
    else
        return hc->ws.b32;
}

template <int LX, typename TI, typename TC, int MODE>
static int launch_local_m(sem_handle* h, const TI* r, const double* r_norm2, TI* z, const TI* minv,
                          cudaStream_t s) {
    const SchwarzData& sc = h->sch;
    const int64_t E = h->parts[0].E;
    constexpr int W = sch_warps<LX, TC>();
    int64_t cap = (int64_t)h->sm_count * 16;
    if (MODE == kSchLocal) {
        // beside the coarse CG: one CTA slot per SM below this kernel's
        // occupancy stays free, so the coarse launches (at most one CTA per SM)
        // run while it does
        static int per_sm = 0;
        if (per_sm == 0) {
            int nb = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, schwarz_local_kernel<LX, TI, TC, MODE>, W * 32, 0);
            per_sm = nb > 1 ? nb - 1 : 1;
        }
        cap = (int64_t)h->sm_count * per_sm;
    }
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((E + W - 1) / W, cap));
    schwarz_local_kernel<LX, TI, TC, MODE><<<grid, W * 32, 0, s>>>(
        r, r_norm2, z, minv, h->mult, sch_table<TC>(sc, 0), sch_table<TC>(sc, 1), sch_table<TC>(sc, 2),
        sch_table<TC>(sc, 3), coarse_rhs<TI>(sc.coarse), E);
    SEM_LAUNCH_CHECK("schwarz_local_kernel");
    h->launches++;
    return SEM_OK;
}

template <int LX, typename TI, typename TC>
static int launch_local_t(sem_handle* h, int mode, const TI* r, const double* r_norm2, TI* z, const TI* minv,
                          cudaStream_t s) {
    return mode == kSchRestrict ? launch_local_m<LX, TI, TC, kSchRestrict>(h, r, r_norm2, z, minv, s)
           : mode == kSchLocal  ? launch_local_m<LX, TI, TC, kSchLocal>(h, r, r_norm2, z, minv, s)
                                : launch_local_m<LX, TI, TC, kSchAll>(h, r, r_norm2, z, minv, s);
}

template <int LX, typename TI, typename TC>
static int launch_prolong_t(sem_handle* h, TI* z, const TI* xc, cudaStream_t s) {
    const SchwarzData& sc = h->sch;
    const int64_t E = h->parts[0].E;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((E + 7) / 8, (int64_t)h->sm_count * 8));
    prolong_kernel<LX, TI, TC><<<grid, 256, 0, s>>>(z, xc, sch_table<TC>(sc, 0), h->mask, E);
    SEM_LAUNCH_CHECK("prolong_kernel");
    h->launches++;
    return SEM_OK;
}

// phase kSchAll / kSchRestrict / kSchLocal: the local part (SchMode);
// phase -1: the prolongation of the element-corner values xc
template <typename TI, typename TC>
static int launch_schwarz_phase(sem_handle* h, int phase, const TI* r, const double* r_norm2, TI* z, const TI* minv,
                                const TI* xc, cudaStream_t s) {
#define SEM_SCH_CASE(LXV)                                                                   \
    case LXV:                                                                                \
        return phase >= 0 ? launch_local_t<LXV, TI, TC>(h, phase, r, r_norm2, z, minv, s)  \
                          : launch_prolong_t<LXV, TI, TC>(h, z, xc, s);
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
// local arithmetic TC, the coarse CG (assembled, 10 Jacobi-PCG iterations) in
// the precision of the data; the input is r / sqrt(*r_norm2) when r_norm2 (a
// device scalar) is given
template <typename TI, typename TC>
static int apply_schwarz(sem_handle* h, const TI* r, const double* r_norm2, TI* z, bool coop, cudaStream_t s) {
    sem_handle* hc = h->sch.coarse;
    const TI* minv;
    if constexpr (std::is_same<TI, double>::value)
        minv = h->minv64;
    else
        minv = h->minv32;
    SchwarzData& sc = h->sch;
    const TI* xc = coarse_csr_x<TI>(h);
    int rc;
    if (!sc.aux) {  // one stream: local part with the restriction, coarse CG, prolongation
        if ((rc = launch_schwarz_phase<TI, TC>(h, kSchAll, r, r_norm2, z, minv, nullptr, s)) ||
            (rc = coarse_csr_solve<TI>(h, coarse_rhs<TI>(hc), 10, coop, s)))
            return rc;
        return launch_schwarz_phase<TI, TC>(h, -1, r, r_norm2, z, minv, xc, s);
    }
    // the coarse CG on the handle's second stream, beside the local solves
    // (the local-solve kernel is queued first, so that it starts while the
    // host is still queueing the coarse CG's launches)
    if ((rc = launch_schwarz_phase<TI, TC>(h, kSchRestrict, r, r_norm2, z, minv, nullptr, s))) return rc;
    SEM_CUDA_TRY(cudaEventRecord(sc.ev_restrict, s));
    if ((rc = launch_schwarz_phase<TI, TC>(h, kSchLocal, r, r_norm2, z, minv, nullptr, s))) return rc;
    SEM_CUDA_TRY(cudaStreamWaitEvent(sc.aux, sc.ev_restrict, 0));
    if ((rc = coarse_csr_solve<TI>(h, coarse_rhs<TI>(hc), 10, coop, sc.aux))) return rc;
    SEM_CUDA_TRY(cudaEventRecord(sc.ev_coarse, sc.aux));
    SEM_CUDA_TRY(cudaStreamWaitEvent(s, sc.ev_coarse, 0));
    return launch_schwarz_phase<TI, TC>(h, -1, r, r_norm2, z, minv, xc, s);
}

// the second stream and its two events (created at the first GMRES solve; a
// handle without them applies the preconditioner on one stream)
static void ensure_aux_stream(sem_handle* h) {
    SchwarzData& sc = h->sch;
    if (sc.aux) return;
    // the highest priority: its small kernels take SM slots as soon as blocks of
    // the local-solve kernel finish
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (cudaStreamCreateWithPriority(&sc.aux, cudaStreamNonBlocking, greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&sc.ev_restrict, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sc.ev_coarse, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (sc.ev_restrict) cudaEventDestroy(sc.ev_restrict);
        if (sc.aux) cudaStreamDestroy(sc.aux);
        sc.aux = nullptr;
        sc.ev_restrict = sc.ev_coarse = nullptr;
    }
}

void free_schwarz(sem_handle* h) {
    SchwarzData& sc = h->sch;
    free_coarse_csr(sc.csr);
    if (sc.aux) {
        cudaStreamSynchronize(sc.aux);
        cudaEventDestroy(sc.ev_restrict);
        cudaEventDestroy(sc.ev_coarse);
        cudaStreamDestroy(sc.aux);
    }
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
        int rc = dalloc(h, &sc.coef, (size_t)kCoefStride * kRegions);
        if (!rc) rc = dalloc(h, &sc.gpart, (size_t)(2 * kGmNV) * kMaxPartials);
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

// One Gram-Schmidt pass over the handle's GMRES basis
template <typename T>
static int gs_pass(sem_handle* h, T* w, int sub_cnt, const double* sub_coef, int dot_cnt, double* dot_out,
                   double* norm_out, cudaStream_t s) {
    SchwarzData& sc = h->sch;
    return krylov_pass<T>(h, w, static_cast<const T*>(sc.V), sc.ld, sub_cnt, sub_coef, dot_cnt, dot_out, norm_out,
                          sc.gpart, sc.gcount, s);
}

// w = mask QQ^T A_L z with the operator of the solve's precision
template <typename T>
static int apply_operator(sem_handle* h, const T* z, T* w, int op_prec, cudaStream_t s) {
    int rc = launch_ax_local(h, z, w, std::is_same<T, float>::value ? SEM_FP32 : op_prec, s);
    return rc ? rc : launch_gs(h, w, std::is_same<T, float>::value, true, s);
}

// A staged operator kernel (fine handle) or the cooperative coarse CG (coarse
// handle's word) that gave up a bounded wait set the error word and returned:
// the solve ends with SEM_ETIMEOUT, the context intact.
static int check_error_words(sem_handle* h, cudaStream_t s) {
    for (sem_handle* q : {h, h->sch.coarse}) {
        int word = 0;
        SEM_CUDA_TRY(cudaMemcpyAsync(&word, device_error_word(q), sizeof(int), cudaMemcpyDeviceToHost, s));
        SEM_CUDA_TRY(cudaStreamSynchronize(s));
        if (word) {
            cudaMemset(device_error_word(q), 0, sizeof(int));
            cudaMemset(q->counters, 0, 16 * sizeof(unsigned));
            if (q == h->sch.coarse) cudaMemset(h->sch.csr.bar, 0, 2 * sizeof(unsigned));
            return fail(SEM_ETIMEOUT, "a bounded device-side wait of the GMRES solve expired");
        }
    }
    return SEM_OK;
}

// Least-squares state of one restart cycle: the Hessenberg columns after the
// Givens rotations, the rotations, and the rotated right-hand side g
struct GmLsq {
    int m = 0;
    std::vector<double> H, g, cs, sn;
    void start(int m_, double beta) {
        m = m_;
        H.assign((size_t)(m + 1) * m, 0.0);
        g.assign(m + 1, 0.0);
        cs.assign(m, 0.0);
        sn.assign(m, 0.0);
        g[0] = beta;
    }
    // column j with entries h[0..j+1]; false on breakdown; *res = |g[j+1]|
    bool add(int j, double* h, double* res) {
        for (int i = 0; i < j; i++) {
            const double t = cs[i] * h[i] + sn[i] * h[i + 1];
            h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
            h[i] = t;
        }
        const double den = std::hypot(h[j], h[j + 1]);
        if (!(den > 0.0) || !std::isfinite(den)) return false;
        cs[j] = h[j] / den;
        sn[j] = h[j + 1] / den;
        h[j] = den;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        for (int i = 0; i <= j; i++) H[(size_t)i * m + j] = h[i];
        *res = std::fabs(g[j + 1]);
        return true;
    }
    void solve(int k, std::vector<double>& y) const {  // H y = g, upper triangular
        for (int i = k - 1; i >= 0; i--) {
            double t = g[i];
            for (int q = i + 1; q < k; q++) t -= H[(size_t)i * m + q] * y[q];
            y[i] = t / H[(size_t)i * m + i];
        }
    }
};

struct GmCycle {
    int k = 0;            // columns completed
    int status = SEM_OK;  // SEM_EBREAKDOWN on a breakdown
};

template <typename T>
static int schwarz_step(sem_handle* h, const sem_solve_opts& o, const T* v, const double* v_norm2, T* z,
                        cudaStream_t s) {
    const bool coop = o.persistent != 0;  // the coarse CG as one cooperative launch
    if constexpr (std::is_same<T, float>::value)
        return apply_schwarz<float, float>(h, v, v_norm2, z, coop, s);
    else
        return o.precond_precision == SEM_FP32 ? apply_schwarz<double, float>(h, v, v_norm2, z, coop, s)
                                               : apply_schwarz<double, double>(h, v, v_norm2, z, coop, s);
}

// One restart cycle with classical Gram-Schmidt once (orth 1) or twice in the
// same step (orth 3): per step z_j = M v_j, w = A z_j, the passes, v_{j+1} =
// w / ||w||, one host read of the coefficients.
template <typename T>
static int cycle_classic(sem_handle* h, const sem_solve_opts& o, int it0, double stop, T* w, GmLsq& ls,
                         GmCycle* out, cudaStream_t s) {
    SchwarzData& sc = h->sch;
    const int m = o.gmres_restart;
    const bool twice = o.gmres_orth == 3;
    T* Vb = static_cast<T*>(sc.V);
    T* Zb = static_cast<T*>(sc.Z);
    double* c1 = sc.coef + kRegA * kCoefStride;
    double* c2 = sc.coef + kRegB * kCoefStride;
    double* nrm = sc.coef + kRegNorm * kCoefStride;
    std::vector<double> hcol(m + 2), hc(2 * kCoefStride + 1);
    int rc;
    for (int j = 0; j < m && it0 + j < o.max_iter; j++) {
        T* vj = Vb + (int64_t)j * sc.ld;
        T* zj = Zb + (int64_t)j * sc.ld;
        if ((rc = schwarz_step<T>(h, o, vj, nullptr, zj, s)) || (rc = apply_operator<T>(h, zj, w, o.precision, s)))
            return rc;
        const int c = j + 1;
        // c1 = V^T w; w -= V c1 (twice: c2 = V^T w; w -= V c2); ||w||^2
        if ((rc = gs_pass<T>(h, w, 0, nullptr, c, c1, nullptr, s))) return rc;
        if (twice && (rc = gs_pass<T>(h, w, c, c1, c, c2, nullptr, s))) return rc;
        if ((rc = gs_pass<T>(h, w, c, twice ? c2 : c1, 0, nullptr, nrm, s))) return rc;
        gm_scale_kernel<T><<<grid_for(h, h->n_local, 256, 8), 256, 0, s>>>(Vb + (int64_t)c * sc.ld, w, nrm,
                                                                           h->n_local);
        SEM_LAUNCH_CHECK("gm_scale_kernel");
        h->launches++;
        if ((rc = read_scalars(hc.data(), sc.coef, 2 * kCoefStride + 1, s))) return rc;
        for (int i = 0; i < c; i++) hcol[i] = hc[i] + (twice ? hc[kCoefStride + i] : 0.0);
        const double ww = hc[2 * kCoefStride];
        hcol[c] = std::sqrt(std::max(ww, 0.0));
        double res = 0.0;
        if (!ls.add(j, hcol.data(), &res)) {
            out->status = SEM_EBREAKDOWN;
            return SEM_OK;
        }
        out->k = c;
        if (res <= stop || !(ww > 0.0)) break;
    }
    return SEM_OK;
}

// One restart cycle with classical Gram-Schmidt twice, the second pass lagged
// into the next step (orth 2, the default; after Swirydowicz et al. 2021).
// Slot j holds u_j: v_j = u_j / rho_j orthogonalised once (rho_j^2 = <u_j, u_j>
// on the device, written by the previous step; slot 0 holds the normalised
// start).  Step j:
//   z_j = M v_j (the Schwarz kernel scales u_j by 1 / rho_j), w = A z_j;
//   one pass: a_i = <X_i, u_j>, b_i = <X_i, w> for i <= j;
//   host: s_i = a_i / rho_j (i < j), rho'_j = sqrt(a_j / rho_j^2 - |s|^2),
//         v_j = V s + rho'_j v'_j, so column j-1 (A z_{j-1} = sum h_i V_i +
//         rho_j v_j) becomes h_i + rho_j s_i with subdiagonal rho_j rho'_j and
//         is rotated; t_i = b_i, kappa = <v'_j, w> = (b_j / rho_j - s.t) / rho'_j;
//   one pass: slot j <- v'_j = (u_j / rho_j - V s) / rho'_j and slot j+1 <-
//         u_{j+1} = w - V t - kappa v'_j, rho_{j+1}^2.
// Column j gets its subdiagonal (and its reorthogonalisation correction) at
// step j+1, so the residual estimate of a column is known one operator
// application later; a cycle that ends after m steps takes the last
// subdiagonal without reorthogonalisation.  In exact arithmetic s = 0 and
// this is FGMRES with classical Gram-Schmidt.
template <typename T>
static int cycle_lagged(sem_handle* h, const sem_solve_opts& o, int it0, double stop, T* w, GmLsq& ls,
                        GmCycle* out, cudaStream_t s) {
    SchwarzData& sc = h->sch;
    const int m = o.gmres_restart;
    const int64_t n = h->n_local;
    T* Xb = static_cast<T*>(sc.V);
    T* Zb = static_cast<T*>(sc.Z);
    double* A = sc.coef + kRegA * kCoefStride;
    double* B = sc.coef + kRegB * kCoefStride;
    double* NR = sc.coef + kRegNorm * kCoefStride;
    double* SC = sc.coef + kRegSc * kCoefStride;
    double* TC = sc.coef + kRegTc * kCoefStride;
    std::vector<double> hc(2 * kCoefStride + 1), hcol(m + 2), pc(m + 1), sv(m + 1), tv(m + 1), up(2 * kCoefStride);
    static int per_sm = 0;
    if (per_sm == 0) {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, gm_dots2_kernel<T, kGmNV>, 256, 0);
        per_sm = std::max(nb, 1);
    }
    const int64_t packs = n / (16 / (int64_t)sizeof(T));
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>({(packs + 255) / 256, (int64_t)h->sm_count * per_sm, (int64_t)kMaxPartials}));
    int rc;
    for (int j = 0;; j++) {
        const bool last = j == m || it0 + j >= o.max_iter;  // no further Arnoldi step in this cycle
        T* uj = Xb + (int64_t)j * sc.ld;
        if (!last) {
            T* zj = Zb + (int64_t)j * sc.ld;
            if ((rc = schwarz_step<T>(h, o, uj, j > 0 ? NR : nullptr, zj, s)) ||
                (rc = apply_operator<T>(h, zj, w, o.precision, s)))
                return rc;
            for (int lo = 0; lo <= j; lo += kGmNV) {
                gm_dots2_kernel<T, kGmNV><<<grid, 256, 0, s>>>(Xb, sc.ld, n, lo, std::min(kGmNV, j + 1 - lo), uj, w,
                                                               h->mult, A + lo, B + lo, sc.gpart, sc.gcount);
                SEM_LAUNCH_CHECK("gm_dots2_kernel");
                h->launches++;
            }
        }
        if ((rc = read_scalars(hc.data(), sc.coef, 2 * kCoefStride + 1, s))) return rc;
        const double rho = j == 0 ? 1.0 : std::sqrt(std::max(hc[2 * kCoefStride], 0.0));
        double rhop = 1.0, ss = 0.0;
        for (int i = 0; i < j; i++) sv[i] = 0.0;
        if (!last && j > 0 && rho > 0.0) {  // reorthogonalisation of v_j
            for (int i = 0; i < j; i++) {
                sv[i] = hc[i] / rho;
                ss += sv[i] * sv[i];
            }
            const double sigma = hc[j] / (rho * rho);
            rhop = std::sqrt(std::max(sigma - ss, 0.0));
            if (!(rhop > 0.0) || !std::isfinite(rhop)) {
                out->status = SEM_EBREAKDOWN;
                return SEM_OK;
            }
        }
        if (j > 0) {  // column j-1 is complete
            for (int i = 0; i < j; i++) hcol[i] = pc[i] + rho * sv[i];
            hcol[j] = rho * rhop;
            double res = 0.0;
            if (!ls.add(j - 1, hcol.data(), &res)) {
                out->status = SEM_EBREAKDOWN;
                return SEM_OK;
            }
            out->k = j;
            if (res <= stop || last || !(rho > 0.0)) break;
        }
        if (last) break;
        // this step's pass: v'_j and u_{j+1}
        double st = 0.0;
        for (int i = 0; i < j; i++) {
            tv[i] = hc[kCoefStride + i];
            st += sv[i] * tv[i];
        }
        const double kappa = (hc[kCoefStride + j] / rho - st) / rhop;
        const double cu = 1.0 / (rho * rhop);
        for (int i = 0; i < j; i++) {
            up[i] = sv[i] / rhop;                         // sc_i
            up[kCoefStride + i] = tv[i] - kappa * up[i];  // tc_i
            pc[i] = tv[i];
        }
        up[j] = cu;
        up[kCoefStride + j] = kappa * cu;
        pc[j] = kappa;
        SEM_CUDA_TRY(cudaMemcpyAsync(SC, up.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, s));
        SEM_CUDA_TRY(
            cudaMemcpyAsync(TC, up.data() + kCoefStride, sizeof(double) * (j + 1), cudaMemcpyHostToDevice, s));
        gm_lagged_update_kernel<T><<<grid, 256, 0, s>>>(Xb, sc.ld, n, j, SC, TC, j > 0 ? 1 : 0, w, h->mult, NR,
                                                        sc.gpart, sc.gcount);
        SEM_LAUNCH_CHECK("gm_lagged_update_kernel");
        h->launches++;
    }
    return SEM_OK;
}

template <typename T>
static int solve_gmres_t(sem_handle* h, const sem_solve_opts& o, sem_solve_stats* st, cudaStream_t s) {
    constexpr bool kMixed = std::is_same<T, float>::value;
    SchwarzData& sc = h->sch;
    const int m = o.gmres_restart;
    const int64_t n = h->n_local;
    T* w;
    if constexpr (kMixed)
        w = h->ws.w32;
    else
        w = h->ws.w;
    T* Vb = static_cast<T*>(sc.V);
    T* Zb = static_cast<T*>(sc.Z);
    double* yd = sc.coef + kRegY * kCoefStride;
    GmLsq ls;
    std::vector<double> y(m);
    double hb[2] = {0.0, 0.0};
    double rel_prev = INFINITY;
    int status = SEM_ENOTCONV, it = 0, cycles = 0, rc;
    for (;;) {
        if ((rc = true_residual(h, h->ws.x, h->ws.b, h->scratch, s)) || (rc = read_scalars(hb, h->scratch, 2, s)) ||
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
        gm_start_kernel<T><<<grid_for(h, n, 256, 8), 256, 0, s>>>(Vb, h->ws.r, 1.0 / beta, n);
        SEM_LAUNCH_CHECK("gm_start_kernel");
        h->launches++;
        ls.start(m, beta);
        GmCycle cyc;
        rc = o.gmres_orth == 2 ? cycle_lagged<T>(h, o, it, stop, w, ls, &cyc, s)
                               : cycle_classic<T>(h, o, it, stop, w, ls, &cyc, s);
        if (rc) return rc;
        // a kernel that gave up a bounded wait leaves unfinished vectors, which
        // can end the cycle as a breakdown: the expired wait is what to report
        if ((rc = check_error_words(h, s))) return rc;
        if (cyc.status == SEM_EBREAKDOWN) {
            status = SEM_EBREAKDOWN;
            break;
        }
        it += cyc.k;
        if (cyc.k > 0) {
            ls.solve(cyc.k, y);
            SEM_CUDA_TRY(cudaMemcpyAsync(yd, y.data(), sizeof(double) * cyc.k, cudaMemcpyHostToDevice, s));
            if ((rc = krylov_update<T>(h, h->ws.x, Zb, sc.ld, yd, cyc.k, s))) return rc;
        }
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
    if (o.gmres_orth < 1 || o.gmres_orth > 3) return fail(SEM_EINVAL, "gmres_orth must be 1, 2 or 3");
    int rc = ensure_workspace(h, mixed);
    if (!rc) rc = ensure_workspace(h->sch.coarse, mixed);
    if (!rc) rc = ensure_krylov(h, m, mixed ? (int)sizeof(float) : (int)sizeof(double));
    if (!rc) ensure_aux_stream(h);
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
    // projection onto previous solutions: the start is the projected solution
    if (o.projection > 0) rc = proj_start(h, o.projection, s);
    if (!rc) rc = mixed ? solve_gmres_t<float>(h, o, &st, s) : solve_gmres_t<double>(h, o, &st, s);
    if (!rc && o.projection > 0 && st.status == SEM_OK) rc = proj_update(h, s);
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
    return rc ? rc : apply_schwarz<double, double>(h, r, nullptr, z, false, s);
}

SEM_API int sem_schwarz_apply32(sem_handle* h, const float* r, float* z, cudaStream_t s) {
    if (!h || !r || !z) return fail(SEM_EINVAL, "null argument");
    if (r == z) return fail(SEM_EINVAL, "z must not alias r");
    if (h->nsolve != 1 || !h->sch.coarse) return fail(SEM_EINVAL, "the handle has no Schwarz preconditioner");
    int rc = ensure_workspace(h->sch.coarse, true);
    return rc ? rc : apply_schwarz<float, float>(h, r, nullptr, z, false, s);
}

}  // extern "C"
