// Native FP64 local operator with line transforms and even/odd splitting
// (variant 9): w = D^T (h1 G) D u (Sec. II-A of Karp et al., eq. "disclap")
// in plain double arithmetic, with the derivative contractions written so
// that GB300's FP64 pipe (1/64 of the FP32 rate, and the bound of the native
// operator) executes fewer instructions per point.
//
// D and D^T of the GLL points are centro-antisymmetric (M_{N-i,N-m} = -M_im),
// so one line y = M x of lx points (N = lx - 1, P = lx/2) splits into
//   e_m = x_m + x_{N-m},  o_m = x_m - x_{N-m}             (m < P)
//   S_i = sum_m A_im o_m,  T_i = sum_m B_im e_m           (i < P)
//   y_i = S_i + T_i,       y_{N-i} = S_i - T_i
// with A_im = (M_im - M_{i,N-m}) / 2, B_im = (M_im + M_{i,N-m}) / 2: 6 FP64
// operations per point for lx = 8 instead of 8 (7 where the result is
// accumulated).  Per point: 18 (forward) + 9 (G weighting) + 20 (backward)
// against 57 for the direct contractions.  The rounding differs from the
// direct sums by O(2^-53 sum |M||x|), the same order as their own error.
//
// Thread layout: a CTA owns EPC elements (2 at lx = 8, else 256/lx^2), lx^2
// threads each.
// Thread (lo, hi) owns the column (i = lo, j = hi) of its element for the
// loads, the G weighting and the output, and one line per direction in the
// transforms: the r-line (k = hi, j = lo), the s-line (k = hi, i = lo) and
// the t-line (j = hi, i = lo), which is its own column and stays in its
// registers.  Element blocks live in shared memory in three arrays (u, then
// w; ur/wr; us/ws) with padded row and plane strides.  Even lx in
// {4, 6, 8, 10, 12}.
#pragma once

#include "sem_ax.cuh"

namespace sem {

// Even/odd tables of every even order in the constant bank: [dir][A/B][P][P]
// (dir 0 = D, 1 = D^T) at ln_coef_off(lx); the unrolled transforms take
// them as constant-bank operands of the FP64 multiplies.
constexpr int ln_coef_off(int lx) {
    return lx == 4 ? 0 : lx == 6 ? 16 : lx == 8 ? 52 : lx == 10 ? 116 : lx == 12 ? 216 : -1;
}
constexpr int kLnCoefTotal = 360;
static __constant__ double c_lncoef[kLnCoefTotal];

template <int LX>
struct LnCfg {
    static constexpr int P = LX / 2;
    static constexpr int N2 = LX * LX, N3 = LX * LX * LX;
    // padded row and plane strides (doubles), chosen by a search over the
    // column, r-, s- and t-line access patterns of a warp for the fewest
    // shared-memory wavefronts (8-byte accesses, half-warp phases)
    static constexpr int LXP = LX == 4 ? 4 : LX == 6 ? 9 : LX == 8 ? 9 : LX == 10 ? 10 : 13;
    static constexpr int N2P = LX == 4 ? 19 : LX == 6 ? 54 : LX == 8 ? 72 : LX == 10 ? 106 : 156;
    static constexpr int SLOT = LX * N2P;  // doubles per element per array
    // elements per CTA: two at lx = 8 (128 threads), else up to 256 threads
    static constexpr int EPC = LX == 8 ? 2 : (256 / N2) > 0 ? (256 / N2) : 1;
    static constexpr int USED = EPC * N2;
    static constexpr int THREADS = ((USED + 31) / 32) * 32;
    static constexpr size_t BYTES = sizeof(double) * 3 * (size_t)EPC * SLOT;
    // CTAs per SM the register allocation is held to.  The FP64 pipe (2
    // thread-operations per cycle per SM) bounds the kernel.  At lx = 8 two
    // CTAs of 128 threads, unconstrained (203 registers in the CG form, no
    // spills): three at a 170-register cap spill and measured 0.9% slower;
    // the other orders take what they need.
    static constexpr int MINB = LX == 8 ? 2 : 1;
    static __host__ __device__ constexpr int at(int k, int j, int i) { return k * N2P + j * LXP + i; }
    static_assert(LX % 2 == 0 && LX >= 4 && LX <= 12, "line transforms need even lx in [4, 12]");
    static_assert(LXP >= LX && N2P >= LX * LXP, "padded strides must cover a plane");
};

// One line: y = M x (ACC: y += M x), x at x[0], x[xst], ..., y at y[0],
// y[yst], ...; M given by its tables A, B at constant-bank offset CA.
template <int LX, int CA, bool ACC>
__device__ __forceinline__ void ln_line(const double* x, int xst, double* y, int yst) {
    constexpr int P = LX / 2, N = LX - 1, PP = P * P;
    const double* A = c_lncoef + CA;
    const double* B = c_lncoef + CA + PP;
    double e[P], o[P];
#pragma unroll
    for (int m = 0; m < P; m++) {
        const double a = x[m * xst], b = x[(N - m) * xst];
        e[m] = a + b;
        o[m] = a - b;
    }
#pragma unroll
    for (int i = 0; i < P; i++) {
        double S = A[i * P] * o[0], T = B[i * P] * e[0];
#pragma unroll
        for (int m = 1; m < P; m++) {
            S = fma(A[i * P + m], o[m], S);
            T = fma(B[i * P + m], e[m], T);
        }
        if (ACC) {
            y[i * yst] = (y[i * yst] + S) + T;
            y[(N - i) * yst] = (y[(N - i) * yst] + S) - T;
        } else {
            y[i * yst] = S + T;
            y[(N - i) * yst] = S - T;
        }
    }
}

// The same transform on a line held in registers: y = M x, or with ACC
// y_i = (y_i + S_i) + T_i and y_{N-i} = (y_{N-i} + S_i) - T_i, the same
// operations in the same order as ln_line.
template <int LX, int CA, bool ACC>
__device__ __forceinline__ void ln_line_reg(const double (&x)[LX], double (&y)[LX]) {
    constexpr int P = LX / 2, N = LX - 1, PP = P * P;
    const double* A = c_lncoef + CA;
    const double* B = c_lncoef + CA + PP;
    double e[P], o[P];
#pragma unroll
    for (int m = 0; m < P; m++) {
        e[m] = x[m] + x[N - m];
        o[m] = x[m] - x[N - m];
    }
#pragma unroll
    for (int i = 0; i < P; i++) {
        double S = A[i * P] * o[0], T = B[i * P] * e[0];
#pragma unroll
        for (int m = 1; m < P; m++) {
            S = fma(A[i * P + m], o[m], S);
            T = fma(B[i * P + m], e[m], T);
        }
        if (ACC) {
            y[i] = (y[i] + S) + T;
            y[N - i] = (y[N - i] + S) - T;
        } else {
            y[i] = S + T;
            y[N - i] = S - T;
        }
    }
}

template <int LX, bool FUSED>
__global__ void __launch_bounds__(LnCfg<LX>::THREADS, LnCfg<LX>::MINB) ax_ln_kernel(AxParams<double> a) {
    using C = LnCfg<LX>;
    constexpr int P = C::P, N2 = C::N2, N3 = C::N3, EPC = C::EPC, SLOT = C::SLOT;
    constexpr int LXP = C::LXP;
    constexpr int CF = ln_coef_off(LX), CB = CF + 2 * P * P;  // forward (D) and backward (D^T) tables
    extern __shared__ __align__(16) unsigned char smem_ln[];
    double* arr = reinterpret_cast<double*>(smem_ln);  // 3 arrays x EPC slots: u | r | s
    __shared__ double sb_beta;
    bool first = false;
    if (FUSED) {
        if (a.st->done) return;  // uniform over the grid
        if (threadIdx.x == 0) sb_beta = cg_beta(a.st);
        first = cg_first(a.st);
    } else if (a.skip_st && a.skip_st->done) {
        return;  // uniform over the grid
    }
    const int tid = threadIdx.x;
    const int el = tid / N2;
    const int t2 = tid - el * N2;            // column (i, j) in the column phases, line id in the transforms
    const int lo = t2 % LX, hi = t2 / LX;    // i / j of the column; also the line coordinates
    const bool active = el < EPC;
    const int slot = (active ? el : 0) * SLOT;
    double* su = arr + 0 * EPC * SLOT + slot;
    double* sr = arr + 1 * EPC * SLOT + slot;
    double* ss = arr + 2 * EPC * SLOT + slot;
    const int64_t ngroups = (a.E + EPC - 1) / EPC;
    double pap = 0.0;
    __syncthreads();
    const double beta = FUSED ? sb_beta : 0.0;
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const int64_t e = g * EPC + el;
        const bool valid = active && e < a.E;
        const int64_t base = e * N3 + t2;  // column (i = lo, j = hi)
        // phase 0: this thread's column of u (or z + beta p; p <- that)
        double ud[LX];
#pragma unroll
        for (int k = 0; k < LX; k++) ud[k] = valid ? ld_stream((FUSED ? a.z : a.u) + base + k * N2) : 0.0;
        if (FUSED) {
            double pold[LX];
#pragma unroll
            for (int k = 0; k < LX; k++) pold[k] = (valid && !first) ? a.p[base + k * N2] : 0.0;
#pragma unroll
            for (int k = 0; k < LX; k++) {
                ud[k] = fma(beta, pold[k], ud[k]);
                if (valid) a.p[base + k * N2] = ud[k];
            }
        }
        if (active) {
#pragma unroll
            for (int k = 0; k < LX; k++) su[C::at(k, hi, lo)] = ud[k];
        }
        // factors of the column's first point, requested now and used after phase 1
        const double* Ge = a.G + 6 * e * N3 + t2;
        double gc[6];
#pragma unroll
        for (int c = 0; c < 6; c++) gc[c] = valid ? ld_stream(Ge + c * N3) : 0.0;
        __syncthreads();
        // phase 1: derivative lines ur (along i) and us (along j) through shared
        // memory; ut along k is this thread's own column, from its registers
        double tcol[LX];  // ut, then wt, of the column
        if (active) {
            ln_line<LX, CF, false>(su + C::at(hi, lo, 0), 1, sr + C::at(hi, lo, 0), 1);
            ln_line<LX, CF, false>(su + C::at(hi, 0, lo), LXP, ss + C::at(hi, 0, lo), LXP);
            ln_line_reg<LX, CF, false>(ud, tcol);
        }
        __syncthreads();
        // phase 2: (wr, ws, wt) = G (ur, us, ut) at the column's points, in
        // the order of the other kernels; the factors of point k + 1 are
        // loaded while point k is computed
        if (active) {
#pragma unroll
            for (int k = 0; k < LX; k++) {
                double gn[6];
                if (k + 1 < LX) {
#pragma unroll
                    for (int c = 0; c < 6; c++) gn[c] = valid ? ld_stream(Ge + c * N3 + (k + 1) * N2) : 0.0;
                }
                const int q = C::at(k, hi, lo);
                const double ur = sr[q], us = ss[q], ut = tcol[k];
                sr[q] = fma(gc[0], ur, fma(gc[1], us, gc[2] * ut));
                ss[q] = fma(gc[1], ur, fma(gc[3], us, gc[4] * ut));
                tcol[k] = fma(gc[2], ur, fma(gc[4], us, gc[5] * ut));
                if (k + 1 < LX) {
#pragma unroll
                    for (int c = 0; c < 6; c++) gc[c] = gn[c];
                }
            }
        }
        __syncthreads();
        // phase 3: w = D^T-lines of wr (into the u array), += those of ws,
        // then += the D^T-line of wt along this thread's own column, in
        // registers (its r and s sums read back once, no barrier needed)
        if (active) ln_line<LX, CB, false>(sr + C::at(hi, lo, 0), 1, su + C::at(hi, lo, 0), 1);
        __syncthreads();
        if (active) ln_line<LX, CB, true>(ss + C::at(hi, 0, lo), LXP, su + C::at(hi, 0, lo), LXP);
        __syncthreads();
        double wcol[LX];
        if (active) {
#pragma unroll
            for (int k = 0; k < LX; k++) wcol[k] = su[C::at(k, hi, lo)];
            ln_line_reg<LX, CB, true>(tcol, wcol);
        }
        if (valid) {
            double pw = 0.0;
#pragma unroll
            for (int k = 0; k < LX; k++) {
                const double wv = wcol[k];
                st_keep<FUSED>(a.w + base + k * N2, wv);
                if (FUSED) pw = fma(ud[k], wv, pw);
            }
            if (FUSED) pap += pw;
        }
        __syncthreads();
    }
    if (FUSED) {
        CGState* cs = a.st;
        double v[1] = {pap};
        grid_sum_finalize<1>(v, a.partials, a.counter, [&](double (&acc)[1]) { cg_set_alpha(cs, acc[0]); });
    }
}

template <int LX, bool FUSED>
inline int launch_ax_ln_t(sem_handle* h, const AxParams<double>& a, cudaStream_t s) {
    using C = LnCfg<LX>;
    static int per_sm = -1;
    if (per_sm < 0) {
        cudaFuncSetAttribute(ax_ln_kernel<LX, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES);
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ax_ln_kernel<LX, FUSED>, C::THREADS, C::BYTES);
        per_sm = nb;
    }
    if (per_sm <= 0) return fail(SEM_EINVAL, "line-transform FP64 operator cannot be resident");
    if (a.dry) return SEM_OK;
    const int64_t ngroups = (a.E + C::EPC - 1) / C::EPC;
    int64_t grid = std::min<int64_t>(ngroups, (int64_t)h->sm_count * per_sm);
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, kMaxPartials));
    ax_ln_kernel<LX, FUSED><<<(int)grid, C::THREADS, C::BYTES, s>>>(a);
    SEM_LAUNCH_CHECK("ax_ln_kernel");
    h->launches++;
    return SEM_OK;
}

template <bool FUSED>
inline int dispatch_ax_ln(sem_handle* h, int lx, const AxParams<double>& a, cudaStream_t s) {
    switch (lx) {
        case 4: return launch_ax_ln_t<4, FUSED>(h, a, s);
        case 6: return launch_ax_ln_t<6, FUSED>(h, a, s);
        case 8: return launch_ax_ln_t<8, FUSED>(h, a, s);
        case 10: return launch_ax_ln_t<10, FUSED>(h, a, s);
        case 12: return launch_ax_ln_t<12, FUSED>(h, a, s);
        default: return fail(SEM_EINVAL, "line-transform FP64 operator needs lx in {4, 6, 8, 10, 12}");
    }
}

}  // namespace sem
