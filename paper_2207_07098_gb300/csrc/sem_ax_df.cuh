// FP64-accurate local operator on the FP32 pipe ("double-float" arithmetic).
//
// On GB300 the FP64 pipe runs at 1/64 of the FP32 rate, so an FP64 ax_helm
// with ~57 FP64 FMAs per point is limited to ~10% of HBM bandwidth.  This
// kernel keeps FP64 accuracy (relative error ~2^-44 per operation, far below
// the 1e-12 parity bar) with pairs of floats x = hi + lo:
//   * exact products with an FMA (p = a*b, e = fma(a, b, -p): p + e = a*b),
//   * sums of the high parts with Knuth's TwoSum (s + err = a + b exactly),
//   * the low-order cross terms (a_hi b_lo + a_lo b_hi) in plain FP32,
// applied to the same contractions and the same G weighting as ax_group.
// The factors are stored pre-split (12 float planes per element: the six hi
// planes then the six lo planes, the same 48 bytes per point as FP64); D is
// split once per CTA; u (double) is split with integer operations (no FP64
// conversion), and each output is rebuilt as double(hi) + double(lo).
#pragma once

#include "sem_ax.cuh"

namespace sem {

struct dfl {
    float h, l;
};

// hi/lo split of a double with integer operations: hi = the double truncated
// to 24 significant bits, lo = the next 24 bits rounded to float.  Exact to
// ~2^-48 relative for |x| in [2^-90, 2^127]; smaller magnitudes become 0.
__device__ __forceinline__ dfl split_double(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
    const unsigned ed = (hi32 >> 20) & 0x7ffu;  // biased FP64 exponent
    const unsigned sign = hi32 & 0x80000000u;
    // top 23 mantissa bits, exponent rebiased 1023 -> 127 (low 8 bits of
    // ed - 896 = low 8 bits of ed with bit 7 flipped)
    const unsigned t = __funnelshift_l(lo32, hi32, 3);
    const unsigned hb = ((t & 0x7fffffffu) ^ 0x40000000u) | sign;
    // remaining 29 mantissa bits, scaled by 2^(ed - 1075)
    const unsigned rem = lo32 & 0x1fffffffu;
    const float lo_mag = __uint2float_rn(rem) * __uint_as_float((ed - 948u) << 23);
    const bool ok = ed > 948u && ed < 1151u;
    dfl r;
    r.h = ok ? __uint_as_float(hb) : 0.0f;
    r.l = ok ? __uint_as_float(__float_as_uint(lo_mag) | sign) : 0.0f;
    return r;
}

// Exact float -> double by bit manipulation (integer pipe; a conversion
// instruction would run on the FP64 pipe, 1/64 of the FP32 rate on GB300).
// Zeros and subnormal floats give a signed zero, Inf/NaN stay Inf/NaN.
__device__ __forceinline__ double float_to_double_bits(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u, e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    unsigned hi, lo;
    if (e == 0u) {
        hi = sign;
        lo = 0u;
    } else {
        hi = sign | ((e == 0xffu ? 0x7ffu : e + 896u) << 20) | (m >> 3);
        lo = m << 29;
    }
    return __hiloint2double((int)hi, (int)lo);
}

// pair -> double: two exact conversions and one FP64 addition
__device__ __forceinline__ double join(dfl a) { return float_to_double_bits(a.h) + float_to_double_bits(a.l); }

// acc += a * b with a, b pairs; (S, E) is an unnormalised running pair.
__device__ __forceinline__ void df_mac(float& S, float& E, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float s = S + p;
    const float bb = s - S;
    const float err = (S - (s - bb)) + (p - bb);
    S = s;
    E += err + e;
}

// (S, E) = a * b as an unnormalised pair: the first term of an accumulation
// (the TwoSum of df_mac against a zero pair would be exact and is skipped)
__device__ __forceinline__ void df_mul(float& S, float& E, float ah, float al, float bh, float bl) {
    S = ah * bh;
    float e = fmaf(ah, bh, -S);
    e = fmaf(ah, bl, e);
    E = fmaf(al, bh, e);
}

__device__ __forceinline__ dfl df_norm(float S, float E) {
    dfl r;
    r.h = S + E;
    r.l = E - (r.h - S);
    return r;
}

template <int LX>
struct DfCfg {
    static constexpr int N2 = LX * LX, N3 = LX * LX * LX, DP = LX + 1;
    static constexpr int EPC = (256 / N2) > 0 ? (256 / N2) : 1;
    static constexpr int USED = EPC * N2;
    static constexpr int THREADS = ((USED + 31) / 32) * 32;
    // floats: D hi/lo (padded rows), then u, wr, ws hi and lo per element slot
    static constexpr size_t FLOATS = 2 * (size_t)LX * DP + 6 * (size_t)EPC * N3;
};

// Gs: [E][12][lx^3] floats (hi planes 0..5, lo planes 6..11); D2: [2][lx][lx]
// (hi then lo).  Same parameters as AxParams<double> otherwise.
struct DfParams {
    const double* u;
    const double* z;
    double* p;
    double* w;
    const float* G2;
    const float* D2;
    int64_t E;
    CGState* st;
    double* partials;
    unsigned int* counter;
    int dry;
};

template <int LX, bool FUSED>
__global__ void __launch_bounds__(DfCfg<LX>::THREADS) ax_df_kernel(DfParams a) {
    using C = DfCfg<LX>;
    constexpr int N2 = C::N2, N3 = C::N3, EPC = C::EPC, DP = C::DP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* sDh = reinterpret_cast<float*>(smem_raw);
    float* sDl = sDh + LX * DP;
    float* suh = sDl + LX * DP;
    float* sul = suh + EPC * N3;
    float* srh = sul + EPC * N3;
    float* srl = srh + EPC * N3;
    float* ssh = srl + EPC * N3;
    float* ssl = ssh + EPC * N3;

    double beta = 0.0;
    bool first = false;
    if (FUSED) {
        if (a.st->done) return;
        beta = cg_beta(a.st);
        first = cg_first(a.st);
    }
    for (int t = threadIdx.x; t < LX * LX; t += blockDim.x) {
        sDh[(t / LX) * DP + (t % LX)] = a.D2[t];
        sDl[(t / LX) * DP + (t % LX)] = a.D2[LX * LX + t];
    }
    const AxThread<LX> th;
    const int so = th.so, ij = th.ij, i = th.i, j = th.j;
    const int64_t ngroups = (a.E + EPC - 1) / EPC;
    double pap = 0.0;
    __syncthreads();
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const int64_t e = g * EPC + th.el;
        const bool valid = th.active && e < a.E;
        const int64_t base = e * N3 + ij;
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
        float uh[LX], ul[LX];
#pragma unroll
        for (int k = 0; k < LX; k++) {
            const dfl v = split_double(ud[k]);
            uh[k] = v.h;
            ul[k] = v.l;
            if (th.active) {
                suh[so + k * N2 + ij] = v.h;
                sul[so + k * N2 + ij] = v.l;
            }
        }
        __syncthreads();
        const float* Ge = a.G2 + e * 12 * N3 + ij;
        float wth[LX], wtl[LX];
#pragma unroll
        for (int k = 0; k < LX; k++) {
            float rS, rE, sS, sE, tS, tE;
#pragma unroll
            for (int l = 0; l < LX; l++) {
                const int qr = so + k * N2 + j * LX + l, qs = so + k * N2 + l * LX + i;
                if (l == 0) {
                    df_mul(rS, rE, sDh[i * DP], sDl[i * DP], suh[qr], sul[qr]);
                    df_mul(sS, sE, sDh[j * DP], sDl[j * DP], suh[qs], sul[qs]);
                    df_mul(tS, tE, sDh[k * DP], sDl[k * DP], uh[0], ul[0]);
                } else {
                    df_mac(rS, rE, sDh[i * DP + l], sDl[i * DP + l], suh[qr], sul[qr]);
                    df_mac(sS, sE, sDh[j * DP + l], sDl[j * DP + l], suh[qs], sul[qs]);
                    df_mac(tS, tE, sDh[k * DP + l], sDl[k * DP + l], uh[l], ul[l]);
                }
            }
            const dfl ur = df_norm(rS, rE), us = df_norm(sS, sE), ut = df_norm(tS, tE);
            float gh[6], gl[6];
#pragma unroll
            for (int c = 0; c < 6; c++) {
                gh[c] = valid ? ld_stream(Ge + c * N3 + k * N2) : 0.f;
                gl[c] = valid ? ld_stream(Ge + (6 + c) * N3 + k * N2) : 0.f;
            }
            float aS, aE, bS, bE, cS, cE;
            // (wr, ws, wt) = G (ur, us, ut), G = [[11 12 13] [12 22 23] [13 23 33]]
            df_mul(aS, aE, gh[0], gl[0], ur.h, ur.l);
            df_mac(aS, aE, gh[1], gl[1], us.h, us.l);
            df_mac(aS, aE, gh[2], gl[2], ut.h, ut.l);
            df_mul(bS, bE, gh[1], gl[1], ur.h, ur.l);
            df_mac(bS, bE, gh[3], gl[3], us.h, us.l);
            df_mac(bS, bE, gh[4], gl[4], ut.h, ut.l);
            df_mul(cS, cE, gh[2], gl[2], ur.h, ur.l);
            df_mac(cS, cE, gh[4], gl[4], us.h, us.l);
            df_mac(cS, cE, gh[5], gl[5], ut.h, ut.l);
            const dfl wr = df_norm(aS, aE), ws = df_norm(bS, bE), wt = df_norm(cS, cE);
            wth[k] = wt.h;
            wtl[k] = wt.l;
            if (th.active) {
                srh[so + k * N2 + ij] = wr.h;
                srl[so + k * N2 + ij] = wr.l;
                ssh[so + k * N2 + ij] = ws.h;
                ssl[so + k * N2 + ij] = ws.l;
            }
        }
        __syncthreads();
        double pw = 0.0;
#pragma unroll
        for (int k = 0; k < LX; k++) {
            float S = 0.f, E = 0.f;
#pragma unroll
            for (int l = 0; l < LX; l++) {
                const int qr = so + k * N2 + j * LX + l, qs = so + k * N2 + l * LX + i;
                if (l == 0) df_mul(S, E, sDh[i], sDl[i], srh[qr], srl[qr]);
                else df_mac(S, E, sDh[l * DP + i], sDl[l * DP + i], srh[qr], srl[qr]);
                df_mac(S, E, sDh[l * DP + j], sDl[l * DP + j], ssh[qs], ssl[qs]);
                df_mac(S, E, sDh[l * DP + k], sDl[l * DP + k], wth[l], wtl[l]);
            }
            const double wv = join(df_norm(S, E));
            if (valid) {
                st_keep<FUSED>(a.w + base + k * N2, wv);
                if (FUSED) pw = fma(ud[k], wv, pw);
            }
        }
        if (FUSED) pap += pw;
        __syncthreads();
    }
    if (FUSED) {
        double v[1] = {pap};
        CGState* st = a.st;
        grid_sum_finalize<1>(v, a.partials, a.counter, [&](double (&acc)[1]) { cg_set_alpha(st, acc[0]); });
    }
}

template <int LX, bool FUSED>
inline int launch_ax_df_t(sem_handle* h, const DfParams& a, cudaStream_t s) {
    using C = DfCfg<LX>;
    constexpr size_t smem = C::FLOATS * sizeof(float);
    static int per_sm = -1;
    if (per_sm < 0) {
        cudaFuncSetAttribute(ax_df_kernel<LX, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ax_df_kernel<LX, FUSED>, C::THREADS, smem);
        per_sm = nb > 0 ? nb : 1;
    }
    if (a.dry) return SEM_OK;
    const int64_t ngroups = (a.E + C::EPC - 1) / C::EPC;
    int64_t grid = std::min<int64_t>(ngroups, (int64_t)h->sm_count * per_sm);
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, kMaxPartials));
    ax_df_kernel<LX, FUSED><<<(int)grid, C::THREADS, smem, s>>>(a);
    SEM_LAUNCH_CHECK("ax_df_kernel");
    h->launches++;
    return SEM_OK;
}

template <bool FUSED>
inline int dispatch_ax_df(sem_handle* h, int lx, const DfParams& a, cudaStream_t s) {
    switch (lx) {
        case 2: return launch_ax_df_t<2, FUSED>(h, a, s);
        case 3: return launch_ax_df_t<3, FUSED>(h, a, s);
        case 4: return launch_ax_df_t<4, FUSED>(h, a, s);
        case 5: return launch_ax_df_t<5, FUSED>(h, a, s);
        case 6: return launch_ax_df_t<6, FUSED>(h, a, s);
        case 7: return launch_ax_df_t<7, FUSED>(h, a, s);
        case 8: return launch_ax_df_t<8, FUSED>(h, a, s);
        case 9: return launch_ax_df_t<9, FUSED>(h, a, s);
        case 10: return launch_ax_df_t<10, FUSED>(h, a, s);
        case 11: return launch_ax_df_t<11, FUSED>(h, a, s);
        case 12: return launch_ax_df_t<12, FUSED>(h, a, s);
        default: return fail(SEM_EINVAL, "FP32-pair operator supports lx <= 12");
    }
}

int dispatch_ax_df_entry(sem_handle* h, int lx, const DfParams& a, bool fused, cudaStream_t s);

// ---------------------------------------------------------------------------
// Line-transform form of the FP32-pair operator (even lx).  D and D^T are
// centro-antisymmetric (M_{N-i,N-l} = -M_il), so with the even and odd parts
// e_m = x_m + x_{N-m}, o_m = x_m - x_{N-m} of a line x (m < lx/2):
//   y_i     = sum_m A_im o_m + sum_m B_im e_m,
//   y_{N-i} = sum_m A_im o_m - sum_m B_im e_m,
// with A_im = (M_im - M_{i,N-m}) / 2, B_im = (M_im + M_{i,N-m}) / 2:
// (lx/2)^2 * 2 products per line instead of lx^2.  A thread owns one line
// in each direction: r-lines (k, j), s-lines (k, i), t-lines (j, i).
// ---------------------------------------------------------------------------

// a + b (sign +1) or a - b (sign -1) of unnormalised pairs, unnormalised result
__device__ __forceinline__ void pair_addsub(float ah, float al, float bh, float bl, float sign, float& h, float& l) {
    const float b = sign * bh;
    const float s = ah + b;
    const float bb = s - ah;
    const float err = (ah - (s - bb)) + (b - bb);
    h = s;
    l = err + (al + sign * bl);
}

// Coefficient tables of the line transforms for every even order, in the
// constant bank: the unrolled transforms read them as immediate constant
// operands of the FP32 multiplies (no shared-memory loads).  Layout per order:
// [dir][A/B][hi/lo][P][P] (dir 0 = D, 1 = D^T), at dfl_coef_off(lx).
constexpr int dfl_coef_off(int lx) {
    return lx == 4 ? 0 : lx == 6 ? 32 : lx == 8 ? 104 : lx == 10 ? 232 : lx == 12 ? 432 : -1;
}
constexpr int kDflCoefTotal = 720;
static __constant__ float c_dflcoef[kDflCoefTotal];
int dfl_set_coef(const float* cf, int lx);

template <int LX>
struct DflCfg {
    static constexpr int P = LX / 2;
    static constexpr int N2 = LX * LX, N3 = LX * LX * LX;
    // padded row and plane strides, chosen (by an offline search over the
    // column, r-, s- and t-line access patterns of a warp) so that no access
    // has more than a 2-way shared-memory bank conflict
    static constexpr int LXP = LX == 4 ? 5 : LX == 6 ? 7 : LX == 8 ? 9 : LX == 10 ? 11 : LX == 12 ? 17 : LX + 1;
    static constexpr int N2P = LX == 4 ? 20 : LX == 6 ? 42 : LX == 8 ? 72 : LX == 10 ? 111 : LX == 12 ? 204 : LX * LXP + 1;
    static constexpr int SLOT = LX * N2P;        // floats per element per array
    static constexpr int EPC = (256 / N2) > 0 ? (256 / N2) : 1;
    static constexpr int USED = EPC * N2;
    static constexpr int THREADS = ((USED + 31) / 32) * 32;
    // coefficient tables: [fwd/bwd][A/B][hi/lo][P][P]
    static constexpr int COEF = 2 * 2 * 2 * P * P;
    static constexpr size_t FLOATS = 8 * (size_t)EPC * SLOT;
    static __host__ __device__ constexpr int at(int k, int j, int i) { return k * N2P + j * LXP + i; }
};

// One line: x at xs[0], xs[st], ..., y written to ys[0], ys[st], ... (both
// hi and lo arrays); coefficient tables A, B (hi, lo) of size P x P.
// CA: constant-bank offset of the A (hi) table; A lo, B hi, B lo follow at P*P strides.
template <int LX, int CA>
__device__ __forceinline__ void df_line(const float* xh, const float* xl, int xst, float* yh, float* yl, int yst) {
    constexpr int P = LX / 2, N = LX - 1, PP = P * P;
    const float* Ah = c_dflcoef + CA;
    const float* Al = c_dflcoef + CA + PP;
    const float* Bh = c_dflcoef + CA + 2 * PP;
    const float* Bl = c_dflcoef + CA + 3 * PP;
    float eh[P], el[P], oh[P], ol[P];
#pragma unroll
    for (int m = 0; m < P; m++) {
        const float ah = xh[m * xst], al = xl[m * xst], bh = xh[(N - m) * xst], bl = xl[(N - m) * xst];
        pair_addsub(ah, al, bh, bl, 1.0f, eh[m], el[m]);
        pair_addsub(ah, al, bh, bl, -1.0f, oh[m], ol[m]);
    }
#pragma unroll
    for (int i = 0; i < P; i++) {
        float sS, sE, tS, tE;
        df_mul(sS, sE, Ah[i * P], Al[i * P], oh[0], ol[0]);
        df_mul(tS, tE, Bh[i * P], Bl[i * P], eh[0], el[0]);
#pragma unroll
        for (int m = 1; m < P; m++) {
            df_mac(sS, sE, Ah[i * P + m], Al[i * P + m], oh[m], ol[m]);
            df_mac(tS, tE, Bh[i * P + m], Bl[i * P + m], eh[m], el[m]);
        }
        float h, l;
        pair_addsub(sS, sE, tS, tE, 1.0f, h, l);
        dfl y = df_norm(h, l);
        yh[i * yst] = y.h;
        yl[i * yst] = y.l;
        pair_addsub(sS, sE, tS, tE, -1.0f, h, l);
        y = df_norm(h, l);
        yh[(N - i) * yst] = y.h;
        yl[(N - i) * yst] = y.l;
    }
}

// Same, accumulating into y (y += M x).
template <int LX, int CA>
__device__ __forceinline__ void df_line_acc(const float* xh, const float* xl, int xst, float* yh, float* yl, int yst) {
    constexpr int P = LX / 2, N = LX - 1, PP = P * P;
    const float* Ah = c_dflcoef + CA;
    const float* Al = c_dflcoef + CA + PP;
    const float* Bh = c_dflcoef + CA + 2 * PP;
    const float* Bl = c_dflcoef + CA + 3 * PP;
    float eh[P], el[P], oh[P], ol[P];
#pragma unroll
    for (int m = 0; m < P; m++) {
        const float ah = xh[m * xst], al = xl[m * xst], bh = xh[(N - m) * xst], bl = xl[(N - m) * xst];
        pair_addsub(ah, al, bh, bl, 1.0f, eh[m], el[m]);
        pair_addsub(ah, al, bh, bl, -1.0f, oh[m], ol[m]);
    }
#pragma unroll
    for (int i = 0; i < P; i++) {
        float sS, sE, tS, tE;
        df_mul(sS, sE, Ah[i * P], Al[i * P], oh[0], ol[0]);
        df_mul(tS, tE, Bh[i * P], Bl[i * P], eh[0], el[0]);
#pragma unroll
        for (int m = 1; m < P; m++) {
            df_mac(sS, sE, Ah[i * P + m], Al[i * P + m], oh[m], ol[m]);
            df_mac(tS, tE, Bh[i * P + m], Bl[i * P + m], eh[m], el[m]);
        }
        float h, l, h2, l2;
        pair_addsub(sS, sE, tS, tE, 1.0f, h, l);
        pair_addsub(yh[i * yst], yl[i * yst], h, l, 1.0f, h2, l2);
        dfl y = df_norm(h2, l2);
        yh[i * yst] = y.h;
        yl[i * yst] = y.l;
        pair_addsub(sS, sE, tS, tE, -1.0f, h, l);
        pair_addsub(yh[(N - i) * yst], yl[(N - i) * yst], h, l, 1.0f, h2, l2);
        y = df_norm(h2, l2);
        yh[(N - i) * yst] = y.h;
        yl[(N - i) * yst] = y.l;
    }
}

struct DflParams {
    const double* u;
    const double* z;
    double* p;
    double* w;
    // pair form of the CG vectors (fused kernel with PAIR): hi and lo planes
    const float* zh;
    const float* zl;
    float* ph;
    float* pl;
    float* wh;
    float* wl;
    const float* G2;
    int64_t E;
    CGState* st;
    double* partials;
    unsigned int* counter;
    int dry;
    // batched form: element-group list of one order, per-solve states and
    // partials (see BatchAxParams)
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

template <int LX, bool FUSED, bool PAIR = false, bool BATCH = false>
__global__ void __launch_bounds__(DflCfg<LX>::THREADS) ax_dfl_kernel(DflParams a) {
    static_assert(!PAIR || FUSED, "the pair form exists for the fused CG kernel only");
    static_assert(!(PAIR && BATCH), "no pair form for batches");
    using C = DflCfg<LX>;
    constexpr int P = C::P, N2 = C::N2, N3 = C::N3, EPC = C::EPC, SLOT = C::SLOT;
    constexpr int N2P = C::N2P, LXP = C::LXP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* arr = reinterpret_cast<float*>(smem_raw);  // 8 arrays x EPC slots: uh ul | rh rl | sh sl | th tl
    constexpr int CF = dfl_coef_off(LX), CB = CF + 4 * P * P;  // forward (D) and backward (D^T) tables
    double beta = 0.0;
    bool first = false;
    __shared__ double red[32];
    __shared__ int is_last;
    __shared__ double sb_beta;
    __shared__ int sb_done, sb_first;
    __shared__ float sb_b2[2];  // beta as a float pair (pair form)
    if (FUSED && !BATCH) {
        if (a.st->done) return;
        // beta divided (and split) once by thread 0: GB300's FP64 pipe is slow
        if (threadIdx.x == 0) {
            sb_beta = cg_beta(a.st);
            sb_b2[0] = (float)sb_beta;
            sb_b2[1] = (float)(sb_beta - (double)sb_b2[0]);
        }
        first = cg_first(a.st);
    }
    const int tid = threadIdx.x;
    const int el = tid / N2;
    const int t2 = tid - el * N2;          // column (i, j) in phase 0, line id in the transforms
    const int lo_ = t2 % LX, hi_ = t2 / LX;  // i / j of the column; also the line coordinates
    const bool active = el < EPC;
    const int slot = (active ? el : 0) * SLOT;
    float* uh = arr + 0 * EPC * SLOT + slot;
    float* ul = arr + 1 * EPC * SLOT + slot;
    float* rh = arr + 2 * EPC * SLOT + slot;
    float* rl = arr + 3 * EPC * SLOT + slot;
    float* sh = arr + 4 * EPC * SLOT + slot;
    float* sl = arr + 5 * EPC * SLOT + slot;
    float* th = arr + 6 * EPC * SLOT + slot;
    float* tl = arr + 7 * EPC * SLOT + slot;
    const int64_t ngroups = BATCH ? a.ngroups : (a.E + EPC - 1) / EPC;
    double pap = 0.0;
    float paph = 0.f, papl = 0.f;  // pair form: <p, A p> as a float pair (no FP64 per group)
    __syncthreads();
    dfl b2 = {0.f, 0.f};
    if (FUSED && !BATCH) {
        beta = sb_beta;
        b2.h = sb_b2[0];
        b2.l = sb_b2[1];
    }
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        int64_t eoff;  // local index of this thread's element
        bool valid;
        int sol = 0;
        if (BATCH) {
            sol = a.solve[g];
            if (FUSED) {
                // the solve's scalars, read and divided once per group by thread 0
                if (threadIdx.x == 0) {
                    const CGState* stg = a.st + sol;
                    // no write to this solve's state can happen before all its groups are done
                    sb_done = stg->done;
                    sb_beta = sb_done ? 0.0 : cg_beta(stg);
                    sb_first = cg_first(stg);
                }
                __syncthreads();
                if (sb_done) {
                    __syncthreads();  // thread 0 rewrites the scalars next round
                    continue;
                }
                beta = sb_beta;
                first = sb_first != 0;
            }
            eoff = a.loc[g] + (int64_t)el * N3;
            valid = active && el < a.cnt[g];
        } else {
            const int64_t e = g * EPC + el;
            eoff = e * N3;
            valid = active && e < a.E;
        }
        const int64_t base = eoff + t2;  // column (i = lo_, j = hi_)
        // phase 0: column of u (or z + beta p), split into pairs
        double ud[LX];
        float cuh[LX], cul[LX];  // the column of u as pairs (PAIR form)
        if (PAIR) {
#pragma unroll
            for (int k = 0; k < LX; k++) {
                float S = valid ? ld_stream(a.zh + base + k * N2) : 0.f;
                float Ee = valid ? ld_stream(a.zl + base + k * N2) : 0.f;
                if (valid && !first) df_mac(S, Ee, b2.h, b2.l, a.ph[base + k * N2], a.pl[base + k * N2]);
                const dfl v = df_norm(S, Ee);
                cuh[k] = v.h;
                cul[k] = v.l;
            }
            if (valid) {
#pragma unroll
                for (int k = 0; k < LX; k++) {
                    a.ph[base + k * N2] = cuh[k];
                    a.pl[base + k * N2] = cul[k];
                }
            }
            if (active) {
#pragma unroll
                for (int k = 0; k < LX; k++) {
                    uh[C::at(k, hi_, lo_)] = cuh[k];
                    ul[C::at(k, hi_, lo_)] = cul[k];
                }
            }
        } else {
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
            for (int k = 0; k < LX; k++) {
                const dfl v = split_double(ud[k]);
                uh[C::at(k, hi_, lo_)] = v.h;
                ul[C::at(k, hi_, lo_)] = v.l;
            }
        }
        }
        // factors of the column's first point, requested now and used after phase 1
        const float* Ge = a.G2 + 12 * eoff + t2;
        float g0h[6], g0l[6];
#pragma unroll
        for (int c = 0; c < 6; c++) {
            g0h[c] = (active && valid) ? ld_stream(Ge + c * N3) : 0.f;
            g0l[c] = (active && valid) ? ld_stream(Ge + (6 + c) * N3) : 0.f;
        }
        __syncthreads();
        // phase 1: derivative lines ur (along i), us (along j), ut (along k)
        if (active) {
            df_line<LX, CF>(uh + C::at(hi_, lo_, 0), ul + C::at(hi_, lo_, 0), 1, rh + C::at(hi_, lo_, 0),
                        rl + C::at(hi_, lo_, 0), 1);  // r-line (k=hi_, j=lo_)
            df_line<LX, CF>(uh + C::at(hi_, 0, lo_), ul + C::at(hi_, 0, lo_), LXP, sh + C::at(hi_, 0, lo_),
                        sl + C::at(hi_, 0, lo_), LXP);  // s-line (k=hi_, i=lo_)
            df_line<LX, CF>(uh + C::at(0, hi_, lo_), ul + C::at(0, hi_, lo_), N2P, th + C::at(0, hi_, lo_),
                        tl + C::at(0, hi_, lo_), N2P);  // t-line (j=hi_, i=lo_)
        }
        __syncthreads();
        // phase 2: (wr, ws, wt) = G (ur, us, ut) at the column's points; the
        // factors of point k + 1 are loaded while point k is computed (those of
        // point 0 were requested before phase 1)
        if (active) {
            float gh[6], gl[6];
#pragma unroll
            for (int c = 0; c < 6; c++) {
                gh[c] = g0h[c];
                gl[c] = g0l[c];
            }
#pragma unroll
            for (int k = 0; k < LX; k++) {
                const int q = C::at(k, hi_, lo_);
                float nh[6], nl[6];
                if (k + 1 < LX) {
#pragma unroll
                    for (int c = 0; c < 6; c++) {
                        nh[c] = valid ? ld_stream(Ge + c * N3 + (k + 1) * N2) : 0.f;
                        nl[c] = valid ? ld_stream(Ge + (6 + c) * N3 + (k + 1) * N2) : 0.f;
                    }
                }
                const float urh = rh[q], url = rl[q], ush = sh[q], usl = sl[q], uth = th[q], utl = tl[q];
                float aS, aE, bS, bE, cS, cE;
                df_mul(aS, aE, gh[0], gl[0], urh, url);
                df_mac(aS, aE, gh[1], gl[1], ush, usl);
                df_mac(aS, aE, gh[2], gl[2], uth, utl);
                df_mul(bS, bE, gh[1], gl[1], urh, url);
                df_mac(bS, bE, gh[3], gl[3], ush, usl);
                df_mac(bS, bE, gh[4], gl[4], uth, utl);
                df_mul(cS, cE, gh[2], gl[2], urh, url);
                df_mac(cS, cE, gh[4], gl[4], ush, usl);
                df_mac(cS, cE, gh[5], gl[5], uth, utl);
                dfl v = df_norm(aS, aE);
                rh[q] = v.h;
                rl[q] = v.l;
                v = df_norm(bS, bE);
                sh[q] = v.h;
                sl[q] = v.l;
                v = df_norm(cS, cE);
                th[q] = v.h;
                tl[q] = v.l;
                if (k + 1 < LX) {
#pragma unroll
                    for (int c = 0; c < 6; c++) {
                        gh[c] = nh[c];
                        gl[c] = nl[c];
                    }
                }
            }
        }
        __syncthreads();
        // phase 3: w = D^T-lines of wr (into the u arrays), then += those of ws
        if (active)
            df_line<LX, CB>(rh + C::at(hi_, lo_, 0), rl + C::at(hi_, lo_, 0), 1, uh + C::at(hi_, lo_, 0),
                        ul + C::at(hi_, lo_, 0), 1);
        __syncthreads();
        if (active)
            df_line_acc<LX, CB>(sh + C::at(hi_, 0, lo_), sl + C::at(hi_, 0, lo_), LXP, uh + C::at(hi_, 0, lo_),
                            ul + C::at(hi_, 0, lo_), LXP);
        __syncthreads();
        // phase 4: += D^T-lines of wt along k; the t-line is this thread's column
        if (active)
            df_line_acc<LX, CB>(th + C::at(0, hi_, lo_), tl + C::at(0, hi_, lo_), N2P, uh + C::at(0, hi_, lo_),
                            ul + C::at(0, hi_, lo_), N2P);
        double pw = 0.0;
        if (PAIR) {
            float S = 0.f, Ee = 0.f;
            if (valid) {
#pragma unroll
                for (int k = 0; k < LX; k++) {
                    const int q = C::at(k, hi_, lo_);
                    const float wvh = uh[q], wvl = ul[q];
                    st_keep<true>(a.wh + base + k * N2, wvh);
                    st_keep<true>(a.wl + base + k * N2, wvl);
                    if (k == 0) df_mul(S, Ee, cuh[0], cul[0], wvh, wvl);
                    else df_mac(S, Ee, cuh[k], cul[k], wvh, wvl);
                }
            }
            if (!BATCH) fpair_add2(paph, papl, S, Ee);
            else pw = (double)S + (double)Ee;
        } else if (valid) {
#pragma unroll
            for (int k = 0; k < LX; k++) {
                const int q = C::at(k, hi_, lo_);
                const double wv = float_to_double_bits(uh[q]) + float_to_double_bits(ul[q]);
                st_keep<FUSED>(a.w + base + k * N2, wv);
                if (FUSED) pw = fma(ud[k], wv, pw);
            }
        }
        if (FUSED && BATCH) {
            double v[1] = {pw};
            block_sum<1>(v, red);
            if (threadIdx.x == 0) {
                a.gpart[a.goff + g] = v[0];
                __threadfence();
                is_last = (atomicAdd(&a.scount[sol], 1u) == (unsigned)a.sgcount[sol] - 1u) ? 1 : 0;
            }
            __syncthreads();
            if (is_last) {
                __threadfence();
                const int f = a.sgfirst[sol], c = a.sgcount[sol];
                double acc[1] = {0.0};
                for (int q = threadIdx.x; q < c; q += blockDim.x) acc[0] += __ldcg(&a.gpart[f + q]);
                block_sum<1>(acc, red);
                if (threadIdx.x == 0) {
                    cg_set_alpha(a.st + sol, acc[0]);
                    a.scount[sol] = 0u;
                }
            }
        } else if (FUSED && !PAIR) {
            pap += pw;
        }
        __syncthreads();
    }
    if (FUSED && !BATCH) {
        CGState* st = a.st;
        if constexpr (PAIR) {
            float h[1] = {paph}, l[1] = {papl};
            grid_sum_finalize_pair<1>(h, l, a.partials, a.counter,
                                      [&](double (&acc)[1]) { cg_set_alpha(st, acc[0]); });
        } else {
            double v[1] = {pap};
            grid_sum_finalize<1>(v, a.partials, a.counter, [&](double (&acc)[1]) { cg_set_alpha(st, acc[0]); });
        }
    }
}

template <int LX, bool FUSED, bool PAIR = false>
inline int launch_ax_dfl_t(sem_handle* h, const DflParams& a, cudaStream_t s) {
    using C = DflCfg<LX>;
    constexpr size_t smem = C::FLOATS * sizeof(float);
    static int per_sm = -1;
    if (per_sm < 0) {
        cudaFuncSetAttribute(ax_dfl_kernel<LX, FUSED, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ax_dfl_kernel<LX, FUSED, PAIR>, C::THREADS, smem);
        per_sm = nb > 0 ? nb : 1;
    }
    if (a.dry) return SEM_OK;
    const int64_t ngroups = (a.E + C::EPC - 1) / C::EPC;
    int64_t grid = std::min<int64_t>(ngroups, (int64_t)h->sm_count * per_sm);
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, kMaxPartials));
    ax_dfl_kernel<LX, FUSED, PAIR><<<(int)grid, C::THREADS, smem, s>>>(a);
    SEM_LAUNCH_CHECK("ax_dfl_kernel");
    h->launches++;
    return SEM_OK;
}

template <bool FUSED>
inline int dispatch_ax_dfl(sem_handle* h, int lx, const DflParams& a, cudaStream_t s) {
    switch (lx) {
        case 4: return launch_ax_dfl_t<4, FUSED>(h, a, s);
        case 6: return launch_ax_dfl_t<6, FUSED>(h, a, s);
        case 8: return launch_ax_dfl_t<8, FUSED>(h, a, s);
        case 10: return launch_ax_dfl_t<10, FUSED>(h, a, s);
        case 12: return launch_ax_dfl_t<12, FUSED>(h, a, s);
        default: return fail(SEM_EINVAL, "line-transform FP32-pair operator needs lx in {4, 6, 8, 10, 12}");
    }
}

template <int LX, bool FUSED>
inline int launch_ax_dfl_batch_t(sem_handle* h, const DflParams& a, cudaStream_t s) {
    using C = DflCfg<LX>;
    constexpr size_t smem = C::FLOATS * sizeof(float);
    static int per_sm = -1;
    if (per_sm < 0) {
        cudaFuncSetAttribute(ax_dfl_kernel<LX, FUSED, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ax_dfl_kernel<LX, FUSED, false, true>, C::THREADS, smem);
        per_sm = nb > 0 ? nb : 1;
    }
    if (a.dry || a.ngroups == 0) return SEM_OK;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(a.ngroups, (int64_t)h->sm_count * per_sm));
    ax_dfl_kernel<LX, FUSED, false, true><<<(int)grid, C::THREADS, smem, s>>>(a);
    SEM_LAUNCH_CHECK("ax_dfl_kernel (batched)");
    h->launches++;
    return SEM_OK;
}

template <bool FUSED>
inline int dispatch_ax_dfl_batch(sem_handle* h, int lx, const DflParams& a, cudaStream_t s) {
    switch (lx) {
        case 4: return launch_ax_dfl_batch_t<4, FUSED>(h, a, s);
        case 6: return launch_ax_dfl_batch_t<6, FUSED>(h, a, s);
        case 8: return launch_ax_dfl_batch_t<8, FUSED>(h, a, s);
        case 10: return launch_ax_dfl_batch_t<10, FUSED>(h, a, s);
        case 12: return launch_ax_dfl_batch_t<12, FUSED>(h, a, s);
        default: return fail(SEM_EINVAL, "batched line-transform operator needs lx in {4, 6, 8, 10, 12}");
    }
}

int dispatch_ax_dfl_batch_entry(sem_handle* h, int lx, const DflParams& a, bool fused, cudaStream_t s);

inline int dispatch_ax_dfl_pair(sem_handle* h, int lx, const DflParams& a, cudaStream_t s) {
    switch (lx) {
        case 4: return launch_ax_dfl_t<4, true, true>(h, a, s);
        case 6: return launch_ax_dfl_t<6, true, true>(h, a, s);
        case 8: return launch_ax_dfl_t<8, true, true>(h, a, s);
        case 10: return launch_ax_dfl_t<10, true, true>(h, a, s);
        case 12: return launch_ax_dfl_t<12, true, true>(h, a, s);
        default: return fail(SEM_EINVAL, "pair-form CG operator needs lx in {4, 6, 8, 10, 12}");
    }
}

int dispatch_ax_dfl_entry(sem_handle* h, int lx, const DflParams& a, bool fused, cudaStream_t s);
int dispatch_ax_dfl_pair_entry(sem_handle* h, int lx, const DflParams& a, cudaStream_t s);

}  // namespace sem
