// Split-precision tensor-core form of the local operator w = A_L u for FP32
// data and lx = 8 (Sec. II-A, eq. "disclap": A^e = D^T G^e D): the D and D^T
// contractions run as BF16 tensor-core products (warp-level mma.sync
// m16n8k16, FP32 accumulation), the G weighting on the FP32 pipe.
//
// BF16 keeps 8 significant bits, so u and D are each split into three BF16
// slices, x = x0 + x1 + x2, taken by successive round-to-nearest (exact for an
// FP32 value: every step removes at least 8 bits).  Of the nine slice
// products the six with combined weight >= 2^-16 are formed,
//   u0 D0 + u1 D0 + u0 D1 + u1 D1 + u2 D0 + u0 D2,
// two per mma (the K = 16 of an mma holds two K = 8 contractions), so each
// 16 x 8 output tile costs three mma and the dropped terms are below 2^-24 of
// |D||u|: the FP32 operator's accuracy class.  wr, ws, wt are split the same
// way for the transposed contractions.
//
// One warp owns one element at a time.  Its slices sit in shared memory in
// [k][j][i] planes with a padded k stride (72 BF16), so the 8 x 8 blocks of
// all three directions load conflict-free with ldmatrix: rows (k, j) for the
// r-contraction, and transposed blocks for the s- and t-contractions
// (ldmatrix .trans).  The outputs of the three directions land in different
// (row, column) layouts; they meet in a padded FP32 point buffer, where the
// G weighting and the final sum read them point by point.
#include <cuda_bf16.h>

#include "sem_ax.cuh"

namespace sem {

constexpr int kTcWarps = 4;                       // elements (warps) per CTA
constexpr int kTcPlane = 8 * 72;                  // BF16 entries of one slice plane
constexpr int kTcFPlane = 8 * 68;                 // FP32 entries of one point-buffer plane
constexpr int kTcWarpBytes = 9 * kTcPlane * 2 + 3 * kTcFPlane * 4;  // 10368 + 6528 bytes

__device__ __forceinline__ int tc_bidx(int k, int j, int i) { return k * 72 + j * 8 + i; }
__device__ __forceinline__ int tc_fidx(int k, int j, int i) { return k * 68 + j * 8 + i; }

// x = x0 + x1 + x2 in BF16 (round-to-nearest at every step; exact for FP32 x)
__device__ __forceinline__ void split3(float x, __nv_bfloat16& h0, __nv_bfloat16& h1, __nv_bfloat16& h2) {
    h0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h0);
    h1 = __float2bfloat16_rn(r1);
    h2 = __float2bfloat16_rn(r1 - __bfloat162float(h1));
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t (&r)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

// d += A (16 x 16, row) * B (16 x 8, col), BF16 in, FP32 accumulate
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// B fragments of the six slice products for one contraction direction:
// pairs (A slices | B slices) = ([0|1], [0;0]), ([0|1], [1;1]), ([2|0], [0;2])
struct TcB {
    uint32_t b[3][2];
};

// One 16-row tile of a contraction: A rows from the slice planes p0, p1, p2
// (shared addresses of the row starts this lane feeds to ldmatrix for the
// halves K = 0..7 and 8..15), B fragments in bf; result in c.
template <bool TRANS>
__device__ __forceinline__ void tc_tile(uint32_t a0_lo, uint32_t a0_hi, uint32_t a2_lo, uint32_t a2_hi,
                                        const TcB& bf, float (&c)[4], int lane) {
    // lanes 0-15 address the K = 0..7 half, 16-31 the K = 8..15 half
    uint32_t A01[4], A20[4];
    const uint32_t addr01 = lane < 16 ? a0_lo : a0_hi;  // [u0 | u1]
    const uint32_t addr20 = lane < 16 ? a2_lo : a2_hi;  // [u2 | u0]
    if (TRANS) {
        ldsm_x4_t(addr01, A01);
        ldsm_x4_t(addr20, A20);
    } else {
        ldsm_x4(addr01, A01);
        ldsm_x4(addr20, A20);
    }
    c[0] = c[1] = c[2] = c[3] = 0.0f;
    mma_bf16(c, A01, bf.b[0][0], bf.b[0][1]);
    mma_bf16(c, A01, bf.b[1][0], bf.b[1][1]);
    mma_bf16(c, A20, bf.b[2][0], bf.b[2][1]);
}

// The three contractions of one element, the r-, s- and t-directions reading
// the slice planes at pr, ps, pt (three planes each, shared addresses).
// sum_into_fr = false: the three results go to the point buffers fr, fs, ft;
// true (transposed contractions): they are summed into fr.
__device__ __forceinline__ void tc_contract(uint32_t pr, uint32_t ps, uint32_t pt, const TcB& bf, float* fr,
                                            float* fs, float* ft, bool sum_into_fr, int lane) {
    const int g = lane >> 2, t = lane & 3;
    const int mi = (lane >> 3) & 1, r = lane & 7;
    constexpr uint32_t P = kTcPlane * 2;  // bytes per slice plane
    // t-direction: A[(j, i)][l] = x[l][j][i]
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int j = 2 * q + mi;
        const uint32_t off = (uint32_t)tc_bidx(r, j, 0) * 2;
        float c[4];
        tc_tile<true>(pt + off, pt + P + off, pt + 2 * P + off, pt + off, bf, c, lane);
        const int ka = 2 * t, kb = 2 * t + 1;
        float* f = sum_into_fr ? fr : ft;
        f[tc_fidx(ka, 2 * q, g)] = c[0];
        f[tc_fidx(kb, 2 * q, g)] = c[1];
        f[tc_fidx(ka, 2 * q + 1, g)] = c[2];
        f[tc_fidx(kb, 2 * q + 1, g)] = c[3];
    }
    if (sum_into_fr) __syncwarp();
    // s-direction: A[(k, i)][l] = x[k][l][i]
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int k = 2 * q + mi;
        const uint32_t off = (uint32_t)tc_bidx(k, r, 0) * 2;
        float c[4];
        tc_tile<true>(ps + off, ps + P + off, ps + 2 * P + off, ps + off, bf, c, lane);
        const int ja = 2 * t, jb = 2 * t + 1;
        if (sum_into_fr) {
            fr[tc_fidx(2 * q, ja, g)] += c[0];
            fr[tc_fidx(2 * q, jb, g)] += c[1];
            fr[tc_fidx(2 * q + 1, ja, g)] += c[2];
            fr[tc_fidx(2 * q + 1, jb, g)] += c[3];
        } else {
            fs[tc_fidx(2 * q, ja, g)] = c[0];
            fs[tc_fidx(2 * q, jb, g)] = c[1];
            fs[tc_fidx(2 * q + 1, ja, g)] = c[2];
            fs[tc_fidx(2 * q + 1, jb, g)] = c[3];
        }
    }
    if (sum_into_fr) __syncwarp();
    // r-direction: A[(k, j)][l] = x[k][j][l]
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int R = 16 * q + 8 * mi + r;
        const uint32_t off = (uint32_t)tc_bidx(R >> 3, R & 7, 0) * 2;
        float c[4];
        tc_tile<false>(pr + off, pr + P + off, pr + 2 * P + off, pr + off, bf, c, lane);
        const int R0 = 16 * q + g, R1 = R0 + 8;
        float* f0 = fr + tc_fidx(R0 >> 3, R0 & 7, 2 * t);
        float* f1 = fr + tc_fidx(R1 >> 3, R1 & 7, 2 * t);
        if (sum_into_fr) {
            f0[0] += c[0];
            f0[1] += c[1];
            f1[0] += c[2];
            f1[1] += c[3];
        } else {
            f0[0] = c[0];
            f0[1] = c[1];
            f1[0] = c[2];
            f1[1] = c[3];
        }
    }
}

template <bool FUSED>
__global__ void __launch_bounds__(kTcWarps * 32) ax_tc_kernel(AxParams<float> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* wb = smem_raw + warp * kTcWarpBytes;
    __nv_bfloat16* sl = reinterpret_cast<__nv_bfloat16*>(wb);                  // 9 slice planes
    float* fb = reinterpret_cast<float*>(wb + 9 * kTcPlane * 2);              // 3 point buffers
    float* fr = fb;
    float* fs = fb + kTcFPlane;
    float* ft = fb + 2 * kTcFPlane;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sl);
    constexpr uint32_t P = kTcPlane * 2;
    __shared__ float s_tbeta;
    __shared__ int s_first;
    if (FUSED) {
        if (a.st->done) return;  // uniform over the grid
        if (threadIdx.x == 0) {
            s_tbeta = (float)cg_beta(a.st);
            s_first = cg_first(a.st) ? 1 : 0;
        }
        __syncthreads();
    }
    const float tbeta = FUSED ? s_tbeta : 0.0f;
    const bool first = FUSED ? (s_first != 0) : false;
    // B fragments: forward B[l][n] = D[n][l], transposed B[l][n] = D[l][n]
    const int g = lane >> 2, t = lane & 3;
    TcB bf, bb;
    {
        __nv_bfloat16 f[2][3], tt[2][3];
        for (int e = 0; e < 2; e++) {
            split3(a.D[g * 8 + 2 * t + e], f[e][0], f[e][1], f[e][2]);   // D[g][2t + e]
            split3(a.D[(2 * t + e) * 8 + g], tt[e][0], tt[e][1], tt[e][2]);  // D[2t + e][g]
        }
        // products ([0|1],[0;0]), ([0|1],[1;1]), ([2|0],[0;2])
        const int bs[3][2] = {{0, 0}, {1, 1}, {0, 2}};
        for (int p = 0; p < 3; p++) {
            bf.b[p][0] = pack_bf16(f[0][bs[p][0]], f[1][bs[p][0]]);
            bf.b[p][1] = pack_bf16(f[0][bs[p][1]], f[1][bs[p][1]]);
            bb.b[p][0] = pack_bf16(tt[0][bs[p][0]], tt[1][bs[p][0]]);
            bb.b[p][1] = pack_bf16(tt[0][bs[p][1]], tt[1][bs[p][1]]);
        }
    }
    float paph = 0.f, papl = 0.f;
    for (int64_t e = (int64_t)blockIdx.x * kTcWarps + warp; e < a.E; e += (int64_t)gridDim.x * kTcWarps) {
        const int64_t eb = e * 512;
        // 1. this lane's 16 points (p = lane + 32 m): u, or z + beta p in the CG
        float uv[16];
#pragma unroll
        for (int m = 0; m < 16; m++) {
            const int64_t L = eb + lane + 32 * m;
            if (FUSED) {
                const float zv = ld_stream(a.z + L);
                const float pv = first ? 0.0f : a.p[L];
                uv[m] = fmaf(tbeta, pv, zv);
            } else {
                uv[m] = ld_stream(a.u + L);
            }
        }
        if (FUSED)
#pragma unroll
            for (int m = 0; m < 16; m++) a.p[eb + lane + 32 * m] = uv[m];
        // 2. slices of u into planes 0..2
#pragma unroll
        for (int m = 0; m < 16; m++) {
            const int p = lane + 32 * m, k = p >> 6, j = (p >> 3) & 7, i = p & 7;
            __nv_bfloat16 h0, h1, h2;
            split3(uv[m], h0, h1, h2);
            sl[0 * kTcPlane + tc_bidx(k, j, i)] = h0;
            sl[1 * kTcPlane + tc_bidx(k, j, i)] = h1;
            sl[2 * kTcPlane + tc_bidx(k, j, i)] = h2;
        }
        __syncwarp();
        // 3. ur, us, ut
        tc_contract(sbase, sbase, sbase, bf, fr, fs, ft, false, lane);
        __syncwarp();
        // 4. weighting by the factors, slices of wr (planes 0..2), ws (3..5), wt (6..8)
        const float* Ge = a.G + e * 6 * 512;
#pragma unroll 4
        for (int m = 0; m < 16; m++) {
            const int p = lane + 32 * m, k = p >> 6, j = (p >> 3) & 7, i = p & 7;
            const int fi = tc_fidx(k, j, i);
            const float ur = fr[fi], us = fs[fi], ut = ft[fi];
            const float g11 = ld_stream(Ge + 0 * 512 + p), g12 = ld_stream(Ge + 1 * 512 + p);
            const float g13 = ld_stream(Ge + 2 * 512 + p), g22 = ld_stream(Ge + 3 * 512 + p);
            const float g23 = ld_stream(Ge + 4 * 512 + p), g33 = ld_stream(Ge + 5 * 512 + p);
            const float wr = fmaf(g11, ur, fmaf(g12, us, g13 * ut));
            const float ws = fmaf(g12, ur, fmaf(g22, us, g23 * ut));
            const float wt = fmaf(g13, ur, fmaf(g23, us, g33 * ut));
            const int bi = tc_bidx(k, j, i);
            __nv_bfloat16 h0, h1, h2;
            split3(wr, h0, h1, h2);
            sl[0 * kTcPlane + bi] = h0;
            sl[1 * kTcPlane + bi] = h1;
            sl[2 * kTcPlane + bi] = h2;
            split3(ws, h0, h1, h2);
            sl[3 * kTcPlane + bi] = h0;
            sl[4 * kTcPlane + bi] = h1;
            sl[5 * kTcPlane + bi] = h2;
            split3(wt, h0, h1, h2);
            sl[6 * kTcPlane + bi] = h0;
            sl[7 * kTcPlane + bi] = h1;
            sl[8 * kTcPlane + bi] = h2;
        }
        __syncwarp();
        // 5. the three transposed contractions, summed into fr
        tc_contract(sbase, sbase + 3 * P, sbase + 6 * P, bb, fr, fs, ft, true, lane);
        __syncwarp();
        // 6. w (+ Helmholtz mass term) out, <p, A p> partial
#pragma unroll
        for (int m = 0; m < 16; m++) {
            const int p = lane + 32 * m, k = p >> 6, j = (p >> 3) & 7, i = p & 7;
            float w = fr[tc_fidx(k, j, i)];
            if (a.mass) w = fmaf(ld_stream(a.mass + eb + p), uv[m], w);
            st_keep<FUSED>(a.w + eb + p, w);
            if (FUSED) fpair_add(paph, papl, uv[m] * w);
        }
        __syncwarp();
    }
    if (FUSED) {
        CGState* st = a.st;
        float h[1] = {paph}, l[1] = {papl};
        grid_sum_finalize_pair<1>(h, l, a.partials, a.counter, [&](double (&acc)[1]) { cg_set_alpha(st, acc[0]); });
    }
}

template <bool FUSED>
static int launch_tc(sem_handle* h, const AxParams<float>& a, cudaStream_t s) {
    constexpr size_t smem = (size_t)kTcWarps * kTcWarpBytes;
    static int per_sm = -1;
    if (per_sm < 0) {
        cudaError_t e = cudaFuncSetAttribute(ax_tc_kernel<FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(ax_tc_kernel)");
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ax_tc_kernel<FUSED>, kTcWarps * 32, smem);
        per_sm = nb > 0 ? nb : 1;
    }
    if (a.dry) return SEM_OK;
    const int64_t ctas = (a.E + kTcWarps - 1) / kTcWarps;
    int64_t grid = std::min<int64_t>(ctas, (int64_t)h->sm_count * per_sm);
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, kMaxPartials));
    ax_tc_kernel<FUSED><<<(int)grid, kTcWarps * 32, smem, s>>>(a);
    SEM_LAUNCH_CHECK("ax_tc_kernel");
    h->launches++;
    return SEM_OK;
}

int dispatch_ax_tc(sem_handle* h, int lx, const AxParams<float>& a, bool fused, cudaStream_t s) {
    if (lx != 8) return fail(SEM_EINVAL, "the tensor-core operator covers lx = 8");
    return fused ? launch_tc<true>(h, a, s) : launch_tc<false>(h, a, s);
}

}  // namespace sem
