// Device helpers of the gather-scatter QQ^T (Sec. II-A of Karp et al.):
// segment sums over the copies of a node, shared by the gather-scatter
// launches and the persistent CG kernel.  Copies are always summed left to
// right in ascending local index, so every caller gets the same bits.
#pragma once

#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

// The loads are latency-bound (scattered 4- or 8-byte accesses), so each
// thread issues the index and value loads of U segments before it sums and
// stores any.
// segment t of a class belongs to a solve that is done (batched, skipping)
__device__ __forceinline__ bool seg_done(const uint16_t* sid, const CGState* st, int64_t t) {
    return sid && st[sid[t]].done;
}

template <typename T, int U>
__device__ __forceinline__ void gs_pairs(T* __restrict__ u, const int2* __restrict__ idx, int64_t n, int64_t t0,
                                         int64_t stride, const uint16_t* sid = nullptr, const CGState* st = nullptr) {
    for (int64_t t = t0; t < n; t += stride * U) {
        int2 q[U];
        T a[U], b[U];
#pragma unroll
        for (int k = 0; k < U; k++)
            q[k] = (t + k * stride < n && !seg_done(sid, st, t + k * stride)) ? idx[t + k * stride] : make_int2(-1, -1);
#pragma unroll
        for (int k = 0; k < U; k++)
            if (q[k].x >= 0) {
                a[k] = u[q[k].x];
                b[k] = u[q[k].y];
            }
#pragma unroll
        for (int k = 0; k < U; k++)
            if (q[k].x >= 0) {
                const T sum = a[k] + b[k];
                u[q[k].x] = sum;
                u[q[k].y] = sum;
            }
    }
}

template <typename T, int U>
__device__ __forceinline__ void gs_quads(T* __restrict__ u, const int4* __restrict__ idx, int64_t n, int64_t t0,
                                         int64_t stride, const uint16_t* sid = nullptr, const CGState* st = nullptr) {
    for (int64_t t = t0; t < n; t += stride * U) {
        int4 q[U];
        T a[U][4];
#pragma unroll
        for (int k = 0; k < U; k++)
            q[k] = (t + k * stride < n && !seg_done(sid, st, t + k * stride)) ? idx[t + k * stride]
                                                                               : make_int4(-1, -1, -1, -1);
#pragma unroll
        for (int k = 0; k < U; k++)
            if (q[k].x >= 0) {
                a[k][0] = u[q[k].x];
                a[k][1] = u[q[k].y];
                a[k][2] = u[q[k].z];
                a[k][3] = u[q[k].w];
            }
#pragma unroll
        for (int k = 0; k < U; k++)
            if (q[k].x >= 0) {
                const T sum = ((a[k][0] + a[k][1]) + a[k][2]) + a[k][3];
                u[q[k].x] = sum;
                u[q[k].y] = sum;
                u[q[k].z] = sum;
                u[q[k].w] = sum;
            }
    }
}

// Octets, other segment sizes and the Dirichlet zero list, threads t0,
// t0 + stride, ... (no skipping)
template <typename T>
__device__ __forceinline__ void gs_rest(T* __restrict__ u, const GSLists& g, int64_t t0, int64_t stride) {
    for (int64_t t = t0; t < g.noct; t += stride) {
        const int4 q0 = g.octs[2 * t], q1 = g.octs[2 * t + 1];
        const T a0 = u[q0.x], a1 = u[q0.y], a2 = u[q0.z], a3 = u[q0.w];
        const T a4 = u[q1.x], a5 = u[q1.y], a6 = u[q1.z], a7 = u[q1.w];
        const T sum = ((((((a0 + a1) + a2) + a3) + a4) + a5) + a6) + a7;
        u[q0.x] = sum; u[q0.y] = sum; u[q0.z] = sum; u[q0.w] = sum;
        u[q1.x] = sum; u[q1.y] = sum; u[q1.z] = sum; u[q1.w] = sum;
    }
    for (int64_t t = t0; t < g.noth; t += stride) {
        const int a = g.oth_off[t], e = g.oth_off[t + 1];
        T sum = u[g.oth_idx[a]];
        for (int q = a + 1; q < e; q++) sum += u[g.oth_idx[q]];
        for (int q = a; q < e; q++) u[g.oth_idx[q]] = sum;
    }
    for (int64_t t = t0; t < g.nzero; t += stride) u[g.zero_idx[t]] = T(0);
}

}  // namespace sem
