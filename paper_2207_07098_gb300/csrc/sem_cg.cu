// Jacobi-preconditioned conjugate gradients (Sec. II-B of Karp et al.) and
// FP64 iterative refinement around an FP32 inner CG.
//
// One CG iteration is three launches, captured in CUDA graphs:
//   K-A  p = z + beta p;  w = A_L p;  alpha = rho / <p, w>     (sem_ax.cu)
//   K-B  w = mask QQ^T w                                       (sem_gs.cu)
//   K-C  x += alpha p;  r -= alpha w;  z = Minv r;  rho = <r, z>, rr = <r, r>
// The scalars live in device memory (CGState) and are produced by the last
// CTA of each reducing launch in a fixed order, so a solve is bit-reproducible.
// Each launch returns at once when the solve is already done, so a graph of
// several iterations can run past convergence without changing the result;
// the host reads the state between graph launches.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

template <typename T>
struct VecT;
template <>
struct VecT<double> {
    using V = double2;
    using M = uchar2;
    static constexpr int W = 2;
};
template <>
struct VecT<float> {
    using V = float4;
    using M = uchar4;
    static constexpr int W = 4;
};

template <typename T>
struct UpdParams {
    T* x;
    const T* p;
    T* r;
    const T* w;
    T* z;
    const T* minv;
    const uint8_t* mult;
    int64_t n;
    CGState* st;
    double* partials;
    unsigned int* counter;
};

template <typename T>
__device__ __forceinline__ void upd_point(T& x, T p, T& r, T w, T& z, T mi, T inv, T ta, T& rz, T& rr) {
    x = fma(ta, p, x);
    r = fma(-ta, w, r);
    z = mi * r;
    rz = fma(r * z, inv, rz);
    rr = fma(r * r, inv, rr);
}

// K-C: x += alpha p; r -= alpha w; z = Minv r; partial sums of <r,z>, <r,r>
// (weights 1/mult).  Per-thread sums of W points in T, then FP64.
template <typename T>
__global__ void __launch_bounds__(256) cg_update_kernel(UpdParams<T> a) {
    using VT = VecT<T>;
    using V = typename VT::V;
    using M = typename VT::M;
    constexpr int W = VT::W;
    if (a.st->done) return;
    __shared__ T inv[256];
    __shared__ T s_ta;  // alpha, converted once by thread 0
    // 1/m per copy count; FP32 kernels divide in FP32 (the same correctly
    // rounded values for m < 256; an FP64 division per thread would occupy
    // GB300's slow FP64 pipe at every launch)
    for (int m = threadIdx.x; m < 256; m += blockDim.x)
        inv[m] = m ? (sizeof(T) == 4 ? (T)(1.0f / (float)m) : (T)(1.0 / m)) : T(0);
    if (threadIdx.x == 0) s_ta = (T)a.st->alpha;
    __syncthreads();
    const T ta = s_ta;
    // per-thread partial sums in T with Kahan compensation, converted to FP64
    // once per thread (FP64 accumulation across threads and CTAs)
    T rzs = T(0), rzc = T(0), rrs = T(0), rrc = T(0);
    auto kahan = [](T& sum, T& c, T v) {
        if constexpr (sizeof(T) == 8) {
            sum += v;  // FP64: plain accumulation (the FP64 pipe is the bottleneck)
        } else {
            const T y = v - c;
            const T t = sum + y;
            c = (t - sum) - y;
            sum = t;
        }
    };
    const int64_t nv = a.n / W;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv; q += (int64_t)gridDim.x * blockDim.x) {
        V x = reinterpret_cast<const V*>(a.x)[q];
        const V p = ld_stream(reinterpret_cast<const V*>(a.p) + q);
        V r = reinterpret_cast<const V*>(a.r)[q];
        const V w = ld_stream(reinterpret_cast<const V*>(a.w) + q);
        const V mi = ld_stream(reinterpret_cast<const V*>(a.minv) + q);
        const M mu = reinterpret_cast<const M*>(a.mult)[q];
        V z;
        T lrz = T(0), lrr = T(0);
        T* xs = reinterpret_cast<T*>(&x);
        const T* ps = reinterpret_cast<const T*>(&p);
        T* rs = reinterpret_cast<T*>(&r);
        const T* ws = reinterpret_cast<const T*>(&w);
        const T* ms = reinterpret_cast<const T*>(&mi);
        T* zs = reinterpret_cast<T*>(&z);
        const unsigned char* us = reinterpret_cast<const unsigned char*>(&mu);
#pragma unroll
        for (int c = 0; c < W; c++) upd_point<T>(xs[c], ps[c], rs[c], ws[c], zs[c], ms[c], inv[us[c]], ta, lrz, lrr);
        reinterpret_cast<V*>(a.x)[q] = x;
        reinterpret_cast<V*>(a.r)[q] = r;
        reinterpret_cast<V*>(a.z)[q] = z;
        kahan(rzs, rzc, lrz);
        kahan(rrs, rrc, lrr);
    }
    if constexpr (sizeof(T) == 4) {
        // float pairs (sum, -compensation) to the block sums: no FP64 per thread
        float h[2] = {rzs, rrs}, l[2] = {-rzc, -rrc};
        if (blockIdx.x == 0) {  // scalar tail
            for (int64_t L = nv * W + threadIdx.x; L < a.n; L += blockDim.x) {
                T x = a.x[L], r = a.r[L], z;
                T lrz = T(0), lrr = T(0);
                upd_point<T>(x, a.p[L], r, a.w[L], z, a.minv[L], inv[a.mult[L]], ta, lrz, lrr);
                a.x[L] = x;
                a.r[L] = r;
                a.z[L] = z;
                fpair_add(h[0], l[0], lrz);
                fpair_add(h[1], l[1], lrr);
            }
        }
        CGState* st = a.st;
        grid_sum_finalize_pair<2>(h, l, a.partials, a.counter,
                                  [&](double (&acc)[2]) { cg_set_rho(st, acc[0], acc[1]); });
    } else {
        double rz = (double)rzs - (double)rzc, rr = (double)rrs - (double)rrc;
        if (blockIdx.x == 0) {  // scalar tail
            for (int64_t L = nv * W + threadIdx.x; L < a.n; L += blockDim.x) {
                T x = a.x[L], r = a.r[L], z;
                T lrz = T(0), lrr = T(0);
                upd_point<T>(x, a.p[L], r, a.w[L], z, a.minv[L], inv[a.mult[L]], ta, lrz, lrr);
                a.x[L] = x;
                a.r[L] = r;
                a.z[L] = z;
                rz += (double)lrz;
                rr += (double)lrr;
            }
        }
        double v[2] = {rz, rr};
        CGState* st = a.st;
        grid_sum_finalize<2>(v, a.partials, a.counter, [&](double (&acc)[2]) { cg_set_rho(st, acc[0], acc[1]); });
    }
}

// CG start: z = Minv r; rho = <r,z>, rr = <r,r>, bb = <b,b>; state reset.
// carry_c > 0: the direction p in memory is kept from the previous solve on
// this state, whose units were carry_c times smaller than this one's (the
// ratio of the two right-hand sides' scalings); the next iteration takes
// p = z + rho / (rho_old_prev * carry_c) p, which is the continued CG step
// with p rescaled by carry_c and its rho_old by carry_c^2 (residual
// replacement).  carry_c <= 0: a fresh start (p = z).
template <typename T>
__global__ void __launch_bounds__(256) cg_init_kernel(const T* __restrict__ b, const T* __restrict__ r,
                                                      T* __restrict__ z, const T* __restrict__ minv,
                                                      const uint8_t* __restrict__ mult, int64_t n, double tol,
                                                      int max_iter, CGState* st, double* partials,
                                                      unsigned int* counter, double carry_c) {
    __shared__ double inv[256];
    for (int m = threadIdx.x; m < 256; m += blockDim.x) inv[m] = m ? 1.0 / m : 0.0;
    __syncthreads();
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x) {
        const double rv = (double)r[L];
        const T zv = minv[L] * r[L];
        z[L] = zv;
        const double iv = inv[mult[L]];
        v[0] = fma(rv * (double)zv, iv, v[0]);
        v[1] = fma(rv * rv, iv, v[1]);
        const double bv = (double)b[L];
        v[2] = fma(bv * bv, iv, v[2]);
    }
    grid_sum_finalize<3>(v, partials, counter, [&](double (&acc)[3]) {
        const double rho_prev = st->rho_old;  // <r, z> that built the kept direction
        st->rho = acc[0];
        st->carry = carry_c > 0.0 ? 1 : 0;
        st->rho_old = carry_c > 0.0 ? rho_prev * carry_c : 1.0;
        st->rr = acc[1];
        st->bb = acc[2];
        st->tol2 = tol * tol * acc[2];
        st->alpha = 0.0;
        st->pap = 0.0;
        st->iter = 0;
        st->max_iter = max_iter;
        const bool conv = (acc[2] == 0.0 || acc[1] <= st->tol2);
        st->done = (conv || max_iter <= 0) ? 1 : 0;
        st->status = (conv || max_iter > 0) ? SEM_OK : SEM_ENOTCONV;
    });
}

// r = b - w (FP64), out[0] = <r, r>, out[1] = <b, b>
__global__ void __launch_bounds__(256) resid_kernel(const double* __restrict__ b, const double* __restrict__ w,
                                                    double* __restrict__ r, const uint8_t* __restrict__ mult,
                                                    int64_t n, double* partials, unsigned int* counter,
                                                    double* out) {
    __shared__ double inv[256];
    for (int m = threadIdx.x; m < 256; m += blockDim.x) inv[m] = m ? 1.0 / m : 0.0;
    __syncthreads();
    double v[2] = {0.0, 0.0};
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x) {
        const double bv = b[L];
        const double rv = bv - w[L];
        r[L] = rv;
        const double iv = inv[mult[L]];
        v[0] = fma(rv * rv, iv, v[0]);
        v[1] = fma(bv * bv, iv, v[1]);
    }
    grid_sum_finalize<2>(v, partials, counter, [&](double (&acc)[2]) {
        out[0] = acc[0];
        out[1] = acc[1];
    });
}

// Refinement: b32 = r32 = float(r / ||r||), d32 = 0 (||r||^2 in rr_in[0]).
__global__ void ir_prepare_kernel(const double* __restrict__ r, const double* rr_in, float* __restrict__ b32,
                                  float* __restrict__ r32, float* __restrict__ d32, int64_t n) {
    const double s = 1.0 / sqrt(rr_in[0]);
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x) {
        const float v = (float)(r[L] * s);
        b32[L] = v;
        r32[L] = v;
        d32[L] = 0.0f;
    }
}

// Refinement: x += ||r|| d32
__global__ void ir_correct_kernel(double* __restrict__ x, const float* __restrict__ d32, const double* rr_in,
                                  int64_t n) {
    const double s = sqrt(rr_in[0]);
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x)
        x[L] = fma(s, (double)d32[L], x[L]);
}

// v *= f (f a power of two: exact)
__global__ void scale_kernel(double* __restrict__ v, double f, int64_t n) {
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x)
        v[L] *= f;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static int launch_scale(sem_handle* h, double* v, double f, cudaStream_t s) {
    scale_kernel<<<grid_for(h, h->n_local, 256, 8), 256, 0, s>>>(v, f, h->n_local);
    SEM_LAUNCH_CHECK("scale_kernel");
    h->launches++;
    return SEM_OK;
}

int launch_cg_update(sem_handle* h, int precision, cudaStream_t s) {
    const int grid = grid_for(h, h->n_local / 4 + 1, 256, 8);
    if (is_f32(precision)) {
        UpdParams<float> a = {h->ws.d32, h->ws.p32, h->ws.r32, h->ws.w32, h->ws.z32, h->minv32, h->mult,
                              h->n_local, h->state + 1, h->partials, h->counters + 3};
        cg_update_kernel<float><<<grid, 256, 0, s>>>(a);
    } else {
        UpdParams<double> a = {h->ws.x, h->ws.p, h->ws.r, h->ws.w, h->ws.z, h->minv64, h->mult,
                               h->n_local, h->state, h->partials, h->counters + 3};
        cg_update_kernel<double><<<grid, 256, 0, s>>>(a);
    }
    SEM_LAUNCH_CHECK("cg_update_kernel");
    h->launches++;
    return SEM_OK;
}

static int launch_ka(sem_handle* h, int precision, cudaStream_t s) {
    if (precision == kPipePrec) return launch_pipe_iteration(h, s);  // all three launches
    return precision == kPairPrec ? launch_pair_ka(h, s) : launch_cg_pupdate_ax(h, precision, s);
}

static int launch_kb_kc(sem_handle* h, int precision, cudaStream_t s) {
    if (precision == kPipePrec) return SEM_OK;
    if (precision == kPairPrec) return launch_pair_rest(h, s);
    // the state slot of the K-A and K-C of this precision (FP32 inner loop: 1)
    const CGState* st = is_f32(precision) ? h->state + 1 : h->state;
    int rc = launch_gs_until_done(h, is_f32(precision) ? (void*)h->ws.w32 : (void*)h->ws.w, is_f32(precision), st, s);
    if (!rc) rc = launch_cg_update(h, precision, s);
    return rc;
}

static int launch_iteration(sem_handle* h, int precision, cudaStream_t s) {
    int rc = launch_ka(h, precision, s);
    return rc ? rc : launch_kb_kc(h, precision, s);
}

// The CG loop graph of `chunk` iterations in cache `g`; with `events`, the
// second K-A of the chunk is bracketed by the handle's timing events.
static int get_graph(sem_handle* h, int precision, int chunk, cudaGraphExec_t* out, GraphCache& g, bool events) {
    // (the pair-form loop has its own precision code and always the line kernel)
    const int variant = precision == kPairPrec   ? kDflVariant
                        : precision == kPipePrec ? ax_variant_for(h, h->parts[0].lx, kClsF64)
                                                 : ax_variant_of_precision(h, h->parts[0].lx, precision);
    if (g.exec && g.key_prec == precision && g.key_chunk == chunk && g.key_variant == variant) {
        *out = g.exec;
        return SEM_OK;
    }
    if (g.exec) {
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
    }
    if (!h->capture_stream) SEM_CUDA_TRY(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    int prc = prepare_cg_kernels(h);
    if (!prc && precision == kPairPrec) prc = prepare_pair_kernels(h);
    if (prc) return prc;
    for (auto& ev : h->ax_ev)
        if (!ev) SEM_CUDA_TRY(cudaEventCreate(&ev));
    cudaStream_t cs = h->capture_stream;
    const int64_t launches_before = h->launches;  // captured kernels are counted per graph launch
    SEM_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int rc = SEM_OK;
    // the K-A that is timed: the second of the chunk (it follows K-C inside the
    // graph, as in steady state; the first one starts after the host check)
    const int timed = !events ? -1 : chunk > 1 ? 1 : 0;
    for (int it = 0; it < chunk && rc == SEM_OK; it++) {
        if (it == timed && cudaEventRecordWithFlags(h->ax_ev[0], cs, cudaEventRecordExternal) != cudaSuccess)
            rc = fail(SEM_ECUDA, "event record");
        if (!rc) rc = launch_ka(h, precision, cs);
        if (it == timed && !rc && cudaEventRecordWithFlags(h->ax_ev[1], cs, cudaEventRecordExternal) != cudaSuccess)
            rc = fail(SEM_ECUDA, "event record");
        if (!rc) rc = launch_kb_kc(h, precision, cs);
    }
    h->launches = launches_before;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g.exec = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    g.key_prec = precision;
    g.key_chunk = chunk;
    g.key_variant = variant;
    *out = g.exec;
    return SEM_OK;
}

struct AxTiming {
    double ms = 0.0;
    int samples = 0;
};

// Iterations of the tail graph: the loop's predicted last iterations run in
// graphs of this size, so a run that ends inside a chunk launches few
// iterations past its end (kernels of a finished solve still launch, then
// return at once).
constexpr int kTailChunk = 4;

// Run CG iterations on state slot `slot` until done.  Returns SEM_OK or an
// error; the solve status is in the state.  With graphs, the duration of one
// K-A of every full-chunk graph launch (the second of the chunk) is added to
// `tm`; a launch that ends the solve before that K-A ran adds nothing.
// `expect` > 0 predicts the iterations of this run (a refinement step takes
// about as many as the one before): once fewer than a chunk remain by that
// count, the loop launches just enough tail graphs to reach it; past the
// predicted end it launches 1, 2, 4, ... tail graphs per check (up to a
// chunk).  Each check reads the state and the device error word back with
// one synchronisation.
static int run_cg_loop(sem_handle* h, int precision, const sem_solve_opts& o, int slot, cudaStream_t s,
                       CGState* out, AxTiming* tm, int expect) {
    const int chunk = std::max(1, std::min(o.graph_chunk, 1024));
    cudaGraphExec_t exec = nullptr, tail = nullptr;
    if (o.use_graph) {
        int rc = get_graph(h, precision, chunk, &exec, h->graph, true);
        if (!rc && expect > 0 && chunk > kTailChunk) rc = get_graph(h, precision, kTailChunk, &tail, h->graph_tail, false);
        if (rc) return rc;
    }
    LoopReadback* rb = h->loop_host;
    SEM_CUDA_TRY(cudaMemcpyAsync(&rb->st, h->state + slot, sizeof(CGState), cudaMemcpyDeviceToHost, s));
    SEM_CUDA_TRY(cudaStreamSynchronize(s));
    *out = rb->st;
    const int iter0 = out->iter;
    int over = 0;  // checks past the predicted end
    const int64_t max_rounds = (int64_t)out->max_iter / (tail ? kTailChunk : chunk) + 3;
    for (int64_t round = 0; !out->done && round < max_rounds; round++) {
        const int iter_before = out->iter;
        const int left = expect - (out->iter - iter0);  // predicted iterations still to run
        bool full = false;
        if (tail && left < chunk) {
            const int k = std::max(1, std::min(chunk / kTailChunk, left > 0 ? (left + kTailChunk - 1) / kTailChunk
                                                                              : 1 << std::min(over++, 16)));
            for (int q = 0; q < k; q++) SEM_CUDA_TRY(cudaGraphLaunch(tail, s));
            h->launches += 3 * (int64_t)kTailChunk * k;
        } else if (exec) {
            SEM_CUDA_TRY(cudaGraphLaunch(exec, s));
            h->launches += 3 * (int64_t)chunk;
            full = true;
        } else {
            for (int it = 0; it < chunk; it++) {
                int rc = launch_iteration(h, precision, s);
                if (rc) return rc;
            }
        }
        SEM_CUDA_TRY(cudaMemcpyAsync(&rb->st, h->state + slot, sizeof(CGState), cudaMemcpyDeviceToHost, s));
        SEM_CUDA_TRY(cudaMemcpyAsync(&rb->err, device_error_word(h), sizeof(int), cudaMemcpyDeviceToHost, s));
        SEM_CUDA_TRY(cudaStreamSynchronize(s));
        *out = rb->st;
        const int err_word = rb->err;
        if (err_word) {
            // a staged kernel gave up waiting: its CTAs skipped the reductions, so
            // the counters are reset and the solve ends with SEM_ETIMEOUT
            cudaMemset(device_error_word(h), 0, sizeof(int));
            cudaMemset(h->counters, 0, 16 * sizeof(unsigned));
            return fail(SEM_ETIMEOUT, "a staged operator kernel gave up waiting for its bulk copies");
        }
        if (full && tm && (chunk == 1 || out->iter - iter_before >= 2)) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, h->ax_ev[0], h->ax_ev[1]) == cudaSuccess) {
                tm->ms += ms;
                tm->samples++;
            } else {
                cudaGetLastError();
            }
        }
    }
    if (!out->done) return fail(SEM_ETIMEOUT, "CG loop did not finish within its iteration budget");
    return SEM_OK;
}

// The CG loop of state slot `slot` as one persistent launch when the options
// and the mesh allow it (opts.persistent: 1 forces it where available, -1
// takes it below kPersistAutoPoints local points), else the graph loop.
static bool use_persist(const sem_handle* h, const sem_solve_opts& o, int precision) {
    if (o.persistent == 0 || precision == kPairPrec || precision == kPipePrec || precision == SEM_FP64_PAIR ||
        precision == SEM_TC_SPLIT || !persist_available(h))
        return false;
    return o.persistent > 0 || h->n_local <= kPersistAutoPoints;
}

static int run_cg(sem_handle* h, int precision, const sem_solve_opts& o, int slot, cudaStream_t s, CGState* out,
                  AxTiming* tm, bool* persisted, int expect = 0) {
    if (!use_persist(h, o, precision)) return run_cg_loop(h, precision, o, slot, s, out, tm, expect);
    *persisted = true;
    int rc = launch_cg_persist(h, precision, slot, s);
    if (rc) return rc;
    SEM_CUDA_TRY(cudaMemcpyAsync(out, h->state + slot, sizeof(CGState), cudaMemcpyDeviceToHost, s));
    SEM_CUDA_TRY(cudaStreamSynchronize(s));
    int err_word = 0;
    SEM_CUDA_TRY(cudaMemcpy(&err_word, device_error_word(h), sizeof(int), cudaMemcpyDeviceToHost));
    if (err_word) {
        cudaMemset(device_error_word(h), 0, sizeof(int));
        cudaMemset(h->counters, 0, 16 * sizeof(unsigned));
        return fail(SEM_ETIMEOUT, "a grid barrier of the persistent CG kernel expired");
    }
    if (!out->done) return fail(SEM_ETIMEOUT, "the persistent CG kernel ended before the solve did");
    return SEM_OK;
}

// rr_bb[0] = ||b - A x||^2, rr_bb[1] = ||b||^2 (unique-node norm), r = b - A x,
// with the native FP64 operator whatever the solve's iterations use
int true_residual(sem_handle* h, const double* x, const double* b, double* rr_bb, cudaStream_t s) {
    int rc = launch_ax_local(h, x, h->ws.w, SEM_FP64, s);
    if (!rc) rc = launch_gs(h, h->ws.w, false, true, s);
    if (rc) return rc;
    resid_kernel<<<grid_for(h, h->n_local, 256, 4), 256, 0, s>>>(b, h->ws.w, h->ws.r, h->mult, h->n_local,
                                                                 h->partials, h->counters + 4, rr_bb);
    SEM_LAUNCH_CHECK("resid_kernel");
    h->launches++;
    return SEM_OK;
}

// Relative tolerance of one inner FP32 solve: opts.inner_tol, relaxed when
// the outer residual `rel` is already close to the target so the last step
// only removes the remaining factor rel / tol (with margin), never looser
// than 0.1 so each refinement step still cuts the residual by ten.
double inner_tolerance(const sem_solve_opts& o, double rel) {
    const double need = 0.3 * o.tol / rel;
    return std::min(0.1, std::max(o.inner_tol, need));
}

bool host_resident(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

static bool is_host_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

static int read_rrbb(sem_handle* h, double* hb, cudaStream_t s) {
    SEM_CUDA_TRY(cudaMemcpyAsync(hb, h->scratch, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SEM_CUDA_TRY(cudaStreamSynchronize(s));
    return SEM_OK;
}

static int solve_single(sem_handle* h, double* x_user, const double* b_user, const sem_solve_opts& o,
                        sem_solve_stats* stats, cudaStream_t s) {
    int rc = ensure_workspace(h, o.mode == SEM_MODE_MIXED_IR);
    if (rc) return rc;
    // inner precision of the mixed mode: FP32, or its tensor-core form
    const int prec = o.mode == SEM_MODE_MIXED_IR ? (o.tc_split ? SEM_TC_SPLIT : SEM_FP32) : o.precision;
    if (o.autotune) {
        if (is_f32(prec) && (rc = autotune_ax(h, true, s))) return rc;
        // the FP64 class computes every true residual
        if ((rc = autotune_ax(h, false, s))) return rc;
    }
    const int64_t n = h->n_local;
    const size_t bytes = sizeof(double) * n;
    const bool xh = is_host_ptr(x_user), bh = is_host_ptr(b_user);
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, s);
    SEM_CUDA_TRY(cudaMemcpyAsync(h->ws.x, x_user, bytes, xh ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    SEM_CUDA_TRY(cudaMemcpyAsync(h->ws.b, b_user, bytes, bh ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    // projection onto previous solutions: the start is the projected solution
    if (o.projection > 0 && (rc = proj_start(h, o.projection, s))) return rc;
    double* rrbb = h->scratch;  // [0] rr, [1] bb
    sem_solve_stats st = {};
    bool first_residual = true;
    AxTiming tm;
    const int64_t launches0 = h->launches;
    CGState hs;
    int status = SEM_OK;
    double hb[2] = {0.0, 0.0};  // ||b - A x||^2, ||b||^2 of the returned x (SEM_FP64 operator)
    bool persisted = false;     // a CG loop ran as one persistent launch
    if (o.mode == SEM_MODE_FP64) {
        // CG with residual replacement: when the recursive residual says
        // "converged" but the true residual ||b - A x|| is still above tol
        // (rounding drift), CG restarts from the true residual, up to four times.
        // With the line-transform FP32-pair operator the CG vectors live as
        // float pairs, and x, b, r are scaled by a power of two (exactly) into
        // the range the pair format represents.
        const bool pipe = o.pipelined != 0;  // pipelined PCG, native FP64 operator
        const bool pair = !pipe && prec == SEM_FP64_PAIR && pair_cg_available(h);
        if (pair && (rc = ensure_pair_workspace(h))) return rc;
        if (pipe && (rc = ensure_pipe_workspace(h))) return rc;
        double scale = 1.0;
        int used = 0;
        // Pipelined PCG in segments of kPipeSeg iterations with residual
        // replacement between them: the recursively updated r, u, w, s, q, z of
        // the pipelined recurrences drift from the vectors they stand for over
        // hundreds of iterations (on the 32^3 workload the recurrence broke down
        // at a true residual of 1e-4 after 1800 iterations), so every segment
        // starts from the true residual and recomputes the others from x and the
        // kept direction p (Cools and Vanroose's residual replacement).  A
        // breakdown restarts from the true residual (at most four times).
        int pipe_base = 0, pipe_breaks = 0;
        bool pipe_live = false;
        for (int seg = 0; pipe; seg++) {
            if ((rc = true_residual(h, h->ws.x, h->ws.b, rrbb, s)) || (rc = read_rrbb(h, hb, s))) return rc;
            const double rel = relative_residual(hb[0], hb[1]);
            if (first_residual) st.relres_start = rel;
            first_residual = false;
            if (!std::isfinite(rel)) {
                status = SEM_EBREAKDOWN;
                break;
            }
            if (hb[1] == 0.0 || rel <= o.tol) {
                status = SEM_OK;
                break;
            }
            if (used >= o.max_iter) {
                status = SEM_ENOTCONV;
                break;
            }
            if (status == SEM_EBREAKDOWN) {
                if (++pipe_breaks > 4) break;
                pipe_live = false;
            }
            const int len = std::min(kPipeSeg, o.max_iter - used);
            if (pipe_live) {
                rc = launch_pipe_replace(h, len, s);
            } else {
                pipe_base = used;
                rc = launch_pipe_init(h, o.tol, len, s);
            }
            if (rc || (rc = run_cg(h, kPipePrec, o, 0, s, &hs, &tm, &persisted))) return rc;
            pipe_live = true;
            used = pipe_base + hs.iter;
            st.relres_recursive = hs.bb > 0 ? std::sqrt(hs.rr / hs.bb) : 0.0;
            status = hs.status == SEM_ENOTCONV ? SEM_OK : hs.status;  // a segment ended: replace and go on
        }
        for (int restart = 0; !pipe; restart++) {
            if ((rc = true_residual(h, h->ws.x, h->ws.b, rrbb, s)) || (rc = read_rrbb(h, hb, s))) return rc;
            const double rel = relative_residual(hb[0], hb[1]);
            if (first_residual) st.relres_start = rel;
            first_residual = false;
            if (!std::isfinite(rel)) {  // NaN or Inf in x0 or b, or a diverged iterate
                status = SEM_EBREAKDOWN;
                break;
            }
            if (restart > 0 && (rel <= o.tol || status != SEM_OK || restart > 4 || used >= o.max_iter)) break;
            if (pair) {
                if (restart == 0 && hb[1] > 0.0) {
                    const int e = std::ilogb(std::sqrt(hb[1]));
                    scale = (e > 16 || e < -16) ? std::ldexp(1.0, e) : 1.0;
                }
                if (scale != 1.0 && ((rc = launch_scale(h, h->ws.x, 1.0 / scale, s)) ||
                                     (rc = launch_scale(h, h->ws.b, 1.0 / scale, s)) ||
                                     (rc = launch_scale(h, h->ws.r, 1.0 / scale, s))))
                    return rc;
                if ((rc = launch_pair_split_x(h, s)) || (rc = launch_pair_init(h, o.tol, o.max_iter - used, s)))
                    return rc;
            } else {
                cg_init_kernel<double><<<grid_for(h, n, 256, 4), 256, 0, s>>>(
                    h->ws.b, h->ws.r, h->ws.z, h->minv64, h->mult, n, o.tol, o.max_iter - used, h->state,
                    h->partials, h->counters + 5, 0.0);
                SEM_LAUNCH_CHECK("cg_init_kernel");
                h->launches++;
            }
            if ((rc = run_cg(h, pair ? kPairPrec : prec, o, 0, s, &hs, &tm, &persisted)))
                return rc;
            if (pair) {
                if ((rc = launch_pair_join_x(h, s))) return rc;
                if (scale != 1.0 && ((rc = launch_scale(h, h->ws.x, scale, s)) ||
                                     (rc = launch_scale(h, h->ws.b, scale, s))))
                    return rc;
            }
            used += hs.iter;
            st.relres_recursive = hs.bb > 0 ? std::sqrt(hs.rr / hs.bb) : 0.0;
            status = hs.status;
        }
        st.iterations = used;
    } else {
        // FP64 refinement around an FP32 inner CG; with ir_carry the inner CG
        // keeps its direction across steps (residual replacement).  A step
        // stopped by max_iter is not judged for stagnation (the CG residual
        // norm is not monotone), and its direction is kept like any other.
        double prev = INFINITY, rn_prev = 0.0;
        bool can_carry = false, capped_last = false;
        int outer = 0, inner = 0, last_inner = 0;
        for (;;) {
            if ((rc = true_residual(h, h->ws.x, h->ws.b, rrbb, s)) || (rc = read_rrbb(h, hb, s))) return rc;
            const double rel = relative_residual(hb[0], hb[1]);
            if (first_residual) st.relres_start = rel;
            first_residual = false;
            st.relres_recursive = rel;
            if (!std::isfinite(rel)) { status = SEM_EBREAKDOWN; break; }
            if (hb[1] == 0.0 || rel <= o.tol) { status = SEM_OK; break; }
            if (outer >= o.max_outer) { status = SEM_ENOTCONV; break; }
            if (outer > 0 && rel > 0.5 * prev && !capped_last) { status = SEM_ESTAGNATE; break; }
            prev = rel;
            // the inner right-hand side is r / ||r||: the kept direction's units
            // were ||r_prev|| / ||r|| times smaller than the new ones
            const double rn = std::sqrt(hb[0]);
            const double carry_c = (o.ir_carry && can_carry && rn > 0.0) ? rn_prev / rn : 0.0;
            ir_prepare_kernel<<<grid_for(h, n, 256, 8), 256, 0, s>>>(h->ws.r, rrbb, h->ws.b32, h->ws.r32,
                                                                     h->ws.d32, n);
            cg_init_kernel<float><<<grid_for(h, n, 256, 4), 256, 0, s>>>(
                h->ws.b32, h->ws.r32, h->ws.z32, h->minv32, h->mult, n, inner_tolerance(o, rel), o.max_iter,
                h->state + 1, h->partials, h->counters + 5, carry_c);
            SEM_LAUNCH_CHECK("ir prepare");
            h->launches += 2;
            if ((rc = run_cg(h, prec, o, 1, s, &hs, &tm, &persisted, last_inner))) return rc;
            inner += hs.iter;
            last_inner = hs.iter;
            capped_last = hs.iter >= o.max_iter;
            can_carry = (hs.status == SEM_OK || hs.status == SEM_ENOTCONV) && hs.iter > 0;
            rn_prev = rn;
            ir_correct_kernel<<<grid_for(h, n, 256, 8), 256, 0, s>>>(h->ws.x, h->ws.d32, rrbb, n);
            SEM_LAUNCH_CHECK("ir_correct_kernel");
            h->launches++;
            outer++;
        }
        st.iterations = inner;
        st.outer_iterations = outer;
    }
    // hb holds the true residual of the final iterate (both loops end right after computing it)
    const double rel_final = relative_residual(hb[0], hb[1]);
    if (o.projection > 0 && status == SEM_OK && rel_final <= o.tol && (rc = proj_update(h, s))) return rc;
    SEM_CUDA_TRY(cudaMemcpyAsync(x_user, h->ws.x, bytes, xh ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    cudaEventRecord(ev1, s);
    SEM_CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    int err_word = 0;
    SEM_CUDA_TRY(cudaMemcpy(&err_word, device_error_word(h), sizeof(int), cudaMemcpyDeviceToHost));
    if (err_word) {
        cudaMemset(device_error_word(h), 0, sizeof(int));
        cudaMemset(h->counters, 0, 16 * sizeof(unsigned));
        return fail(SEM_ETIMEOUT, "a staged operator kernel gave up waiting for its bulk copies");
    }
    st.relres = relative_residual(hb[0], hb[1]);
    // SEM_OK promises the tolerance on the true residual, whatever the loop reported
    if (status == SEM_OK && !(st.relres <= o.tol)) status = std::isfinite(st.relres) ? SEM_ENOTCONV : SEM_EBREAKDOWN;
    st.time_ms = ms;
    st.ax_variant = (o.mode == SEM_MODE_FP64 && o.pipelined) ? ax_variant_for(h, h->parts[0].lx, kClsF64)
                                                              : ax_variant_of_precision(h, h->parts[0].lx, prec);
    st.status = status;
    st.launches_per_iteration = persisted ? 0 : 3;
    st.kernel_launches = h->launches - launches0;
    st.ax_samples = tm.samples;
    st.ax_ms = tm.samples ? tm.ms / tm.samples : 0.0;
    if (stats) *stats = st;
    if (status != SEM_OK) {
        const char* what = status == SEM_ENOTCONV   ? "not converged within max_iter / max_outer"
                           : status == SEM_EBREAKDOWN ? "CG breakdown (p^T A p <= 0 or non-finite residual)"
                                                      : "refinement stagnated";
        set_error(what);
    }
    return status;
}

}  // namespace sem

using namespace sem;

extern "C" {

SEM_API int sem_cg_solve(sem_handle* h, double* x, const double* b, const sem_solve_opts* opts,
                         sem_solve_stats* stats, cudaStream_t s) {
    if (!h || !x || !b) return fail(SEM_EINVAL, "null argument");
    if (h->nsolve != 1) return fail(SEM_EINVAL, "batch handle: use sem_cg_solve_batch");
    sem_solve_opts o;
    sem_solve_opts_default(&o);
    if (opts) o = *opts;
    if (!(o.tol > 0.0) || o.max_iter < 0 ||
        (o.mode != SEM_MODE_FP64 && o.mode != SEM_MODE_MIXED_IR && o.mode != SEM_MODE_GMRES))
        return fail(SEM_EINVAL, "bad solve options");
    if (o.mode == SEM_MODE_MIXED_IR && !(o.inner_tol > 0.0 && o.inner_tol < 1.0))
        return fail(SEM_EINVAL, "inner_tol must be in (0, 1)");
    if (o.mode == SEM_MODE_FP64 && (!valid_precision(o.precision) || is_f32(o.precision)))
        return fail(SEM_EINVAL, "FP64 mode takes SEM_FP64, SEM_FP64_NATIVE or SEM_FP64_PAIR");
    if (o.projection < 0 || o.projection > 64) return fail(SEM_EINVAL, "projection must be in [0, 64]");
    if (o.mode == SEM_MODE_GMRES) return solve_gmres(h, x, b, o, stats, s);
    return solve_single(h, x, b, o, stats, s);
}

}  // extern "C"
