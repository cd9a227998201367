// Matrix-free local operator w = A_L u with A^e = D^T (h1 G^e) D
// (Sec. II-A of Karp et al., eq. "disclap"), in FP64 and FP32, plus the CG
// variant that fuses the search-direction update p = z + beta p and the
// partial sums of <p, A p> into the same pass (Sec. II-B, P-CG).
//
// Thread layout: a CTA owns EPC elements; each element is handled by lx^2
// threads, thread (i, j) owning the column u[:, j, i] in registers.  The
// element block u[k][j][i] is staged in shared memory; r- and s-derivatives
// read it from there, the t-derivative comes from the register column.  The
// six factors G are streamed once per point (coalesced along i), the
// weighted derivatives wr, ws go back to shared memory and the transposed
// contraction produces w.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "sem_ax.cuh"
#include "sem_ax_df.cuh"

namespace sem {

int* device_error_word(sem_handle* h) { return reinterpret_cast<int*>(h->scratch + 8); }

int ax_variant_for(const sem_handle* h, int lx, int cls) {
    const int v = h->ax_variant[cls][lx];
    // the pair kernels carry no Helmholtz mass term: a Helmholtz handle takes the native ones
    if (cls == kClsPair && h->hmass64) return ax_variant_for(h, lx, kClsF64);
    if (cls == kClsPair) {
        // pinned 5 or 6 where it applies, else the line-transform form, else the
        // general pair kernel; orders neither covers use the native FP64 kernels
        if (v == kDflVariant && bulk_supported(lx)) return v;
        if (v == kDfVariant && lx <= 12) return v;
        if (bulk_supported(lx)) return kDflVariant;
        return lx <= 12 ? kDfVariant : ax_variant_for(h, lx, kClsF64);
    }
    if (cls == kClsF32 && v == kTcVariant && lx == 8) return v;
    // the bulk-staged and line-transform kernels carry no Helmholtz mass term
    // (it would cost the Poisson hot path registers): a Helmholtz handle
    // takes the slab kernel
    if (h->hmass64) return 0;
    if (cls == kClsF64 && v == kLnVariant && bulk_supported(lx)) return v;
    return (v > 0 && v <= kBulkVariantsMax && bulk_fits(lx, v, cls == kClsF32)) ? v : 0;
}

int ax_variant_of_precision(const sem_handle* h, int lx, int precision) {
    if (precision == SEM_TC_SPLIT && lx == 8) return kTcVariant;
    return precision == SEM_FP64_NATIVE ? 0 : ax_variant_for(h, lx, precision_class(precision));
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

template <typename T>
static int dispatch_variant(sem_handle* h, int lx, AxParams<T> a, bool fused, int variant, cudaStream_t s) {
    if constexpr (std::is_same<T, double>::value) {
        if (variant == kDfVariant && lx <= 12) {
            DfParams d = {};
            d.u = a.u;
            d.z = a.z;
            d.p = a.p;
            d.w = a.w;
            d.G2 = h->G2 + (a.G - h->G64) * 2;  // same element offset in the 12-plane layout
            d.D2 = h->D2[lx];
            d.E = a.E;
            d.st = a.st;
            d.partials = a.partials;
            d.counter = a.counter;
            d.dry = a.dry;
            return dispatch_ax_df_entry(h, lx, d, fused, s);
        }
        if (variant == kDflVariant && bulk_supported(lx)) {
            DflParams d = {};
            d.u = a.u;
            d.z = a.z;
            d.p = a.p;
            d.w = a.w;
            d.G2 = h->G2 + (a.G - h->G64) * 2;
            d.E = a.E;
            d.st = a.st;
            d.partials = a.partials;
            d.counter = a.counter;
            d.dry = a.dry;
            return dispatch_ax_dfl_entry(h, lx, d, fused, s);
        }
    }
    if constexpr (std::is_same<T, double>::value) {
        if (variant == kLnVariant && bulk_supported(lx) && !a.mass) return dispatch_ax_ln_entry(h, lx, a, fused, s);
    }
    if constexpr (std::is_same<T, float>::value) {
        if (variant == kTcVariant && lx == 8) return dispatch_ax_tc(h, lx, a, fused, s);
    }
    if (variant == kDfVariant || variant == kDflVariant || variant == kTcVariant || variant == kLnVariant) variant = 0;
    a.variant = variant;
    a.err = device_error_word(h);
    a.wait_budget = h->test_stall ? 100000000LL : 4000000000LL;  // ~50 ms / ~2 s at 2 GHz
    a.tx_extra = h->test_stall ? 16u : 0u;
    const bool bulk_ok = variant > 0 && bulk_fits(lx, variant, sizeof(T) == 4) && aligned16(a.w) &&
                         (fused ? (aligned16(a.z) && aligned16(a.p)) : aligned16(a.u)) && aligned16(a.G);
    if (!bulk_ok) a.variant = 0;
    if constexpr (std::is_same<T, double>::value) {
        return bulk_ok ? dispatch_ax_bulk_f64(h, lx, a, fused, s) : dispatch_ax_f64(h, lx, a, fused, s);
    } else {
        return bulk_ok ? dispatch_ax_bulk_f32(h, lx, a, fused, s) : dispatch_ax_f32(h, lx, a, fused, s);
    }
}

int launch_ax_local(sem_handle* h, const void* u, void* w, int precision, cudaStream_t s) {
    for (int q = 0; q < h->nsolve; q++) {
        const MeshPart& p = h->parts[q];
        int rc;
        if (is_f32(precision)) {
            AxParams<float> a = {};
            a.u = (const float*)u + p.loc_off;
            a.w = (float*)w + p.loc_off;
            a.G = h->G32 + 6 * p.loc_off;
            a.D = h->D32[p.lx];
            a.E = p.E;
            a.mass = h->hmass32 ? h->hmass32 + p.loc_off : nullptr;
            rc = dispatch_variant<float>(h, p.lx, a, false, ax_variant_of_precision(h, p.lx, precision), s);
        } else {
            AxParams<double> a = {};
            a.u = (const double*)u + p.loc_off;
            a.w = (double*)w + p.loc_off;
            a.G = h->G64 + 6 * p.loc_off;
            a.D = h->D64[p.lx];
            a.E = p.E;
            a.mass = h->hmass64 ? h->hmass64 + p.loc_off : nullptr;
            rc = dispatch_variant<double>(h, p.lx, a, false, ax_variant_of_precision(h, p.lx, precision), s);
        }
        if (rc) return rc;
    }
    return SEM_OK;
}

int launch_ax_local_until_done(sem_handle* h, const double* u, double* w, const CGState* st, cudaStream_t s) {
    const MeshPart& p = h->parts[0];
    AxParams<double> a = {};
    a.u = u;
    a.w = w;
    a.G = h->G64;
    a.D = h->D64[p.lx];
    a.E = p.E;
    a.mass = h->hmass64;
    a.skip_st = st;
    return dispatch_variant<double>(h, p.lx, a, false, ax_variant_for(h, p.lx, kClsF64), s);
}

// K-A of a CG iteration on a single-mesh handle: p = z + beta p; w = A_L p;
// alpha = rho / <p, w>.
int launch_cg_pupdate_ax(sem_handle* h, int precision, cudaStream_t s) {
    const MeshPart& p = h->parts[0];
    if (is_f32(precision)) {
        AxParams<float> a = {};
        a.w = h->ws.w32;
        a.G = h->G32;
        a.D = h->D32[p.lx];
        a.E = p.E;
        a.z = h->ws.z32;
        a.p = h->ws.p32;
        a.st = h->state + 1;
        a.partials = h->partials;
        a.counter = h->counters + 2;
        a.mass = h->hmass32;
        return dispatch_variant<float>(h, p.lx, a, true, ax_variant_of_precision(h, p.lx, precision), s);
    }
    AxParams<double> a = {};
    a.w = h->ws.w;
    a.G = h->G64;
    a.D = h->D64[p.lx];
    a.E = p.E;
    a.z = h->ws.z;
    a.p = h->ws.p;
    a.st = h->state;
    a.partials = h->partials;
    a.counter = h->counters + 2;
    a.mass = h->hmass64;
    return dispatch_variant<double>(h, p.lx, a, true, ax_variant_of_precision(h, p.lx, precision), s);
}

// Set kernel attributes and cache occupancies of the CG kernels of this
// handle before any stream capture (those calls are kept out of captures).
int prepare_cg_kernels(sem_handle* h) {
    for (const MeshPart& p : h->parts) {
        for (int cls = 0; cls < 3; cls++)
            for (int fused = 0; fused < 2; fused++) {
                const int v = ax_variant_for(h, p.lx, cls);
                int rc;
                if (cls == kClsF32) {
                    AxParams<float> a = {};
                    a.dry = 1;
                    a.variant = v;
                    rc = v == kTcVariant ? dispatch_ax_tc(h, p.lx, a, fused != 0, 0)
                         : v > 0        ? dispatch_ax_bulk_f32(h, p.lx, a, fused != 0, 0)
                                        : dispatch_ax_f32(h, p.lx, a, fused != 0, 0);
                    // SEM_TC_SPLIT solves take the tensor-core kernel at lx = 8
                    if (!rc && p.lx == 8 && v != kTcVariant) {
                        a.variant = kTcVariant;
                        rc = dispatch_ax_tc(h, p.lx, a, fused != 0, 0);
                    }
                } else {
                    AxParams<double> a = {};
                    a.dry = 1;
                    a.G = h->G64;
                    if (v == kDfVariant || v == kDflVariant || v == kLnVariant) {
                        rc = dispatch_variant<double>(h, p.lx, a, fused != 0, v, 0);
                    } else {
                        a.variant = v;
                        rc = v > 0 ? dispatch_ax_bulk_f64(h, p.lx, a, fused != 0, 0)
                                   : dispatch_ax_f64(h, p.lx, a, fused != 0, 0);
                    }
                    // the plain FP64 kernel also serves SEM_FP64_NATIVE
                    if (!rc && v > 0) rc = dispatch_ax_f64(h, p.lx, a, fused != 0, 0);
                }
                if (rc) return rc;
            }
    }
    return SEM_OK;
}

// Autotuner: time every operator variant of the class that fits (shared-slab
// staging, the bulk-staged (elements per CTA, stages) configurations, the
// tensor-core form (FP32, lx = 8) and the line-transform form (native FP64,
// even lx <= 12)) on
// this handle's own factors with the plain kernel, a few launches each after a
// warm-up, and keep the fastest per order (FP32 class, or native FP64 class).
// The fused CG kernel uses the same choice.  Runs once per handle and class,
// outside any capture.  The pair class needs no timing (its line-transform
// form is the faster one wherever it applies).
int autotune_ax(sem_handle* h, bool fp32, cudaStream_t s) {
    int rc = ensure_workspace(h, fp32);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    SEM_CUDA_TRY(cudaEventCreate(&e0));
    SEM_CUDA_TRY(cudaEventCreate(&e1));
    for (const MeshPart& p : h->parts) {
        if (h->ax_variant[fp32][p.lx] >= 0) continue;
        // candidates: every variant that fits; each is warmed up, then all are
        // timed in three interleaved rounds (best round per variant), so a
        // clock ramp or a noisy launch does not decide the choice
        auto run = [&](int v, int dry) -> int {
            if (fp32) {
                AxParams<float> a = {};
                a.u = h->ws.z32 + p.loc_off;
                a.w = h->ws.w32 + p.loc_off;
                a.G = h->G32 + 6 * p.loc_off;
                a.D = h->D32[p.lx];
                a.E = p.E;
                a.dry = dry;
                a.mass = h->hmass32 ? h->hmass32 + p.loc_off : nullptr;
                return dispatch_variant<float>(h, p.lx, a, false, v, s);
            }
            AxParams<double> a = {};
            a.u = h->ws.z + p.loc_off;
            a.w = h->ws.w + p.loc_off;
            a.G = h->G64 + 6 * p.loc_off;
            a.D = h->D64[p.lx];
            a.E = p.E;
            a.dry = dry;
            a.mass = h->hmass64 ? h->hmass64 + p.loc_off : nullptr;
            return dispatch_variant<double>(h, p.lx, a, false, v, s);
        };
        std::vector<int> cand;
        for (int v = 0; v <= kLnVariant; v++) {
            if (v > kBulkVariantsMax && !(v == kTcVariant && fp32 && p.lx == 8) &&
                !(v == kLnVariant && !fp32 && bulk_supported(p.lx) && !h->hmass64))
                continue;
            if (v > 0 && v <= kBulkVariantsMax && (!bulk_fits(p.lx, v, fp32) || h->hmass64)) continue;
            if (run(v, 1)) {  // does not fit / cannot be resident: not a candidate
                set_error("");
                continue;
            }
            int rc2 = SEM_OK;
            for (int w = 0; w < 2 && !rc2; w++) rc2 = run(v, 0);
            if (rc2) return rc2;
            cand.push_back(v);
        }
        std::vector<float> best_ms(cand.size(), 1e30f);
        for (int round = 0; round < 3; round++)
            for (size_t c = 0; c < cand.size(); c++) {
                int rc2 = SEM_OK;
                cudaEventRecord(e0, s);
                for (int w = 0; w < 5 && !rc2; w++) rc2 = run(cand[c], 0);
                cudaEventRecord(e1, s);
                if (rc2) return rc2;
                SEM_CUDA_TRY(cudaEventSynchronize(e1));
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                best_ms[c] = std::min(best_ms[c], ms);
            }
        int best_v = 0;
        float best = 1e30f;
        for (size_t c = 0; c < cand.size(); c++)
            if (best_ms[c] < best) {
                best = best_ms[c];
                best_v = cand[c];
            }
        h->ax_variant[fp32][p.lx] = best_v;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return SEM_OK;
}

// w = B u
template <typename T>
__global__ void mass_kernel(const T* __restrict__ u, const double* __restrict__ B, T* __restrict__ w, int64_t n) {
    for (int64_t L = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; L < n; L += (int64_t)gridDim.x * blockDim.x)
        w[L] = (T)(B[L] * (double)u[L]);
}

int launch_mass(sem_handle* h, const double* u, double* w, cudaStream_t s) {
    mass_kernel<double><<<grid_for(h, h->n_local, 256, 8), 256, 0, s>>>(u, h->B64, w, h->n_local);
    SEM_LAUNCH_CHECK("mass_kernel");
    h->launches++;
    return SEM_OK;
}

int launch_mass32(sem_handle* h, const float* u, float* w, cudaStream_t s) {
    mass_kernel<float><<<grid_for(h, h->n_local, 256, 8), 256, 0, s>>>(u, h->B64, w, h->n_local);
    SEM_LAUNCH_CHECK("mass_kernel");
    h->launches++;
    return SEM_OK;
}

}  // namespace sem

using namespace sem;

extern "C" {

SEM_API int sem_ax(sem_handle* h, void* w, const void* u, int precision, int assemble, cudaStream_t s) {
    if (!h || !w || !u) return fail(SEM_EINVAL, "null argument");
    if (!valid_precision(precision)) return fail(SEM_EINVAL, "unknown precision");
    if (w == u) return fail(SEM_EINVAL, "w must not alias u");
    if (!aligned16(w) || !aligned16(u)) return fail(SEM_EINVAL, "u and w must be 16-byte aligned");
    int rc = launch_ax_local(h, u, w, precision, s);
    if (rc == SEM_OK && assemble) rc = launch_gs(h, w, is_f32(precision), true, s);
    return rc;
}

SEM_API int sem_mass(sem_handle* h, void* w, const void* u, int precision, int assemble, cudaStream_t s) {
    if (!h || !w || !u) return fail(SEM_EINVAL, "null argument");
    int rc;
    if (is_f32(precision))
        rc = launch_mass32(h, (const float*)u, (float*)w, s);
    else if (valid_precision(precision))
        rc = launch_mass(h, (const double*)u, (double*)w, s);
    else
        return fail(SEM_EINVAL, "unknown precision");
    if (rc == SEM_OK && assemble) rc = launch_gs(h, w, is_f32(precision), true, s);
    return rc;
}

}  // extern "C"
