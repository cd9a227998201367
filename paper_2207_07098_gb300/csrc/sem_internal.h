// Internal declarations of libsem: the handle, error plumbing, and device
// helpers shared by the translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/sem.h"

namespace sem {

constexpr int kMaxLx = 16;
constexpr int kReduceThreads = 256;
constexpr int kMaxPartials = 4096;  // upper bound on CTAs of a reducing launch
constexpr int kBulkVariantsMax = 4;  // operator variants 1..4 are bulk-staged
constexpr int kDfVariant = 5;        // FP64 data, FP32-pair arithmetic (FP64 precisions only)
constexpr int kDflVariant = 6;       // same, line-transform form with even/odd splitting (even lx)
constexpr int kMultiVariant = 7;     // batches: one slab launch over the groups of every order
constexpr int kTcVariant = 8;        // FP32 data, BF16 split-precision tensor-core contractions (lx = 8)
constexpr int kLnVariant = 9;        // native FP64, line transforms with even/odd splitting (even lx <= 12)
// operator classes, each with its own tuned or pinned variant per order:
// native FP64 (variants 0..4), FP32 (0..4), FP32-pair arithmetic on FP64 data (5, 6)
constexpr int kClsF64 = 0, kClsF32 = 1, kClsPair = 2;
// class of a sem_precision value (SEM_FP64_NATIVE: the FP64 class, variant 0)
// float data: SEM_FP32 and its tensor-core form SEM_TC_SPLIT
inline bool is_f32(int precision) { return precision == SEM_FP32 || precision == SEM_TC_SPLIT; }
inline int precision_class(int precision) {
    return is_f32(precision) ? kClsF32 : precision == SEM_FP64_PAIR ? kClsPair : kClsF64;
}
inline bool valid_precision(int precision) {
    return precision == SEM_FP64 || precision == SEM_FP32 || precision == SEM_FP64_NATIVE ||
           precision == SEM_FP64_PAIR || precision == SEM_TC_SPLIT;
}

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define SEM_CUDA_TRY(call)                                  \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return ::sem::cuda_fail(e_, #call); \
    } while (0)

#define SEM_LAUNCH_CHECK(what)                              \
    do {                                                    \
        cudaError_t e_ = cudaGetLastError();                \
        if (e_ != cudaSuccess) return ::sem::cuda_fail(e_, what); \
    } while (0)

// ---------------------------------------------------------------------------
// solver scalars living in device memory (one per solve)
// ---------------------------------------------------------------------------
struct CGState {
    double rho;       // <r, z> of the current iterate
    double rho_old;   // <r, z> of the previous iterate
    double alpha;     // step length of the current iteration
    double pap;       // <p, A p>
    double rr;        // <r, r>
    double bb;        // <b, b>
    double tol2;      // (tol * ||b||)^2 threshold on rr, set at init
    double scale;     // refinement: ||r|| of the outer residual
    int iter;         // iterations done
    int max_iter;
    int done;         // 1 once converged, failed or out of iterations
    int status;       // SEM_OK / SEM_ENOTCONV / SEM_EBREAKDOWN
    int carry;        // 1: the first iteration continues a direction p kept from an
                      // earlier solve (rho_old rescaled to match) instead of p = z
};

// ---------------------------------------------------------------------------
// one mesh (a handle holds one, or many for a batch)
// ---------------------------------------------------------------------------
struct MeshPart {
    int E = 0;
    int lx = 0;
    int64_t elem_off = 0;  // first element in the handle's element numbering
    int64_t loc_off = 0;   // first local index
    int64_t n_local = 0;
    int64_t n_unique = 0;
    int64_t n_free = 0;
};

// Gather-scatter lists.  Every node with >= 2 copies is one segment whose
// local indices are listed in ascending order.  Segments of free nodes are
// split by size (2, 4, 8 copies: index vectors; any other count: CSR) and
// ordered by their first local index; segments of Dirichlet nodes are kept as
// CSR (they are only summed when the mask is not applied); `zero` lists every
// local copy of every Dirichlet node.
// Per-segment solve of a batch (index into the CG states) for each segment
// class; a gather-scatter given these and the states skips the segments of
// converged solves.  sid == nullptr: no skipping.
struct GsSkip {
    const uint16_t* sid[5] = {};  // pairs, quads, octets, other sizes, Dirichlet zero list
    const struct CGState* st = nullptr;
    // single-mesh CG loop: the whole launch returns at once when this solve
    // is done (a graph launch runs past the end of the solve; its operator and
    // update kernels return at once too, and A p is recomputed before use)
    const struct CGState* done_st = nullptr;
};

struct GSLists {
    int2* pairs = nullptr;
    int4* quads = nullptr;
    int4* octs = nullptr;      // two int4 per segment
    int* oth_off = nullptr;    // [noth + 1]
    int* oth_idx = nullptr;
    int* dir_off = nullptr;    // [ndir + 1]
    int* dir_idx = nullptr;
    int* zero_idx = nullptr;   // [nzero]
    int64_t npair = 0, nquad = 0, noct = 0, noth = 0, ndir = 0, nzero = 0;
    int64_t n_shared = 0;      // local points in segments
};

struct Workspace {
    // FP64 CG vectors
    double* r = nullptr;
    double* p = nullptr;
    double* z = nullptr;
    double* w = nullptr;
    double* x = nullptr;
    double* b = nullptr;
    // FP32 inner vectors
    float* r32 = nullptr;
    float* p32 = nullptr;
    float* z32 = nullptr;
    float* w32 = nullptr;
    float* d32 = nullptr;
    float* b32 = nullptr;
    // FP64 mode in pair form: x, p, r, w, z (hi, lo planes each), Minv (hi, lo)
    float* pv[12] = {};
    // pipelined CG: u, w, m, n, z, q, s, p (FP64)
    double* pipe[8] = {};
    bool have64 = false, have32 = false;
};

// Work lists of a batch handle (device arrays).
//  * K-A groups: for every order lx present, EPC(lx) consecutive elements of one
//    solve per group; groups of a solve are contiguous.  A group's partial sum
//    goes to gpart[global group index].
//  * point tiles: up to kTile consecutive local points of one solve, for the
//    vector updates and reductions; partials tpart[tile][3].
struct LxGroups {
    int lx = 0;
    int64_t ngroups = 0;
    int64_t goff = 0;         // global index of this list's first group
    int64_t* loc = nullptr;   // [ngroups] local index of the group's first element
    int* cnt = nullptr;       // [ngroups] elements in the group
    int* solve = nullptr;     // [ngroups]
};

struct BatchPlan {
    std::vector<LxGroups> lxg;
    int64_t ngroups = 0;
    int* sgfirst = nullptr;   // [nsolve] first global group of the solve
    int* sgcount = nullptr;   // [nsolve]
    int64_t ntiles = 0;
    int64_t* tloc = nullptr;  // [ntiles]
    int* tlen = nullptr;      // [ntiles]
    int* tsolve = nullptr;    // [ntiles]
    int* stfirst = nullptr;   // [nsolve]
    int* stcount = nullptr;   // [nsolve]
    double* gpart = nullptr;  // [ngroups]
    double* tpart = nullptr;  // [ntiles * 3]
    unsigned int* scount = nullptr;  // [nsolve] per-solve ticket counters
    double* rrbb = nullptr;   // [nsolve * 2]
    int* act = nullptr;       // [nsolve] solves taking part in an inner solve
    double* itol = nullptr;   // [nsolve] inner relative tolerance of each active solve
    double* carry = nullptr;  // [nsolve] refinement: rescaling of the kept direction (0 = restart)
    // the slab groups above as one list for the multi-order launch (same global
    // group numbering): local index, element count, solve and order of each group
    int64_t* uloc = nullptr;
    int* ucnt = nullptr;
    int* usolve = nullptr;
    uint8_t* ulx = nullptr;
    bool multi_ok = false;    // every order present is within the multi-order kernel's range
    // operator configuration per class [kClsF64 / kClsF32]: 1 = one multi-order
    // launch, 0 = one launch per order with ovar[cls][lx] (0 slab, 1..4 bulk-staged,
    // FP32 only), -1 = not chosen yet (autotuned at the first solve)
    int kcfg[2] = {-1, -1};
    int ovar[2][kMaxLx + 1] = {};
    // group lists cut to the element count of a bulk-staged variant, per
    // elements-per-CTA (index 0: 1, 1: 2, 2: 4); built when first needed
    struct BulkSet {
        std::vector<LxGroups> lists;  // one per order present, in lxg's order
        int64_t ngroups = 0;
        int* sgfirst = nullptr;   // [nsolve]
        int* sgcount = nullptr;   // [nsolve]
        double* gpart = nullptr;  // [ngroups]
        bool built = false;
    } bulk[3];
    // solve of every gather-scatter segment (batches of at most 65535 solves)
    uint16_t* sid[5] = {};
    bool sid_ready = false;
    bool ready = false;
};

constexpr int kTile = 4096;

// sqrt(rr / bb) of a true residual: NaN when either norm is not finite (a
// non-finite right-hand side or iterate), 0 for a zero right-hand side.
inline double relative_residual(double rr, double bb) {
    if (!std::isfinite(rr) || !std::isfinite(bb)) return NAN;
    return bb > 0 ? std::sqrt(rr / bb) : 0.0;
}

// Projection space of a single-mesh handle (sem_proj.cu): L slots of
// A-orthonormal xt_i and bt_i = A xt_i, l of them in use, the last start xbar.
struct ProjSpace {
    int L = 0;
    int l = 0;
    int64_t ld = 0;               // leading dimension of xt, bt (n_local rounded up to 4)
    double* xt = nullptr;         // [L][ld]
    double* bt = nullptr;         // [L][ld]
    double* xbar = nullptr;       // [n_local]
    double* coef = nullptr;       // [L + 2] coefficients of the current projection
    double* gpart = nullptr;      // Gram-Schmidt block partials
    unsigned int* gcount = nullptr;
};

// Assembled coarse matrix of the Schwarz preconditioner (sem_coarse.cu): CSR
// over the free unique corner nodes, its Jacobi inverse, every row's
// element-corner copies, the CG vectors (x, r, z, p0, p1, q per precision),
// the solution at the element corners, and the CG scalars
struct CoarseCsr {
    int nc = 0;
    int* rowptr = nullptr;
    int* col = nullptr;
    double* val64 = nullptr;
    float* val32 = nullptr;
    double* dinv64 = nullptr;
    float* dinv32 = nullptr;
    int* gptr = nullptr;  // [nc + 1]
    int* gidx = nullptr;  // element-corner copies of the rows
    void* vec[2] = {};    // FP64, FP32: [6][nc]
    void* xl[2] = {};     // FP64, FP32: the solution at the element corners [E][8]
    double* st = nullptr;
    double* partials = nullptr;
    unsigned int* counter = nullptr;
    unsigned int* bar = nullptr;  // grid barrier of the cooperative form: arrivals, generation
};
int build_coarse_csr(sem_handle* h, const int64_t* cgid, const uint8_t* cmask);
void free_coarse_csr(CoarseCsr& cc);
template <typename T>
int coarse_csr_solve(sem_handle* h, const T* rc_local, int iters, bool coop,
                     cudaStream_t s);  // iters Jacobi-PCG from 0; coop: one cooperative launch
template <typename T>
const T* coarse_csr_x(const sem_handle* h);

// Two-level Schwarz preconditioner and FGMRES storage (sem_gmres.cu; built
// at set-up with SEM_FLAG_SCHWARZ, single-mesh handles)
struct SchwarzData {
    sem_handle* coarse = nullptr;  // the same elements at lx = 2 on their corner nodes
    double* fac = nullptr;         // [E][6] sqrt(2 / L_d), h1m 4 / L_d^2 (box lengths L_d, mean h1)
    float* fac32 = nullptr;
    double* S = nullptr;           // [(lx-2)^2] interior modes of the reference element (node major)
    double* lam = nullptr;         // [lx-2] their eigenvalues
    double* Pw = nullptr;          // [lx^3][8] trilinear weights of the corners at the GLL nodes
    float* S32 = nullptr;          // FP32 copies of S, lam, Pw, fac (FP32 preconditioner arithmetic)
    float* lam32 = nullptr;
    float* Pw32 = nullptr;
    int m = 0;                     // FGMRES restart length of the storage below
    int elem = 0;                  // bytes per entry of V and Z (8 FP64, 4 mixed)
    int64_t ld = 0;                // their leading dimension (n_local rounded up to 4)
    void* V = nullptr;             // [m + 1][n_local] Arnoldi basis
    void* Z = nullptr;             // [m][n_local] preconditioned basis
    double* coef = nullptr;        // Gram-Schmidt coefficients, norm and y on the device
    double* gpart = nullptr;       // Gram-Schmidt block partials
    unsigned int* gcount = nullptr;
    CoarseCsr csr;                 // the assembled coarse problem
    cudaStream_t aux = nullptr;    // the coarse CG's stream (beside the local solves)
    cudaEvent_t ev_restrict = nullptr, ev_coarse = nullptr;
};

// What the CG loop reads back after each graph launch, in one pinned block.
struct LoopReadback {
    CGState st;
    int err;
};

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    int key_prec = -1;
    int key_chunk = 0;
    int key_variant = -1;
    const void* key_ptr = nullptr;
};

}  // namespace sem

struct sem_handle {
    int device = 0;
    int sm_count = 0;
    int nsolve = 1;
    int E = 0;           // total elements
    int lx = 0;          // common lx (0 for a mixed-order batch)
    int64_t n_local = 0;
    int64_t n_unique = 0;
    int64_t n_free = 0;
    std::vector<sem::MeshPart> parts;
    // basis per lx (index lx): D in FP64 and FP32
    double* D64[sem::kMaxLx + 1] = {};
    float* D32[sem::kMaxLx + 1] = {};
    float* D2[sem::kMaxLx + 1] = {};   // [2][lx][lx]: hi and lo floats of D
    // set-up data
    double* G64 = nullptr;     // [E][6][lx^3], h1 folded in
    float* G32 = nullptr;
    float* G2 = nullptr;       // [E][12][lx^3]: hi planes then lo planes of G64 (FP32-pair kernel)
    double* B64 = nullptr;     // [n_local] mass
    double* minv64 = nullptr;  // [n_local]
    double* hmass64 = nullptr; // [n_local] Helmholtz mass term h2 B (null: Poisson operator)
    double* drdx = nullptr;    // [E][9][lx^3] dr_s/dx_l (SEM_FLAG_METRICS; gradient operators)
    float* hmass32 = nullptr;
    float* minv32 = nullptr;
    uint8_t* mult = nullptr;   // [n_local] copies of the node
    uint8_t* mask = nullptr;   // [n_local]
    sem::GSLists gs;
    // reductions and solver state
    double* partials = nullptr;       // [kMaxPartials * 4]
    unsigned int* counters = nullptr; // [16]
    sem::CGState* state = nullptr;       // [2 nsolve + 2]: solve / outer states, then inner states
    sem::CGState* state_host = nullptr;  // pinned mirror
    sem::LoopReadback* loop_host = nullptr;  // pinned: the CG loop's state and error word, read with one sync
    double* scratch = nullptr;        // [64] small device scratch
    sem::Workspace ws;
    sem::GraphCache graph;
    sem::GraphCache graph_tail;  // kTailChunk iterations, no timing events: the predicted end of a CG run
    sem::ProjSpace proj;
    sem::SchwarzData sch;
    sem::BatchPlan batch;
    cudaStream_t capture_stream = nullptr;
    cudaEvent_t ax_ev[2] = {nullptr, nullptr};  // bracket one K-A per graph (single: 2nd, batch: 1st)
    int64_t launches = 0;                        // kernels launched by this handle
    int test_stall = 0;                          // SEM_FLAG_TEST_STALL: bulk copies never complete a stage
    int ax_variant[3][sem::kMaxLx + 1];          // tuned or pinned operator variant per [class][lx], -1 = not tuned
    size_t device_bytes = 0;
};

namespace sem {

// allocation helper that records bytes in the handle
template <typename T>
int dalloc(sem_handle* h, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return SEM_OK;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(SEM_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    h->device_bytes += count * sizeof(T);
    return SEM_OK;
}

int ensure_workspace(sem_handle* h, bool fp32);

// ---- launches implemented in the .cu files (all enqueue on `s`) ----------
// ax: w = A_L u (local).  T = double or float.  `native` selects the plain
// FP64 kernel for double.
int launch_ax_local(sem_handle* h, const void* u, void* w, int precision, cudaStream_t s);
// gs (+ mask)
int launch_gs(sem_handle* h, void* u, bool fp32, bool apply_mask, cudaStream_t s);
// masked QQ^T of a batch that leaves the segments of solves already done
int launch_gs_skip(sem_handle* h, void* u, bool fp32, const GsSkip& skip, cudaStream_t s);
// QQ^T + mask that returns at once when the CG state `st` is done (CG loop)
int launch_gs_until_done(sem_handle* h, void* u, bool fp32, const CGState* st, cudaStream_t s);
// w = B u
int launch_mass(sem_handle* h, const double* u, double* w, cudaStream_t s);
int launch_mass32(sem_handle* h, const float* u, float* w, cudaStream_t s);
// fused CG pieces
int launch_cg_pupdate_ax(sem_handle* h, int precision, cudaStream_t s);   // K-A
int launch_cg_update(sem_handle* h, int precision, cudaStream_t s);       // K-C
int launch_cg_init(sem_handle* h, int precision, cudaStream_t s);         // z, rho, rr, bb
int launch_dot(sem_handle* h, const double* a, const double* b, double* out, cudaStream_t s);
int launch_residual(sem_handle* h, const double* b, const double* ax, double* r,
                    double* rr_out, cudaStream_t s);  // r = b - ax, rr_out[0] = <r,r>
int grid_for(sem_handle* h, int64_t work_items, int threads, int per_sm);
int prepare_cg_kernels(sem_handle* h);
// FP64 CG with float-pair vectors (sem_cg_pair.cu)
constexpr int kPairPrec = 100;  // "precision" code of the pair-form CG loop
constexpr int kPipePrec = 101;  // "precision" code of the pipelined CG loop (sem_cg_pipe.cu)
int ensure_pipe_workspace(sem_handle* h);
int launch_pipe_init(sem_handle* h, double tol, int max_iter, cudaStream_t s);
int launch_pipe_iteration(sem_handle* h, cudaStream_t s);
// residual replacement of a pipelined solve in progress (ws.r = b - A x already
// computed): the recurrence vectors recomputed from x and p, seg more iterations
int launch_pipe_replace(sem_handle* h, int seg, cudaStream_t s);
constexpr int kPipeSeg = 50;  // pipelined iterations between residual replacements
// native FP64 w = A_L u that returns at once when st->done (inside CG graphs)
int launch_ax_local_until_done(sem_handle* h, const double* u, double* w, const CGState* st, cudaStream_t s);
bool pair_cg_available(const sem_handle* h);
int ensure_pair_workspace(sem_handle* h);
int refresh_pair_minv(sem_handle* h, cudaStream_t s);
// projection onto previous solutions (sem_proj.cu)
int proj_start(sem_handle* h, int max_vectors, cudaStream_t s);
int proj_update(sem_handle* h, cudaStream_t s);
void free_projection(sem_handle* h);
// two-level Schwarz + FGMRES (sem_gmres.cu)
void free_schwarz(sem_handle* h);
int solve_gmres(sem_handle* h, double* x_user, const double* b_user, const sem_solve_opts& o,
                sem_solve_stats* stats, cudaStream_t s);
// pieces of the CG driver used by other solvers (sem_cg.cu)
int true_residual(sem_handle* h, const double* x, const double* b, double* rr_bb, cudaStream_t s);
bool host_resident(const void* p);
int launch_pair_split_x(sem_handle* h, cudaStream_t s);
int launch_pair_join_x(sem_handle* h, cudaStream_t s);
int launch_pair_init(sem_handle* h, double tol, int max_iter, cudaStream_t s);
int launch_pair_ka(sem_handle* h, cudaStream_t s);
int launch_pair_rest(sem_handle* h, cudaStream_t s);
int prepare_pair_kernels(sem_handle* h);
int autotune_ax(sem_handle* h, bool fp32, cudaStream_t s);
// whole CG in one cooperative launch (sem_cg_persist.cu): single-mesh handles, lx <= 10
constexpr int kPersistMaxLx = 10;
constexpr int64_t kPersistAutoPoints = (int64_t)1 << 20;  // automatic below this many local points
bool persist_available(const sem_handle* h);
int launch_cg_persist(sem_handle* h, int precision, int slot, cudaStream_t s);
// operator variant of class cls (kClsF64 / kClsF32 / kClsPair) for order lx
int ax_variant_for(const sem_handle* h, int lx, int cls);
// variant a precision uses for order lx (SEM_FP64_NATIVE: 0)
int ax_variant_of_precision(const sem_handle* h, int lx, int precision);
int* device_error_word(sem_handle* h);
double inner_tolerance(const sem_solve_opts& o, double rel);

}  // namespace sem
