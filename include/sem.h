/*
 * sem.h -- C ABI of libsem, a GB300 (sm_103a) library for the
 * spectral-element pressure-Poisson solve of Karp et al., "Large-Scale Direct
 * Numerical Simulations of Turbulence Using GPUs and Modern Fortran"
 * (arXiv 2207.07098).
 *
 * The library solves  mask * QQ^T A_L x = b  where
 *   A_L   is the block-diagonal matrix of the element operators
 *         A^e = D^T G^e D, scaled by a coefficient h1 at every quadrature
 *         point (Sec. II-A, eq. "disclap" and the definitions of D and G^e
 *         below it; h1 as in the Helmholtz operator of the same section),
 *   QQ^T  is the gather-scatter (direct-stiffness summation) over nodes that
 *         several elements share (Sec. II-A, "QQ^T A_L u_L = A u_L"),
 *   mask  zeroes homogeneous Dirichlet nodes,
 * with Jacobi-preconditioned conjugate gradients (Sec. II-B, P-CG), in FP64
 * or with FP64 iterative refinement around an FP32 inner CG.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Local vectors have n_L = E * lx^3 entries in element-major layout
 *   [e][k][j][i] (i fastest), lx = N + 1 GLL points per direction.  For a
 *   batch handle, the local vectors of all solves are concatenated in solve
 *   order.
 * - Vector arguments of sem_ax, sem_gs, sem_mass, sem_dot and the getters are
 *   DEVICE pointers (e.g. torch tensors' data_ptr()) of the element type that
 *   the precision argument names (double for SEM_FP64, float otherwise),
 *   16-byte aligned.  sem_cg_solve and sem_cg_solve_batch accept host or
 *   device pointers for x and b (host buffers are copied in and out inside
 *   the call).  Set-up arrays (coordinates, ids, mask, h1) are HOST pointers.
 * - The caller owns every pointer it passes; the handle owns everything the
 *   library allocates (geometric factors, preconditioner, gather-scatter
 *   lists, solver work vectors) and sem_destroy frees it.
 * - All work is enqueued on the given stream (0 = legacy default stream).
 *   Calls that return results to the host (sem_cg_solve*) synchronise it.
 * - Every call returns a sem_status.  On failure sem_last_error() returns a
 *   message for the calling thread.  A handle is not thread-safe: calls on
 *   one handle must be serialised by the caller.
 */
#ifndef SEM_H
#define SEM_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SEM_API __attribute__((visibility("default")))

/* Opaque handle: one mesh (sem_setup) or a batch of meshes (sem_setup_batch)
 * with everything the library derived from it. */
typedef struct sem_handle sem_handle;

typedef enum sem_status {
    SEM_OK = 0,
    SEM_EINVAL = 1,       /* bad argument, mesh or alignment */
    SEM_ENOMEM = 2,       /* device or host allocation failed */
    SEM_ECUDA = 3,        /* a CUDA runtime call failed */
    SEM_ENOTCONV = 4,     /* max iterations reached; outputs are valid iterates */
    SEM_EBREAKDOWN = 5,   /* p^T A p <= 0 or a non-finite scalar in CG */
    SEM_ESTAGNATE = 6,    /* refinement step failed to halve the FP64 residual */
    SEM_ETIMEOUT = 7      /* a bounded device-side wait expired */
} sem_status;

/* Arithmetic of one operator application or of the inner solve. */
typedef enum sem_precision {
    SEM_FP64 = 0,        /* double data, FP64 arithmetic (unit roundoff 2^-53): the fastest of
                            the native FP64 kernels (variants 0..4 and 9, autotuned per handle); holds
                            the 1e-12 relative parity bar on every input tested, including
                            smooth fields whose sums cancel */
    SEM_FP32 = 1,        /* float data, FP32 arithmetic and accumulation */
    SEM_FP64_NATIVE = 2, /* double data, the plain shared-slab FP64 kernel (variant 0) */
    SEM_FP64_PAIR = 3,   /* double data, FP32-pair ("double-float") arithmetic on the FP32 pipe:
                            48 significant bits, unit roundoff 2^-48, about 4x the speed of
                            SEM_FP64 on GB300 (whose FP64 pipe runs at 1/64 of the FP32 rate).
                            Relative error vs exact FP64: ~1e-15..1e-14 on rough fields, up to
                            a few 1e-12 where the element sums cancel (smooth fields), always
                            within 64 * 2^-48 |D^T||h1 G||D||u| pointwise.  Range: inputs are
                            split into two floats, so |u| below 2^-75 or at or above 2^128 (and
                            Inf/NaN) is read as 0; the solver rescales x and b by a power of two
                            to keep them inside it.  Variant 6 (line transforms, even lx <= 12)
                            or 5 (lx <= 12); other orders fall back to SEM_FP64 */
    SEM_TC_SPLIT = 4     /* float data, the FP32 operator with its D and D^T contractions on
                            the tensor cores: u, D (and the weighted derivatives) split into
                            three BF16 slices each, the six slice products of weight >= 2^-16
                            formed by warp-level mma.sync with FP32 accumulation, the G
                            weighting in FP32 (variant 8; lx = 8, other orders fall back to
                            SEM_FP32).  Same accuracy class as SEM_FP32 */
} sem_precision;

typedef enum sem_solve_mode {
    SEM_MODE_FP64 = 0,     /* plain FP64 Jacobi-PCG */
    SEM_MODE_MIXED_IR = 1, /* FP64 refinement around an FP32 inner Jacobi-PCG */
    SEM_MODE_GMRES = 2     /* the paper's pressure solver (Sec. II-B): restarted flexible GMRES
                              with a two-level additive Schwarz preconditioner (element-interior
                              fast-diagonalisation solves, point Jacobi on inter-element nodes,
                              a coarse grid on the element corners solved by 10 Jacobi-PCG
                              iterations); handles set up with SEM_FLAG_SCHWARZ.  precision
                              SEM_FP64 / SEM_FP64_NATIVE (native FP64 operator) or SEM_FP64_PAIR:
                              FP64 Krylov vectors, the true residual checked at every restart.
                              precision SEM_FP32: mixed form, every restart cycle an FP32
                              flexible GMRES solve (operator, preconditioner, basis in FP32) of
                              A d = r for the true FP64 residual r, x += d in FP64; a cycle stops
                              at inner_tol of its start residual or at gmres_restart steps */
} sem_solve_mode;

typedef struct sem_info {
    int nsolve;              /* 1 for sem_setup, number of meshes for a batch */
    int E;                   /* elements (sum over the batch) */
    int lx;                  /* points per direction (0 for a mixed-order batch) */
    int64_t n_local;         /* local points E * lx^3 (sum over the batch) */
    int64_t n_unique;        /* distinct global nodes */
    int64_t n_free;          /* distinct global nodes with mask = 1 */
    int64_t n_shared;        /* local points that belong to a node with >= 2 copies */
    size_t device_bytes;     /* device memory held by the handle */
} sem_info;

typedef struct sem_solve_opts {
    double tol;          /* relative residual ||b - A x|| / ||b|| to reach (1e-10) */
    int max_iter;        /* max CG iterations (FP64 mode) or inner iterations per
                            refinement step (mixed mode).  In mixed mode a step that stops at
                            this cap is not judged for stagnation, and with ir_carry its
                            direction is kept: with ir_carry = 1, max_iter ~100-200 bounds the
                            iterations between residual replacements (ill-conditioned
                            problems) */
    int mode;            /* sem_solve_mode */
    double inner_tol;    /* mixed mode: inner relative tolerance (1e-5; with ir_carry = 1,
                            about 1e-2) */
    int max_outer;       /* mixed mode: max refinement steps (100) */
    int precision;       /* FP64 mode: operator of the CG iterations, SEM_FP64 (default),
                            SEM_FP64_NATIVE or SEM_FP64_PAIR (with SEM_FP64_PAIR the CG vectors
                            are float pairs too where variant 6 applies).  The true residual
                            that decides convergence is always computed with SEM_FP64 */
    int use_graph;       /* capture the CG iterations in CUDA graphs (1) */
    int graph_chunk;     /* CG iterations per graph launch between host checks (32).  Mixed
                            mode: a refinement step after the first predicts its length from
                            the step before and, once fewer than graph_chunk iterations remain
                            by that count, launches graphs of 4 iterations instead (the
                            iterates are the same) */
    int autotune;        /* time the operator-kernel variants on this handle's data at the
                            first solve of each precision and keep the fastest (1) */
    int ir_carry;        /* mixed mode: from the second refinement step on, the inner CG
                            keeps its search direction (rescaled to the new residual)
                            instead of restarting from p = z, i.e. it continues as CG whose
                            residual was replaced by the true FP64 one (residual
                            replacement).  With frequent replacements (inner_tol ~1e-2) the
                            inner iterations then add up to about the FP64 PCG count on
                            moderately conditioned problems (32^3 deformed cube: 1511
                            against 1779 restarted at 1e-5, solve 14% faster; 256-box
                            batch 13% faster).  When many iterations pass between
                            replacements (tight inner_tol, or an ill-conditioned problem:
                            the 25 M-point periodic annulus, 24% slower) the replaced
                            residual differs too much from the recursive one and
                            restarting is faster, hence the default (0) */
    int persistent;      /* run each CG loop as ONE persistent (cooperative) launch whose CTAs
                            meet at bounded grid barriers, instead of graphs of three launches
                            per iteration: 1 always, -1 below 2^20 local points, 0 never (the
                            default: on the 32 K-point cube the graph loop is as fast or faster,
                            2.2 against 2.8 ms FP64, 3.1 against 3.1 ms mixed, because each
                            phase is bound by dependent-load latency, not by launches).
                            Single-mesh handles, lx <= 10, SEM_FP32 inner solves and SEM_FP64 /
                            SEM_FP64_NATIVE (slab operator); not for SEM_FP64_PAIR.  GMRES mode:
                            nonzero runs the coarse CG of the Schwarz preconditioner as one
                            cooperative launch with bounded grid barriers */
    int tc_split;        /* mixed mode: the inner FP32 CG applies the operator as SEM_TC_SPLIT
                            (tensor-core contractions) instead of the CUDA-core FP32 kernels (0) */
    int gmres_restart;   /* GMRES mode: Krylov vectors per restart cycle (20) */
    int pipelined;       /* FP64 mode: pipelined PCG (Ghysels and Vanroose 2014; the paper's
                            work on reducing communication in CG, Sec. II-B): the PCG iterates
                            with one reduction phase per iteration instead of two, at the cost
                            of more vector traffic; native FP64 operator (0 = standard PCG) */
    int projection;      /* projection onto previous solutions (Sec. II-B, after Fischer
                            1998): 0 (default) off; L in 1..64: the solve starts from the
                            A-orthogonal projection of its solution onto the space of earlier
                            solution increments kept by the handle (the x passed in is then
                            ignored), and a converged solve adds its increment, A-orthonormalised;
                            a full space (L vectors) restarts from the latest solution, as the
                            paper's GPU runs reset theirs every 20 solves.  Single-mesh handles; the space
                            (2 L + 1 FP64 vectors) stays with the handle until
                            sem_projection_reset or sem_destroy */
    int precond_precision; /* GMRES mode with an FP64 precision: arithmetic of the Schwarz
                            preconditioner's local solves, restriction and prolongation,
                            SEM_FP64 (default) or SEM_FP32 (FP32 arithmetic on the FP64 vectors;
                            the coarse CG stays FP64).  Flexible GMRES accepts any
                            preconditioner: this changes iteration counts, not the accuracy
                            the solve reaches */
    int gmres_orth;      /* GMRES mode: orthogonalisation of the Arnoldi basis.  2 (default):
                            classical Gram-Schmidt twice, the second pass lagged into the next
                            step, so every step reads the basis twice (dots, then one combined
                            update; Swirydowicz et al. 2021); 3: classical Gram-Schmidt twice
                            within each step (three passes over the basis); 1: once (two
                            passes, less orthogonality; the true residual at each restart still
                            decides convergence) */
} sem_solve_opts;

typedef struct sem_solve_stats {
    int status;               /* sem_status of this solve */
    int iterations;           /* CG iterations (all inner iterations in mixed mode) */
    int outer_iterations;     /* refinement steps (0 in FP64 mode) */
    double relres;            /* TRUE residual ||b - A x|| / ||b||, recomputed with the
                                 SEM_FP64 operator (native FP64 arithmetic) */
    double relres_recursive;  /* last recursive residual estimate of the CG loop */
    double time_ms;           /* device time of the solve (CUDA events) */
    int64_t kernel_launches;  /* kernels this solve launched (graph nodes included) */
    double ax_ms;             /* mean duration of the fused p-update + ax_helm kernel, sampled
                                 with CUDA events once per graph launch (0 if not sampled) */
    int ax_samples;           /* number of such samples */
    int ax_variant;           /* operator kernel used by the CG loop: 0 = shared-slab staging,
                                 1..4 = bulk-copy staging (elements per CTA, stages) =
                                 (1,3), (2,2), (2,3), (4,2), lx in {4,6,8,10,12};
                                 5 = FP64 data in FP32-pair arithmetic (lx <= 12);
                                 6 = as 5 with even/odd line transforms (even lx <= 12);
                                 5 and 6 serve SEM_FP64_PAIR only;
                                 7 (batches) = one slab launch over the element groups
                                 of every order (orders up to lx = 10);
                                 8 = BF16 split-precision tensor-core contractions for
                                 FP32 data (SEM_TC_SPLIT; lx = 8; an FP32 autotuning
                                 candidate);
                                 9 = native FP64 with even/odd line transforms (even
                                 lx <= 12; an FP64 autotuning candidate, not for
                                 Helmholtz handles) */
    double relres_start;      /* true relative residual of the start (after projection, when on) */
    int launches_per_iteration;  /* kernel launches of one CG iteration: 3 for one mesh
                                 (operator, gather-scatter, update), 0 when the CG ran
                                 as one persistent launch, -1 for GMRES; for a batch the
                                 operator launches (1 with variant 7, else one per
                                 order) + 2 */
} sem_solve_stats;

/* Mesh of one member of a batch (host pointers; see sem_setup). */
typedef struct sem_mesh_desc {
    int E;
    int lx;
    const double* coords;   /* [3][E][lx^3] */
    const int64_t* gid;     /* [E lx^3] */
    const uint8_t* mask;    /* [E lx^3] */
    const double* h1;       /* [E lx^3] or NULL for h1 = 1 */
} sem_mesh_desc;

/* Set-up flag: pin operator kernel variant v: 0..4 for SEM_FP64 and SEM_FP32,
 * 5 or 6 for SEM_FP64_PAIR, 8 for SEM_FP32, 9 for SEM_FP64 (the other
 * precisions stay autotuned). */
#define SEM_FLAG_VARIANT(v) ((int)(((v) + 1) & 0xF))

/* Set-up flag for testing failure detection: the bulk-staged operator kernels
 * announce 16 bytes more than they copy, so no stage ever completes, and the
 * first CTA of the persistent CG kernel leaves before its first grid barrier;
 * the bounded waits (shortened to ~50 ms) expire, the kernels record the
 * failure and return, and the solve reports SEM_ETIMEOUT.  No fault, no hang. */
#define SEM_FLAG_TEST_STALL 0x100

/* Set-up flag: also keep the metric terms dr_s/dx_l per point (9 doubles per
 * local point) for the gradient, divergence and curl operators and the
 * pressure right-hand side (sem_grad, sem_div, sem_curl, sem_pressure_rhs). */
#define SEM_FLAG_METRICS 0x200

/* Set-up flag (sem_setup only): build the two-level Schwarz preconditioner of
 * the GMRES pressure solve (SEM_MODE_GMRES): box lengths and mean h1 of every
 * element, a coarse handle on the element corners (lx = 2), the interior
 * modes of the reference element. */
#define SEM_FLAG_SCHWARZ 0x400

/* Fill *opts with the defaults listed above. */
SEM_API void sem_solve_opts_default(sem_solve_opts* opts);

/* Message of the last failed call on this thread ("" if none). */
SEM_API const char* sem_last_error(void);

/* GLL nodes xi[lx], weights rho[lx] and derivative matrix D[lx*lx]
 * (D[i*lx+j] = l_j'(xi_i)) on [-1,1] (Sec. II-A: GLL points xi_i and the
 * differentiation matrix D).  Host pointers; any may be NULL.
 * 2 <= lx <= 16, else SEM_EINVAL. */
SEM_API int sem_gll(int lx, double* xi, double* rho, double* D);

/* Build a handle for one mesh (Sec. II-A).
 *   E       number of hexahedral elements (>= 1)
 *   lx      points per direction, 2..16
 *   coords  HOST [3][E][lx^3] node coordinates x, y, z
 *   gid     HOST [E lx^3] global node ids: equal ids <=> same node (this is Q)
 *   mask    HOST [E lx^3] 0 on homogeneous Dirichlet nodes, 1 elsewhere
 *   h1      HOST [E lx^3] coefficient at every node, or NULL for h1 = 1
 *   flags   0, or SEM_FLAG_VARIANT(v) to pin the operator kernel variant v
 *           (see sem_solve_stats.ax_variant) instead of autotuning it;
 *           variants a kernel does not cover fall back to 0
 * Computes on the device the geometric factors G_st = rho rho rho J
 * sum_l dr_s/dx_l dr_t/dx_l (h1 folded in), the mass B = rho rho rho J and
 * the Jacobi diagonal, and on the host the gather-scatter lists.
 * Errors: SEM_EINVAL for bad sizes, a mask that differs between copies of
 * a node, or a non-positive Jacobian; SEM_ENOMEM; SEM_ECUDA.  On error *h is
 * NULL and nothing is leaked.  Synchronises the stream. */
SEM_API int sem_setup(sem_handle** h, int E, int lx, const double* coords,
                      const int64_t* gid, const uint8_t* mask, const double* h1,
                      int flags, cudaStream_t stream);

/* Build one handle for nsolve independent meshes (orders may differ).
 * Global ids are local to each mesh.  Same errors as sem_setup. */
SEM_API int sem_setup_batch(sem_handle** h, int nsolve, const sem_mesh_desc* meshes,
                            int flags, cudaStream_t stream);

/* Free everything the handle owns.  NULL is accepted. */
SEM_API int sem_destroy(sem_handle* h);

/* Sizes and memory of a handle. */
SEM_API int sem_get_info(const sem_handle* h, sem_info* info);

/* Per-solve local offsets of a batch handle: offsets[s] = first local index
 * of solve s, offsets[nsolve] = n_local (host array of nsolve+1 entries). */
SEM_API int sem_get_offsets(const sem_handle* h, int64_t* offsets);

/* Turn the handle's operator into the Helmholtz operator of the velocity
 * solve (Sec. II-A: the implicit viscous term of the P_N-P_N splitting gives
 * a Helmholtz equation; Sec. II-B solves it with P-CG):
 *   A_L u = D^T (h1 G) D u + h2 B u,  B = rho rho rho J (diagonal GLL mass),
 * h1 as given at set-up (typically 1/Re), h2 per point (typically gamma_0/dt).
 *   h2  HOST [n_local] finite, >= 0 (for a batch: all meshes concatenated),
 *       or NULL to return to the Poisson operator
 * Every later sem_ax and solve on the handle uses it, and the Jacobi
 * preconditioner becomes Minv = mask / QQ^T (diag(A_L) + h2 B).  With h2 > 0
 * the operator is SPD without Dirichlet nodes.  While a Helmholtz term is set
 * the operator runs on the shared-slab kernels (or the tensor-core kernel for
 * SEM_TC_SPLIT): SEM_FP64_PAIR falls back to SEM_FP64 and the bulk-staged
 * variants to the slab kernel.  Errors: SEM_EINVAL (negative or
 * non-finite h2, device pointer), SEM_ENOMEM, SEM_ECUDA.  Synchronises the
 * stream. */
SEM_API int sem_set_helmholtz(sem_handle* h, const double* h2, cudaStream_t stream);

/* w = A_L u (assemble = 0) or w = mask * QQ^T A_L u (assemble = 1)
 * (Sec. II-A, eq. disclap and A = QQ^T A_L).  u, w: device [n_local] of the
 * precision's type; w must not alias u. */
SEM_API int sem_ax(sem_handle* h, void* w, const void* u, int precision, int assemble,
                   cudaStream_t stream);

/* u <- QQ^T u in place, then u <- mask * u if apply_mask (Sec. II-A).  Copies
 * of a node are summed in ascending local index, so the result is
 * bit-reproducible.  u: device [n_local], double (every SEM_FP64* precision:
 * FP64 sums) or float (SEM_FP32). */
SEM_API int sem_gs(sem_handle* h, void* u, int precision, int apply_mask, cudaStream_t stream);

/* w = B u (diagonal mass, B = rho rho rho J), then mask * QQ^T if assemble.
 * Used to form right-hand sides b = mask QQ^T (B f). */
SEM_API int sem_mass(sem_handle* h, void* w, const void* u, int precision, int assemble,
                     cudaStream_t stream);

/* result[0] = <a, b> over unique nodes = sum_L a_L b_L / mult_L, accumulated
 * in FP64 in a fixed order (deterministic).  a, b: device double [n_local];
 * result: device double[1] (batch handle: double[nsolve], one per solve). */
SEM_API int sem_dot(sem_handle* h, const double* a, const double* b, double* result,
                    cudaStream_t stream);

/* result[q] = <a, b> over the unique nodes of mesh q, like sem_dot, but the
 * call allocates nothing and uses no memory owned by the handle: its scratch
 * (one FP64 partial sum per CTA and a ticket counter) is a fixed device
 * array inside the library.  The paper has no counterpart; this exists for
 * callers that cannot call cudaMalloc at the point where they need the
 * product -- code recording a CUDA graph by stream capture (allocation is
 * refused during a capture), applications whose device memory is held by
 * their own pool allocator, latency-critical loops (cudaMalloc/cudaFree can
 * synchronise the device).
 *   h       handle from sem_setup / sem_setup_batch (read only)
 *   a, b    device double [n_local]
 *   result  device double[nsolve]
 * Each CTA sums a fixed chunk of 32768 points, so the result is the same on
 * every GPU; it equals sem_dot's up to rounding order.  Limit: at most
 * 134,217,728 local points per mesh (4096 partial sums; the array takes
 * 33 KB on every GPU that loads the library, until the process exits), else
 * SEM_EINVAL.  The first call on each device looks up the array's device
 * address; make that first call before any stream capture.  All calls share
 * the array: each clears its counter first, and calls that overlap on the GPU
 * (unordered streams) race and give wrong results. */
SEM_API int sem_dot_noalloc(const sem_handle* h, const double* a, const double* b, double* result,
                            cudaStream_t stream);

/* Gradient, divergence and curl of nodal fields by collocation (Sec. II-A:
 * the GLL nodal basis and D; the derivatives the pressure equation's right
 * side needs): du/dx_l = sum_s (dr_s/dx_l) (D_s u), element by element, so
 * the results are local fields that may jump across element faces.  All
 * vectors are device double [n_local]; outputs must not alias inputs.  The
 * handle must have been set up with SEM_FLAG_METRICS, else SEM_EINVAL. */
SEM_API int sem_grad(sem_handle* h, const double* u, double* gx, double* gy, double* gz, cudaStream_t stream);
SEM_API int sem_div(sem_handle* h, const double* vx, const double* vy, const double* vz, double* out,
                    cudaStream_t stream);
SEM_API int sem_curl(sem_handle* h, const double* vx, const double* vy, const double* vz, double* cx, double* cy,
                     double* cz, cudaStream_t stream);

/* Right-hand side of the pressure equation of the P_N-P_N splitting (Sec.
 * II-A, eq. "pressure"): -lap p = -div(vhat) / dt + (1/Re) div(curl(omega)),
 * in the weak form the Poisson solve takes, b = mask QQ^T (B f) with f the
 * collocation values of the right side (the same quadrature as sem_mass).
 *   vx, vy, vz  device [n_local] the explicit velocity vhat
 *   wx, wy, wz  device [n_local] the explicit vorticity omega, or all NULL
 *               (the term is dropped)
 *   dt, Re      time step and Reynolds number (> 0)
 *   b           device [n_local] output, assembled and masked
 * Uses the handle's FP64 work vectors; SEM_FLAG_METRICS required. */
SEM_API int sem_pressure_rhs(sem_handle* h, const double* vx, const double* vy, const double* vz,
                             const double* wx, const double* wy, const double* wz, double dt, double Re,
                             double* b, cudaStream_t stream);

/* Copies of set-up data (device outputs):
 *   G  [E][6][lx^3] factors h1*G11, h1*G12, h1*G13, h1*G22, h1*G23, h1*G33
 *   B  [n_local] mass rho rho rho J
 * Either pointer may be NULL.  Single-mesh handles only. */
SEM_API int sem_get_geometry(const sem_handle* h, double* G, double* B, cudaStream_t stream);

/* Jacobi preconditioner Minv = mask / (QQ^T diag(A_L)) (device double [n_local]). */
SEM_API int sem_get_jacobi(const sem_handle* h, double* minv, cudaStream_t stream);

/* Solve mask QQ^T A_L x = b with Jacobi-PCG (Sec. II-B) or mixed-precision
 * refinement.  x: [n_local] initial guess in, solution out; b: [n_local]
 * assembled right-hand side (equal on all copies of a node, 0 on Dirichlet
 * nodes).  Host or device pointers.  opts NULL = defaults; stats may be NULL.
 * Returns SEM_OK only when the true residual ||b - A x|| / ||b|| of the
 * returned x, recomputed with SEM_FP64, is at most tol; else SEM_ENOTCONV,
 * SEM_EBREAKDOWN (also for a non-finite initial residual: a NaN or Inf in x0
 * or b) or SEM_ESTAGNATE (x holds the last iterate), or an error.
 * Synchronises the stream. */
SEM_API int sem_cg_solve(sem_handle* h, double* x, const double* b, const sem_solve_opts* opts,
                         sem_solve_stats* stats, cudaStream_t stream);

/* z = M^-1 r with the two-level Schwarz preconditioner of SEM_MODE_GMRES
 * (handle set up with SEM_FLAG_SCHWARZ): point Jacobi, the fast-
 * diagonalisation solves of the element interiors, and the coarse-grid
 * correction (10 Jacobi-PCG iterations on the element corners), masked.
 * r, z: device double [n_local], r assembled; z must not alias r. */
SEM_API int sem_schwarz_apply(sem_handle* h, const double* r, double* z, cudaStream_t stream);

/* The same preconditioner on FP32 vectors with FP32 arithmetic in the local
 * solves, restriction and prolongation (the coarse CG stays FP64): the form
 * the mixed GMRES solve applies.  r, z: device float [n_local], r assembled;
 * z must not alias r.  Errors: SEM_EINVAL (null, aliasing, no Schwarz data). */
SEM_API int sem_schwarz_apply32(sem_handle* h, const float* r, float* z, cudaStream_t stream);

/* Projection space of a handle (sem_solve_opts.projection): drop every kept
 * vector (the next solve starts from x = 0), and the number kept now. */
SEM_API int sem_projection_reset(sem_handle* h);
SEM_API int sem_projection_size(const sem_handle* h, int* count);

/* All solves of a batch handle at once: x, b concatenated [n_local];
 * stats: host array of nsolve entries (may be NULL).  Every CG iteration
 * advances all unconverged solves with one set of launches: the operator (one
 * launch over the groups of every order, or one launch per order, whichever
 * the first solve's autotuning measured faster on this handle; a variant
 * pinned at set-up selects one launch per order), one gather-scatter and one
 * vector update.  Returns the worst status over the batch. */
SEM_API int sem_cg_solve_batch(sem_handle* h, double* x, const double* b,
                               const sem_solve_opts* opts, sem_solve_stats* stats,
                               cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SEM_H */
