/*
 * FP64 CPU oracle of the spectral-element Poisson solve (TEST INFRASTRUCTURE).
 *
 * This library exists only to check the CUDA path.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product library never links, calls or falls back to it, and the two share
 * no code.
 *
 * Every routine is a plain, slow, sequential restatement of the paper's
 * definitions (Karp et al., "Large-Scale Direct Numerical Simulations of
 * Turbulence Using GPUs and Modern Fortran", Sec. II-A and II-B):
 *   GLL nodes/weights and derivative matrix D .......... Sec. II-A, def. of D
 *   geometric factors G^e_st, mass B ................... Sec. II-A, def. of G
 *   local stiffness action A^e u = D^T G D u (with h1) . Sec. II-A, eq. (disclap)
 *   Helmholtz mass term h2 B u (velocity solve) ........ Sec. II-A, Helmholtz form
 *   gather-scatter QQ^T and Dirichlet mask ............. Sec. II-A, A = QQ^T A_L
 *   point-Jacobi diagonal, preconditioned CG ........... Sec. II-B (P-CG, Jacobi)
 *   FP64 iterative refinement around an FP32 inner CG .. Sec. V outlook on
 *                                                         lower precision
 * Layout: element-major local vectors [E][k][j][i], i fastest, n_L = E*lx^3.
 * Geometric factors are stored as six arrays G[s][n_L], s = 11,12,13,22,23,33.
 *
 * Parity pins: see the header of oracle/__init__.py.
 */
#ifndef SEM_ORACLE_H
#define SEM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_problem or_problem;

/* GLL nodes xi[0..N], weights rho[0..N] (Sec. II-A; textbook Legendre facts). */
void or_gll(int N, double* xi, double* rho);
/* D[i*lx + j] = l_j'(xi_i), the collocation derivative matrix (Sec. II-A). */
void or_dmat(int N, const double* xi, double* D);

/* Build the discrete problem.  coords [3][E][lx^3]; gid [n_L]; mask [n_L]
 * (0 = Dirichlet); h1 [n_L] or NULL for h1 = 1.  Returns NULL on error
 * (non-positive Jacobian, lx out of range, inconsistent mask). */
or_problem* or_setup(int E, int lx, const double* coords, const int64_t* gid,
                     const uint8_t* mask, const double* h1);
void or_free(or_problem* p);
int64_t or_n_local(const or_problem* p);
int64_t or_n_unique(const or_problem* p);

/* Copies of the set-up data: G [6][n_L], B [n_L] (rho rho rho J), mult [n_L]
 * (number of local copies of the node), Jacobi Minv [n_L]. */
void or_get_geom(const or_problem* p, double* G, double* B);
void or_get_mult(const or_problem* p, double* mult);
void or_get_minv(const or_problem* p, double* minv);
void or_get_dmat(const or_problem* p, double* D);

/* Helmholtz operator: A_L u = D^T (h1 G) D u + h2 B u from now on, Jacobi
 * diagonal with h2 B (h2 [n_L] copied; NULL returns to Poisson). */
void or_set_h2(or_problem* p, const double* h2);

/* w = A_L u (local, unassembled). */
void or_ax_local(const or_problem* p, const double* u, double* w);
/* |D^T| |h1 G| |D| |u| per element: the magnitude of the terms of A^e u. */
void or_ax_local_abs(const or_problem* p, const double* u, double* w);
/* u <- QQ^T u (sum over the copies of each node, in ascending local index);
 * then u <- mask * u if apply_mask. */
void or_gs(const or_problem* p, double* u, int apply_mask);
/* w = mask * QQ^T A_L u */
void or_ax(const or_problem* p, const double* u, double* w);
/* w = B u (local diagonal mass), then mask * QQ^T if assemble */
void or_mass(const or_problem* p, const double* u, double* w, int assemble);
/* <a,b> over unique nodes = sum_L a_L b_L / mult_L */
double or_dot(const or_problem* p, const double* a, const double* b);

/* Jacobi-PCG (Sec. II-B) on mask*QQ^T A_L x = b.  x holds the initial guess
 * on entry.  Stops when ||r||/||b|| <= tol (recursive residual) or after
 * max_iter iterations.  iters = iterations done; relres = TRUE residual
 * ||b - A x|| / ||b|| recomputed at the end.  When hist is not NULL it
 * receives the recursive relative residual after each iteration (max_iter
 * entries).  Returns 0 on convergence, 1 if max_iter was reached, 2 on
 * breakdown (p^T A p <= 0 or non-finite). */
int or_pcg(const or_problem* p, const double* b, double* x, double tol, int max_iter,
           int* iters, double* relres, double* hist);

/* Iterative refinement: outer FP64 residual r = b - A x, inner Jacobi-PCG in
 * FP32 arithmetic (FP32 vectors, FP32 operator, FP64 dot products) on
 * A d = r/||r|| to inner_tol, then x += ||r|| d.  Stops when the true FP64
 * residual ||b - A x||/||b|| <= tol, after max_outer outer steps, or when an
 * outer step whose inner solve reached inner_tol fails to halve the residual
 * (stagnation, return 3); a step stopped by max_inner is not judged.
 * outer_hist receives the true relative residual after each outer step.
 * carry = 0: every inner solve starts CG afresh (first direction z).
 * carry = 1: from the second outer step on, the inner CG keeps the search
 * direction of the previous step (rescaled to the new residual's units) and
 * continues as CG whose residual was replaced by the true one (residual
 * replacement, van der Vorst and Ye 2000).  The paper's Sec. V outlook names
 * lower precision without giving an algorithm: both variants are this
 * implementation's reading. */
int or_ir(const or_problem* p, const double* b, double* x, double tol, double inner_tol,
          int max_outer, int max_inner, int carry, int* outer_iters, int* inner_iters,
          double* relres, double* outer_hist);

/* Number of OpenMP threads the element loops use (1 without OpenMP). */
int or_threads(void);

#ifdef __cplusplus
}
#endif
#endif
