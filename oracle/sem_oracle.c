/*
 * FP64 CPU oracle of the spectral-element Poisson solve (TEST INFRASTRUCTURE,
 * see sem_oracle.h).  Plain loops, no blocking or fusion beyond what the
 * definitions state.  Element loops and vector updates may run under OpenMP;
 * every reduction (dot products, gather-scatter sums) is sequential in a
 * fixed order, so results do not depend on the thread count.
 */
#include "sem_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

struct or_problem {
    int E, lx;
    int64_t n;          /* n_L = E * lx^3 */
    int64_t n_unique;   /* number of distinct global ids */
    double* D;          /* [lx][lx] */
    double* rho;        /* [lx] */
    double* G;          /* [6][n] : G11 G12 G13 G22 G23 G33 */
    double* B;          /* [n] */
    double* h1;         /* [n] */
    double* h2;         /* [n] mass coefficient of the Helmholtz operator, NULL: Poisson */
    uint8_t* mask;      /* [n] */
    double* mult;       /* [n] */
    double* minv;       /* [n] */
    int64_t* order;     /* [n] local indices sorted by (gid, local index) */
    int64_t* grp;       /* [n_unique + 1] start of each id's run in order[] */
};

int or_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* GLL nodes, weights and derivative matrix (Sec. II-A).                     */
/* ------------------------------------------------------------------------ */

/* Legendre P_N(x) and P_{N-1}(x) by the three-term recurrence
 * (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1}. */
static void legendre(int N, long double x, long double* pN, long double* pNm1) {
    long double p0 = 1.0L, p1 = x;
    if (N == 0) { *pN = 1.0L; *pNm1 = 0.0L; return; }
    for (int n = 1; n < N; n++) {
        long double p2 = ((2.0L * n + 1.0L) * x * p1 - (long double)n * p0) / (n + 1.0L);
        p0 = p1;
        p1 = p2;
    }
    *pN = p1;
    *pNm1 = p0;
}

void or_gll(int N, double* xi, double* rho) {
    /* xi_0 = -1, xi_N = 1; interior nodes are the roots of P_N'.  Newton on
     * P_N' from the Chebyshev-Gauss-Lobatto guesses -cos(pi i / N), with
     * P_N'  = N (x P_N - P_{N-1}) / (x^2 - 1) and, from Legendre's equation,
     * P_N'' = (2 x P_N' - N(N+1) P_N) / (1 - x^2).
     * Weights rho_i = 2 / (N (N+1) P_N(xi_i)^2). */
    const long double pi = 3.141592653589793238462643383279502884L;
    xi[0] = -1.0;
    xi[N] = 1.0;
    for (int i = 1; i < N; i++) {
        long double x = -cosl(pi * i / N);
        for (int it = 0; it < 100; it++) {
            long double pN, pNm1;
            legendre(N, x, &pN, &pNm1);
            long double d1 = N * (x * pN - pNm1) / (x * x - 1.0L);
            long double d2 = (2.0L * x * d1 - (long double)N * (N + 1) * pN) / (1.0L - x * x);
            long double dx = d1 / d2;
            x -= dx;
            if (fabsl(dx) < 1e-19L) break;
        }
        xi[i] = (double)x;
    }
    for (int i = 0; i <= N; i++) {
        long double pN, pNm1;
        legendre(N, (long double)xi[i], &pN, &pNm1);
        rho[i] = (double)(2.0L / ((long double)N * (N + 1) * pN * pN));
    }
}

void or_dmat(int N, const double* xi, double* D) {
    /* D_ij = l_j'(xi_i): off the diagonal (P_N(xi_i)/P_N(xi_j)) / (xi_i - xi_j);
     * D_00 = -N(N+1)/4, D_NN = N(N+1)/4, other diagonal entries 0. */
    int lx = N + 1;
    long double* P = (long double*)malloc(sizeof(long double) * lx);
    for (int i = 0; i < lx; i++) {
        long double pm;
        legendre(N, (long double)xi[i], &P[i], &pm);
    }
    for (int i = 0; i < lx; i++)
        for (int j = 0; j < lx; j++) {
            long double v;
            if (i != j) v = (P[i] / P[j]) / ((long double)xi[i] - (long double)xi[j]);
            else if (i == 0) v = -(long double)N * (N + 1) / 4.0L;
            else if (i == N) v = (long double)N * (N + 1) / 4.0L;
            else v = 0.0L;
            D[i * lx + j] = (double)v;
        }
    free(P);
}

/* ------------------------------------------------------------------------ */
/* Gather-scatter bookkeeping: sort local indices by (gid, local index).     */
/* ------------------------------------------------------------------------ */

typedef struct { int64_t gid, idx; } gid_pair;

static int cmp_pair(const void* a, const void* b) {
    const gid_pair* x = (const gid_pair*)a;
    const gid_pair* y = (const gid_pair*)b;
    if (x->gid != y->gid) return x->gid < y->gid ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Geometric factors (Sec. II-A):                                            */
/* (G_st)_ijk = rho_i rho_j rho_k J_ijk sum_l (dr_s/dx_l)(dr_t/dx_l),         */
/* J = det(dx/dr), B_ijk = rho_i rho_j rho_k J_ijk.                           */
/* ------------------------------------------------------------------------ */

static int geometry(or_problem* p, const double* coords) {
    const int lx = p->lx;
    const int n3 = lx * lx * lx;
    const int64_t n = p->n;
    const double* X = coords;
    const double* Y = coords + n;
    const double* Z = coords + 2 * n;
    int bad = 0;
#pragma omp parallel for reduction(| : bad) schedule(static)
    for (int e = 0; e < p->E; e++) {
        const int64_t o = (int64_t)e * n3;
        for (int k = 0; k < lx; k++)
            for (int j = 0; j < lx; j++)
                for (int i = 0; i < lx; i++) {
                    /* derivatives of x, y, z along r (index i), s (j), t (k) */
                    double d[3][3] = {{0}};
                    const double* c[3] = {X + o, Y + o, Z + o};
                    for (int m = 0; m < 3; m++)
                        for (int l = 0; l < lx; l++) {
                            d[m][0] += p->D[i * lx + l] * c[m][k * lx * lx + j * lx + l];
                            d[m][1] += p->D[j * lx + l] * c[m][k * lx * lx + l * lx + i];
                            d[m][2] += p->D[k * lx + l] * c[m][l * lx * lx + j * lx + i];
                        }
                    const double a = d[0][0], b = d[0][1], cc = d[0][2];
                    const double dd = d[1][0], ee = d[1][1], ff = d[1][2];
                    const double g = d[2][0], h = d[2][1], kk = d[2][2];
                    const double J = a * (ee * kk - ff * h) - b * (dd * kk - ff * g) + cc * (dd * h - ee * g);
                    if (!(J > 0.0)) { bad = 1; continue; }
                    /* rows of the inverse Jacobian: grad r, grad s, grad t */
                    double inv[3][3];
                    inv[0][0] = (ee * kk - ff * h) / J;
                    inv[0][1] = (cc * h - b * kk) / J;
                    inv[0][2] = (b * ff - cc * ee) / J;
                    inv[1][0] = (ff * g - dd * kk) / J;
                    inv[1][1] = (a * kk - cc * g) / J;
                    inv[1][2] = (cc * dd - a * ff) / J;
                    inv[2][0] = (dd * h - ee * g) / J;
                    inv[2][1] = (b * g - a * h) / J;
                    inv[2][2] = (a * ee - b * dd) / J;
                    const double w = p->rho[i] * p->rho[j] * p->rho[k];
                    const int64_t L = o + k * lx * lx + j * lx + i;
                    const int ss[6] = {0, 0, 0, 1, 1, 2};
                    const int tt[6] = {0, 1, 2, 1, 2, 2};
                    for (int q = 0; q < 6; q++) {
                        double acc = 0.0;
                        for (int l = 0; l < 3; l++) acc += inv[ss[q]][l] * inv[tt[q]][l];
                        p->G[q * n + L] = w * J * acc;
                    }
                    p->B[L] = w * J;
                }
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Local operator A^e u = D^T G D u with h1 at the quadrature points          */
/* (Sec. II-A, eq. disclap; h1 scales G as in the Helmholtz operator).       */
/* ------------------------------------------------------------------------ */

void or_ax_local(const or_problem* p, const double* u, double* w) {
    const int lx = p->lx;
    const int n3 = lx * lx * lx;
    const int64_t n = p->n;
#pragma omp parallel
    {
        double* ur = (double*)malloc(sizeof(double) * n3);
        double* us = (double*)malloc(sizeof(double) * n3);
        double* ut = (double*)malloc(sizeof(double) * n3);
#pragma omp for schedule(static)
        for (int e = 0; e < p->E; e++) {
            const int64_t o = (int64_t)e * n3;
            const double* ue = u + o;
            /* ur = (I x I x D) u, us = (I x D x I) u, ut = (D x I x I) u */
            for (int k = 0; k < lx; k++)
                for (int j = 0; j < lx; j++)
                    for (int i = 0; i < lx; i++) {
                        double a = 0.0, b = 0.0, c = 0.0;
                        for (int l = 0; l < lx; l++) {
                            a += p->D[i * lx + l] * ue[k * lx * lx + j * lx + l];
                            b += p->D[j * lx + l] * ue[k * lx * lx + l * lx + i];
                            c += p->D[k * lx + l] * ue[l * lx * lx + j * lx + i];
                        }
                        const int q = k * lx * lx + j * lx + i;
                        ur[q] = a;
                        us[q] = b;
                        ut[q] = c;
                    }
            /* (wr, ws, wt) = h1 G (ur, us, ut) with G symmetric */
            for (int q = 0; q < n3; q++) {
                const int64_t L = o + q;
                const double g11 = p->G[0 * n + L], g12 = p->G[1 * n + L], g13 = p->G[2 * n + L];
                const double g22 = p->G[3 * n + L], g23 = p->G[4 * n + L], g33 = p->G[5 * n + L];
                const double a = ur[q], b = us[q], c = ut[q];
                const double h = p->h1[L];
                ur[q] = h * (g11 * a + g12 * b + g13 * c);
                us[q] = h * (g12 * a + g22 * b + g23 * c);
                ut[q] = h * (g13 * a + g23 * b + g33 * c);
            }
            /* w = (I x I x D^T) wr + (I x D^T x I) ws + (D^T x I x I) wt */
            for (int k = 0; k < lx; k++)
                for (int j = 0; j < lx; j++)
                    for (int i = 0; i < lx; i++) {
                        double acc = 0.0;
                        for (int l = 0; l < lx; l++) acc += p->D[l * lx + i] * ur[k * lx * lx + j * lx + l];
                        for (int l = 0; l < lx; l++) acc += p->D[l * lx + j] * us[k * lx * lx + l * lx + i];
                        for (int l = 0; l < lx; l++) acc += p->D[l * lx + k] * ut[l * lx * lx + j * lx + i];
                        /* Helmholtz: + h2 B u, the GLL-quadrature mass term (v, h2 u) */
                        const int64_t L = o + k * lx * lx + j * lx + i;
                        if (p->h2) acc += p->h2[L] * p->B[L] * ue[k * lx * lx + j * lx + i];
                        w[L] = acc;
                    }
        }
        free(ur);
        free(us);
        free(ut);
    }
}

/* ------------------------------------------------------------------------ */
/* Magnitude of the terms of A^e u: the same three stages with |D|, |G|, |u| */
/* (|D^T| |h1 G| |D| |u|).  An evaluation of A^e u in arithmetic of unit     */
/* roundoff eps errs by at most about (number of sequential operations) x    */
/* eps times this, pointwise (the running error bound of a sum of products). */
/* Test infrastructure: it scales the parity tolerance of cancelling inputs. */
/* ------------------------------------------------------------------------ */

void or_ax_local_abs(const or_problem* p, const double* u, double* w) {
    const int lx = p->lx;
    const int n3 = lx * lx * lx;
    const int64_t n = p->n;
#pragma omp parallel
    {
        double* ur = (double*)malloc(sizeof(double) * n3);
        double* us = (double*)malloc(sizeof(double) * n3);
        double* ut = (double*)malloc(sizeof(double) * n3);
#pragma omp for schedule(static)
        for (int e = 0; e < p->E; e++) {
            const int64_t o = (int64_t)e * n3;
            const double* ue = u + o;
            for (int k = 0; k < lx; k++)
                for (int j = 0; j < lx; j++)
                    for (int i = 0; i < lx; i++) {
                        double a = 0.0, b = 0.0, c = 0.0;
                        for (int l = 0; l < lx; l++) {
                            a += fabs(p->D[i * lx + l]) * fabs(ue[k * lx * lx + j * lx + l]);
                            b += fabs(p->D[j * lx + l]) * fabs(ue[k * lx * lx + l * lx + i]);
                            c += fabs(p->D[k * lx + l]) * fabs(ue[l * lx * lx + j * lx + i]);
                        }
                        const int q = k * lx * lx + j * lx + i;
                        ur[q] = a;
                        us[q] = b;
                        ut[q] = c;
                    }
            for (int q = 0; q < n3; q++) {
                const int64_t L = o + q;
                const double g11 = fabs(p->G[0 * n + L]), g12 = fabs(p->G[1 * n + L]), g13 = fabs(p->G[2 * n + L]);
                const double g22 = fabs(p->G[3 * n + L]), g23 = fabs(p->G[4 * n + L]), g33 = fabs(p->G[5 * n + L]);
                const double a = ur[q], b = us[q], c = ut[q];
                const double h = fabs(p->h1[L]);
                ur[q] = h * (g11 * a + g12 * b + g13 * c);
                us[q] = h * (g12 * a + g22 * b + g23 * c);
                ut[q] = h * (g13 * a + g23 * b + g33 * c);
            }
            for (int k = 0; k < lx; k++)
                for (int j = 0; j < lx; j++)
                    for (int i = 0; i < lx; i++) {
                        double acc = 0.0;
                        for (int l = 0; l < lx; l++) acc += fabs(p->D[l * lx + i]) * ur[k * lx * lx + j * lx + l];
                        for (int l = 0; l < lx; l++) acc += fabs(p->D[l * lx + j]) * us[k * lx * lx + l * lx + i];
                        for (int l = 0; l < lx; l++) acc += fabs(p->D[l * lx + k]) * ut[l * lx * lx + j * lx + i];
                        const int64_t L = o + k * lx * lx + j * lx + i;
                        if (p->h2) acc += fabs(p->h2[L] * p->B[L] * u[L]);
                        w[L] = acc;
                    }
        }
        free(ur);
        free(us);
        free(ut);
    }
}

/* ------------------------------------------------------------------------ */
/* QQ^T: every copy of a node receives the sum over all its copies, summed   */
/* in ascending local index (Sec. II-A, A = QQ^T A_L).                        */
/* ------------------------------------------------------------------------ */

void or_gs(const or_problem* p, double* u, int apply_mask) {
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < p->n_unique; g++) {
        double s = 0.0;
        for (int64_t c = p->grp[g]; c < p->grp[g + 1]; c++) s += u[p->order[c]];
        for (int64_t c = p->grp[g]; c < p->grp[g + 1]; c++) u[p->order[c]] = s;
    }
    if (apply_mask) {
#pragma omp parallel for schedule(static)
        for (int64_t L = 0; L < p->n; L++)
            if (!p->mask[L]) u[L] = 0.0;
    }
}

void or_ax(const or_problem* p, const double* u, double* w) {
    or_ax_local(p, u, w);
    or_gs(p, w, 1);
}

void or_mass(const or_problem* p, const double* u, double* w, int assemble) {
#pragma omp parallel for schedule(static)
    for (int64_t L = 0; L < p->n; L++) w[L] = p->B[L] * u[L];
    if (assemble) or_gs(p, w, 1);
}

double or_dot(const or_problem* p, const double* a, const double* b) {
    double s = 0.0;
    for (int64_t L = 0; L < p->n; L++) s += a[L] * b[L] / p->mult[L];
    return s;
}

/* ------------------------------------------------------------------------ */
/* Point-Jacobi: exact diagonal of A^e (Sec. II-B, P-CG with a Jacobi-type   */
/* preconditioner).  For point (i,j,k), with h1 at the quadrature points:    */
/*  d = sum_l D_li^2 h1 G11(l,j,k) + sum_l D_lj^2 h1 G22(i,l,k)              */
/*    + sum_l D_lk^2 h1 G33(i,j,l)                                           */
/*    + 2 h1(i,j,k) (D_ii D_jj G12 + D_ii D_kk G13 + D_jj D_kk G23)(i,j,k)    */
/* then d <- QQ^T d and Minv = mask / d.                                     */
/* ------------------------------------------------------------------------ */

static void jacobi(or_problem* p) {
    const int lx = p->lx;
    const int n3 = lx * lx * lx;
    const int64_t n = p->n;
    double* d = p->minv;
    const double* D = p->D;
#pragma omp parallel for schedule(static)
    for (int e = 0; e < p->E; e++) {
        const int64_t o = (int64_t)e * n3;
        for (int k = 0; k < lx; k++)
            for (int j = 0; j < lx; j++)
                for (int i = 0; i < lx; i++) {
                    double s = 0.0;
                    for (int l = 0; l < lx; l++) {
                        const int64_t La = o + k * lx * lx + j * lx + l;
                        const int64_t Lb = o + k * lx * lx + l * lx + i;
                        const int64_t Lc = o + l * lx * lx + j * lx + i;
                        s += D[l * lx + i] * D[l * lx + i] * p->h1[La] * p->G[0 * n + La];
                        s += D[l * lx + j] * D[l * lx + j] * p->h1[Lb] * p->G[3 * n + Lb];
                        s += D[l * lx + k] * D[l * lx + k] * p->h1[Lc] * p->G[5 * n + Lc];
                    }
                    const int64_t L = o + k * lx * lx + j * lx + i;
                    const double dii = D[i * lx + i], djj = D[j * lx + j], dkk = D[k * lx + k];
                    s += 2.0 * p->h1[L] *
                         (dii * djj * p->G[1 * n + L] + dii * dkk * p->G[2 * n + L] + djj * dkk * p->G[4 * n + L]);
                    if (p->h2) s += p->h2[L] * p->B[L];  /* Helmholtz mass term on the diagonal */
                    d[L] = s;
                }
    }
    or_gs(p, d, 0);
    for (int64_t L = 0; L < n; L++) d[L] = p->mask[L] ? 1.0 / d[L] : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Set-up.                                                                   */
/* ------------------------------------------------------------------------ */

or_problem* or_setup(int E, int lx, const double* coords, const int64_t* gid,
                     const uint8_t* mask, const double* h1) {
    if (E < 1 || lx < 2 || lx > 16) return NULL;
    or_problem* p = (or_problem*)calloc(1, sizeof(or_problem));
    const int n3 = lx * lx * lx;
    p->E = E;
    p->lx = lx;
    p->n = (int64_t)E * n3;
    const int64_t n = p->n;
    double* xi = (double*)malloc(sizeof(double) * lx);
    p->rho = (double*)malloc(sizeof(double) * lx);
    p->D = (double*)malloc(sizeof(double) * lx * lx);
    or_gll(lx - 1, xi, p->rho);
    or_dmat(lx - 1, xi, p->D);
    free(xi);
    p->G = (double*)malloc(sizeof(double) * 6 * n);
    p->B = (double*)malloc(sizeof(double) * n);
    p->h1 = (double*)malloc(sizeof(double) * n);
    p->mask = (uint8_t*)malloc(n);
    p->mult = (double*)malloc(sizeof(double) * n);
    p->minv = (double*)malloc(sizeof(double) * n);
    p->order = (int64_t*)malloc(sizeof(int64_t) * n);
    for (int64_t L = 0; L < n; L++) {
        p->h1[L] = h1 ? h1[L] : 1.0;
        p->mask[L] = mask[L] ? 1 : 0;
    }
    /* copies of each global id, ordered by local index */
    gid_pair* pr = (gid_pair*)malloc(sizeof(gid_pair) * n);
    for (int64_t L = 0; L < n; L++) { pr[L].gid = gid[L]; pr[L].idx = L; }
    qsort(pr, (size_t)n, sizeof(gid_pair), cmp_pair);
    int64_t nu = 0;
    for (int64_t c = 0; c < n; c++)
        if (c == 0 || pr[c].gid != pr[c - 1].gid) nu++;
    p->n_unique = nu;
    p->grp = (int64_t*)malloc(sizeof(int64_t) * (nu + 1));
    int64_t g = -1;
    for (int64_t c = 0; c < n; c++) {
        if (c == 0 || pr[c].gid != pr[c - 1].gid) p->grp[++g] = c;
        p->order[c] = pr[c].idx;
    }
    p->grp[nu] = n;
    free(pr);
    int inconsistent = 0;
    for (int64_t q = 0; q < nu; q++) {
        const int64_t cnt = p->grp[q + 1] - p->grp[q];
        for (int64_t c = p->grp[q]; c < p->grp[q + 1]; c++) {
            p->mult[p->order[c]] = (double)cnt;
            if (p->mask[p->order[c]] != p->mask[p->order[p->grp[q]]]) inconsistent = 1;
        }
    }
    if (inconsistent || geometry(p, coords) != 0) {
        or_free(p);
        return NULL;
    }
    jacobi(p);
    return p;
}

void or_free(or_problem* p) {
    if (!p) return;
    free(p->D); free(p->rho); free(p->G); free(p->B); free(p->h1); free(p->h2); free(p->mask);
    free(p->mult); free(p->minv); free(p->order); free(p->grp);
    free(p);
}

/* Helmholtz operator (Sec. II-A: the velocity equation's implicit viscous term
 * gives a Helmholtz problem; h1 weighs the stiffness, h2 the mass): from now on
 * A_L u = D^T (h1 G) D u + h2 B u, and the Jacobi diagonal includes h2 B.
 * h2 = NULL returns to the Poisson operator. */
void or_set_h2(or_problem* p, const double* h2) {
    free(p->h2);
    p->h2 = NULL;
    if (h2) {
        p->h2 = (double*)malloc(sizeof(double) * p->n);
        memcpy(p->h2, h2, sizeof(double) * p->n);
    }
    jacobi(p);
}

int64_t or_n_local(const or_problem* p) { return p->n; }
int64_t or_n_unique(const or_problem* p) { return p->n_unique; }
void or_get_geom(const or_problem* p, double* G, double* B) {
    if (G) memcpy(G, p->G, sizeof(double) * 6 * p->n);
    if (B) memcpy(B, p->B, sizeof(double) * p->n);
}
void or_get_mult(const or_problem* p, double* mult) { memcpy(mult, p->mult, sizeof(double) * p->n); }
void or_get_minv(const or_problem* p, double* minv) { memcpy(minv, p->minv, sizeof(double) * p->n); }
void or_get_dmat(const or_problem* p, double* D) { memcpy(D, p->D, sizeof(double) * p->lx * p->lx); }

/* ------------------------------------------------------------------------ */
/* Jacobi-preconditioned CG (Sec. II-B).                                     */
/* ------------------------------------------------------------------------ */

int or_pcg(const or_problem* p, const double* b, double* x, double tol, int max_iter,
           int* iters, double* relres, double* hist) {
    const int64_t n = p->n;
    double* r = (double*)malloc(sizeof(double) * n);
    double* z = (double*)malloc(sizeof(double) * n);
    double* pp = (double*)calloc((size_t)n, sizeof(double));
    double* w = (double*)malloc(sizeof(double) * n);
    int status = 1, it = 0;
    or_ax(p, x, w);
    for (int64_t L = 0; L < n; L++) r[L] = b[L] - w[L];
    const double bnorm = sqrt(or_dot(p, b, b));
    double rho_old = 1.0;
    if (bnorm == 0.0) {
        for (int64_t L = 0; L < n; L++) x[L] = 0.0;
        status = 0;
    }
    while (status == 1 && it < max_iter) {
        for (int64_t L = 0; L < n; L++) z[L] = p->minv[L] * r[L];
        const double rho = or_dot(p, r, z);
        const double beta = (it == 0) ? 0.0 : rho / rho_old;
        for (int64_t L = 0; L < n; L++) pp[L] = z[L] + beta * pp[L];
        or_ax(p, pp, w);
        const double pap = or_dot(p, pp, w);
        if (!(pap > 0.0) || !isfinite(pap)) { status = 2; break; }
        const double alpha = rho / pap;
        for (int64_t L = 0; L < n; L++) {
            x[L] += alpha * pp[L];
            r[L] -= alpha * w[L];
        }
        rho_old = rho;
        it++;
        const double rel = sqrt(or_dot(p, r, r)) / bnorm;
        if (hist) hist[it - 1] = rel;
        if (rel <= tol) status = 0;
    }
    *iters = it;
    /* true residual */
    or_ax(p, x, w);
    for (int64_t L = 0; L < n; L++) r[L] = b[L] - w[L];
    *relres = bnorm > 0.0 ? sqrt(or_dot(p, r, r)) / bnorm : 0.0;
    free(r); free(z); free(pp); free(w);
    return status;
}

/* ------------------------------------------------------------------------ */
/* FP32 operator pieces for the inner solve of iterative refinement.         */
/* Same definitions as above, evaluated with float data and float arithmetic.*/
/* ------------------------------------------------------------------------ */

typedef struct {
    float* D;
    float* G;   /* [6][n] */
    float* h1;
    float* minv;
    float* hb;  /* [n] float(h2 B) of a Helmholtz operator, NULL: Poisson */
} or_f32;

static void ax_local_f32(const or_problem* p, const or_f32* f, const float* u, float* w) {
    const int lx = p->lx;
    const int n3 = lx * lx * lx;
    const int64_t n = p->n;
#pragma omp parallel
    {
        float* ur = (float*)malloc(sizeof(float) * n3);
        float* us = (float*)malloc(sizeof(float) * n3);
        float* ut = (float*)malloc(sizeof(float) * n3);
#pragma omp for schedule(static)
        for (int e = 0; e < p->E; e++) {
            const int64_t o = (int64_t)e * n3;
            const float* ue = u + o;
            for (int k = 0; k < lx; k++)
                for (int j = 0; j < lx; j++)
                    for (int i = 0; i < lx; i++) {
                        float a = 0.0f, b = 0.0f, c = 0.0f;
                        for (int l = 0; l < lx; l++) {
                            a += f->D[i * lx + l] * ue[k * lx * lx + j * lx + l];
                            b += f->D[j * lx + l] * ue[k * lx * lx + l * lx + i];
                            c += f->D[k * lx + l] * ue[l * lx * lx + j * lx + i];
                        }
                        const int q = k * lx * lx + j * lx + i;
                        ur[q] = a;
                        us[q] = b;
                        ut[q] = c;
                    }
            for (int q = 0; q < n3; q++) {
                const int64_t L = o + q;
                const float g11 = f->G[0 * n + L], g12 = f->G[1 * n + L], g13 = f->G[2 * n + L];
                const float g22 = f->G[3 * n + L], g23 = f->G[4 * n + L], g33 = f->G[5 * n + L];
                const float a = ur[q], b = us[q], c = ut[q];
                const float h = f->h1[L];
                ur[q] = h * (g11 * a + g12 * b + g13 * c);
                us[q] = h * (g12 * a + g22 * b + g23 * c);
                ut[q] = h * (g13 * a + g23 * b + g33 * c);
            }
            for (int k = 0; k < lx; k++)
                for (int j = 0; j < lx; j++)
                    for (int i = 0; i < lx; i++) {
                        float acc = 0.0f;
                        for (int l = 0; l < lx; l++) acc += f->D[l * lx + i] * ur[k * lx * lx + j * lx + l];
                        for (int l = 0; l < lx; l++) acc += f->D[l * lx + j] * us[k * lx * lx + l * lx + i];
                        for (int l = 0; l < lx; l++) acc += f->D[l * lx + k] * ut[l * lx * lx + j * lx + i];
                        const int64_t L = o + k * lx * lx + j * lx + i;
                        if (f->hb) acc += f->hb[L] * u[L];
                        w[L] = acc;
                    }
        }
        free(ur);
        free(us);
        free(ut);
    }
}

static void gs_f32(const or_problem* p, float* u) {
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < p->n_unique; g++) {
        float s = 0.0f;
        for (int64_t c = p->grp[g]; c < p->grp[g + 1]; c++) s += u[p->order[c]];
        for (int64_t c = p->grp[g]; c < p->grp[g + 1]; c++) u[p->order[c]] = s;
    }
#pragma omp parallel for schedule(static)
    for (int64_t L = 0; L < p->n; L++)
        if (!p->mask[L]) u[L] = 0.0f;
}

static double dot_f32(const or_problem* p, const float* a, const float* b) {
    double s = 0.0;
    for (int64_t L = 0; L < p->n; L++) s += (double)a[L] * (double)b[L] / p->mult[L];
    return s;
}

/* inner Jacobi-PCG in FP32 from d = 0; returns iterations */
/* FP32 PCG from d = 0.  pp is the search direction (n floats, owned by the
 * caller).  *carry <= 0: a fresh start (first direction = z).  *carry > 0:
 * pp holds the direction of an earlier solve and *carry the <r, z> that went
 * into it, rescaled to this right-hand side's units; the first direction is
 * then z + (<r, z> / *carry) pp, i.e. CG continues after its residual was
 * replaced by b (residual replacement).  On return *carry = the <r, z> of the
 * last direction taken (0 if none). */
static int pcg_f32(const or_problem* p, const or_f32* f, const float* b, float* d,
                   double tol, int max_iter, float* pp, double* carry) {
    const int64_t n = p->n;
    float* r = (float*)malloc(sizeof(float) * n);
    float* z = (float*)malloc(sizeof(float) * n);
    float* w = (float*)malloc(sizeof(float) * n);
    for (int64_t L = 0; L < n; L++) { r[L] = b[L]; d[L] = 0.0f; }
    const double bnorm = sqrt(dot_f32(p, b, b));
    const int carried = *carry > 0.0;
    double rho_old = carried ? *carry : 1.0;
    *carry = 0.0;
    int it = 0;
    while (bnorm > 0.0 && it < max_iter) {
        for (int64_t L = 0; L < n; L++) z[L] = f->minv[L] * r[L];
        const double rho = dot_f32(p, r, z);
        const float beta = (it == 0 && !carried) ? 0.0f : (float)(rho / rho_old);
        for (int64_t L = 0; L < n; L++) pp[L] = z[L] + beta * pp[L];
        ax_local_f32(p, f, pp, w);
        gs_f32(p, w);
        const double pap = dot_f32(p, pp, w);
        if (!(pap > 0.0) || !isfinite(pap)) break;
        const float alpha = (float)(rho / pap);
        for (int64_t L = 0; L < n; L++) {
            d[L] += alpha * pp[L];
            r[L] -= alpha * w[L];
        }
        rho_old = rho;
        *carry = rho;
        it++;
        if (sqrt(dot_f32(p, r, r)) / bnorm <= tol) break;
    }
    free(r); free(z); free(w);
    return it;
}

int or_ir(const or_problem* p, const double* b, double* x, double tol, double inner_tol,
          int max_outer, int max_inner, int carry, int* outer_iters, int* inner_iters,
          double* relres, double* outer_hist) {
    const int64_t n = p->n;
    const int lx = p->lx;
    or_f32 f;
    f.D = (float*)malloc(sizeof(float) * lx * lx);
    f.G = (float*)malloc(sizeof(float) * 6 * n);
    f.h1 = (float*)malloc(sizeof(float) * n);
    f.minv = (float*)malloc(sizeof(float) * n);
    for (int q = 0; q < lx * lx; q++) f.D[q] = (float)p->D[q];
    for (int64_t q = 0; q < 6 * n; q++) f.G[q] = (float)p->G[q];
    for (int64_t L = 0; L < n; L++) { f.h1[L] = (float)p->h1[L]; f.minv[L] = (float)p->minv[L]; }
    f.hb = NULL;
    if (p->h2) {
        f.hb = (float*)malloc(sizeof(float) * n);
        for (int64_t L = 0; L < n; L++) f.hb[L] = (float)(p->h2[L] * p->B[L]);
    }
    double* r = (double*)malloc(sizeof(double) * n);
    double* w = (double*)malloc(sizeof(double) * n);
    float* r32 = (float*)malloc(sizeof(float) * n);
    float* d32 = (float*)malloc(sizeof(float) * n);
    float* pp = (float*)calloc((size_t)n, sizeof(float));
    const double bnorm = sqrt(or_dot(p, b, b));
    int status = 1, outer = 0, inner = 0;
    double prev = INFINITY, rel = 0.0, rn_prev = 0.0, rho_carry = 0.0;
    int capped_last = 0;
    for (;;) {
        or_ax(p, x, w);
        for (int64_t L = 0; L < n; L++) r[L] = b[L] - w[L];
        const double rn = sqrt(or_dot(p, r, r));
        rel = bnorm > 0.0 ? rn / bnorm : 0.0;
        if (outer > 0 && outer_hist) outer_hist[outer - 1] = rel;
        if (rel <= tol) { status = 0; break; }
        if (outer >= max_outer) { status = 1; break; }
        /* stagnation is judged only after an inner solve that reached its
         * tolerance: one stopped by max_inner may leave a larger residual (CG
         * does not shrink the residual norm monotonically) */
        if (outer > 0 && rel > 0.5 * prev && !capped_last) { status = 3; break; }
        prev = rel;
        for (int64_t L = 0; L < n; L++) r32[L] = (float)(r[L] / rn);
        /* carried direction: the previous step's units were 1/rn_prev, these
         * are 1/rn, so pp scales by c = rn_prev / rn and its <r, z> by c^2;
         * folding one c into the <r, z> leaves pp as it is */
        rho_carry = (carry && outer > 0 && rho_carry > 0.0) ? rho_carry * (rn_prev / rn) : 0.0;
        const int it_step = pcg_f32(p, &f, r32, d32, inner_tol, max_inner, pp, &rho_carry);
        inner += it_step;
        capped_last = it_step >= max_inner;
        for (int64_t L = 0; L < n; L++) x[L] += rn * (double)d32[L];
        rn_prev = rn;
        outer++;
    }
    *outer_iters = outer;
    *inner_iters = inner;
    *relres = rel;
    free(f.D); free(f.G); free(f.h1); free(f.minv); free(f.hb);
    free(r); free(w); free(r32); free(d32); free(pp);
    return status;
}
