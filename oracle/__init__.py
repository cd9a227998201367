"""FP64 CPU oracle of the spectral-element Poisson solve -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library
(``paper_2207_07098_gb300``) never imports, links or falls back to it, and the
two share no code; only the seeded input generators in ``workloads`` serve
both.

The arithmetic lives in ``sem_oracle.c`` (plain sequential loops, FP64),
built into ``liboracle.so`` by :func:`build` and reached through ctypes.
Each routine restates a definition of Karp et al. (Sec. II-A: GLL basis,
derivative matrix D, geometric factors G, local operator A^e = D^T G D,
QQ^T; Sec. II-B: Jacobi-preconditioned CG).

What pins the oracle to something other than itself (tests/test_oracle_*.py):

* GLL: sum of weights = 2; closed-form nodes and weights for N = 1..4
  (tests/golden/gll_closed_forms.txt); exact quadrature of x^k, k <= 2N-1;
  symmetric nodes.
* D: exact derivative of every polynomial of degree <= N; zero row sums;
  centro-symmetry; 1-D stiffness D^T W D equal to closed forms (N = 1, 2) and
  to exact integrals of Lagrange-basis derivatives built with numpy
  polynomials.
* Geometry: closed form for affine elements; total volume (unit cube, also
  deformed; annulus = 255 pi).
* A: kernel contains constants (Neumann); closed Kronecker form on affine
  meshes; symmetry; positive definiteness on the masked space; entrywise
  equality with a dense matrix assembled from explicit Kronecker products,
  numpy Jacobians and an explicit Q on 1-8 deformed elements.
* QQ^T: multiplicities 1/2/4/8 from mesh structure; sum invariance.
* Jacobi: diagonal of the dense assembled matrix.
* Gradient, divergence, curl: exact for polynomials of degree <= N on
  (sheared) affine meshes; curl grad = 0 and div curl = 0 there; spectral
  convergence on deformed meshes; pressure right-hand side of a gradient
  field equal to the mass-weighted Laplacian.
* FGMRES with the two-level Schwarz preconditioner: the fast-diagonalisation
  local solve equals the dense interior solve on box elements; prolongation
  reproduces trilinear fields; FGMRES with the identity reaches the dense
  solution; the preconditioner cuts iterations against Jacobi-PCG.
* Pipelined PCG: the iterates and recursive residuals of Jacobi-PCG within
  rounding on small problems; dense solution.
* Projection onto previous solutions: A-orthonormal basis; exact recovery of
  a solution in the span; equality with a dense Galerkin projection; fewer
  iterations on a slowly varying sequence of right-hand sides; reset when full.
* Helmholtz (h2 B mass term): constants give exactly the assembled h2 B;
  dense K + Q^T diag(h2 B) Q; its diagonal; SPD without Dirichlet nodes (PCG
  = dense solve); spectral convergence of -lap u + lambda u = f.
* PCG: dense direct solve on tiny meshes; spectral convergence to
  sin(pi x) sin(pi y) sin(pi z); at most n_free iterations on tiny meshes.
* IR: reaches the FP64 solution; monotone outer residuals.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "sem_oracle.c")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, -O2, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "sem_oracle.h"))):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", _SO + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    _lib = configure(ctypes.CDLL(_SO))
    return _lib


def configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    lib.or_gll.argtypes = [ctypes.c_int, _dp, _dp]
    lib.or_dmat.argtypes = [ctypes.c_int, _dp, _dp]
    lib.or_setup.restype = ctypes.c_void_p
    lib.or_setup.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _i64p, _u8p, _dp]
    lib.or_free.argtypes = [ctypes.c_void_p]
    lib.or_n_local.restype = ctypes.c_int64
    lib.or_n_local.argtypes = [ctypes.c_void_p]
    lib.or_n_unique.restype = ctypes.c_int64
    lib.or_n_unique.argtypes = [ctypes.c_void_p]
    for name in ("or_get_mult", "or_get_minv", "or_get_dmat"):
        getattr(lib, name).argtypes = [ctypes.c_void_p, _dp]
    lib.or_get_geom.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.or_set_h2.argtypes = [ctypes.c_void_p, _dp]
    lib.or_ax_local.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.or_ax_local_abs.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.or_ax.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.or_gs.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int]
    lib.or_mass.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_int]
    lib.or_dot.restype = ctypes.c_double
    lib.or_dot.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.or_pcg.restype = ctypes.c_int
    lib.or_pcg.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_double, ctypes.c_int, _ip, _dp, _dp]
    lib.or_ir.restype = ctypes.c_int
    lib.or_ir.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_double, ctypes.c_double,
                          ctypes.c_int, ctypes.c_int, ctypes.c_int, _ip, _ip, _dp, _dp]
    lib.or_threads.restype = ctypes.c_int
    return lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def threads() -> int:
    """OpenMP threads the oracle's element loops use."""
    return _load().or_threads()


def gll(N: int):
    """GLL nodes and weights of order N (Newton on P_N', long double)."""
    lib = _load()
    xi = np.zeros(N + 1)
    rho = np.zeros(N + 1)
    lib.or_gll(N, _d(xi), _d(rho))
    return xi, rho


def dmat(N: int, xi: np.ndarray | None = None) -> np.ndarray:
    """Derivative matrix D[i, j] = l_j'(xi_i)."""
    lib = _load()
    if xi is None:
        xi, _ = gll(N)
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    D = np.zeros((N + 1, N + 1))
    lib.or_dmat(N, _d(xi), _d(D))
    return D


class Problem:
    """The discrete Poisson problem of one mesh, held by the C oracle."""

    def __init__(self, mesh, h1: np.ndarray | None = None):
        lib = _load()
        self.lib = lib
        self.mesh = mesh
        self.E, self.lx = mesh.E, mesh.lx
        coords = np.ascontiguousarray(mesh.coords, dtype=np.float64)
        gid = np.ascontiguousarray(mesh.gid, dtype=np.int64)
        mask = np.ascontiguousarray(mesh.mask, dtype=np.uint8)
        self._h1 = None if h1 is None else np.ascontiguousarray(h1, dtype=np.float64)
        self.h = lib.or_setup(mesh.E, mesh.lx, _d(coords), gid.ctypes.data_as(_i64p),
                              mask.ctypes.data_as(_u8p),
                              None if self._h1 is None else _d(self._h1))
        if not self.h:
            raise ValueError("oracle set-up rejected the mesh (J <= 0, lx out of range or "
                             "mask differing between copies of a node)")
        self.n = int(lib.or_n_local(self.h))
        self.n_unique = int(lib.or_n_unique(self.h))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.or_free(h)
            self.h = None

    # set-up data --------------------------------------------------------
    def geom(self):
        G = np.zeros((6, self.n))
        B = np.zeros(self.n)
        self.lib.or_get_geom(self.h, _d(G), _d(B))
        return G, B

    def mult(self):
        m = np.zeros(self.n)
        self.lib.or_get_mult(self.h, _d(m))
        return m

    def minv(self):
        m = np.zeros(self.n)
        self.lib.or_get_minv(self.h, _d(m))
        return m

    def dmat(self):
        D = np.zeros((self.lx, self.lx))
        self.lib.or_get_dmat(self.h, _d(D))
        return D

    def set_h2(self, h2):
        """Helmholtz operator A_L u = D^T (h1 G) D u + h2 B u (the velocity
        solve's implicit viscous term, Sec. II-A); None returns to Poisson.
        The Jacobi diagonal is rebuilt with the h2 B term."""
        if h2 is None:
            self.lib.or_set_h2(self.h, None)
        else:
            self.lib.or_set_h2(self.h, _d(np.ascontiguousarray(h2, dtype=np.float64)))

    # operators ----------------------------------------------------------
    def ax_local(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        w = np.zeros(self.n)
        self.lib.or_ax_local(self.h, _d(u), _d(w))
        return w

    def ax_local_abs(self, u):
        """|D^T| |h1 G| |D| |u| per element (magnitude of the terms of A_L u),
        the scale of the rounding error of any evaluation of A_L u."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        w = np.zeros(self.n)
        self.lib.or_ax_local_abs(self.h, _d(u), _d(w))
        return w

    def ax(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        w = np.zeros(self.n)
        self.lib.or_ax(self.h, _d(u), _d(w))
        return w

    def gs(self, u, mask: bool = True):
        w = np.array(u, dtype=np.float64, copy=True)
        self.lib.or_gs(self.h, _d(w), 1 if mask else 0)
        return w

    def mass(self, u, assemble: bool = True):
        u = np.ascontiguousarray(u, dtype=np.float64)
        w = np.zeros(self.n)
        self.lib.or_mass(self.h, _d(u), _d(w), 1 if assemble else 0)
        return w

    def dot(self, a, b) -> float:
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        return float(self.lib.or_dot(self.h, _d(a), _d(b)))

    # solvers ------------------------------------------------------------
    def pcg(self, b, x0=None, tol: float = 1e-10, max_iter: int = 100000, hist: bool = False):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        h = np.zeros(max_iter) if hist else None
        st = self.lib.or_pcg(self.h, _d(b), _d(x), tol, max_iter, ctypes.byref(it),
                             ctypes.byref(rr), None if h is None else _d(h))
        info = dict(status=int(st), iters=int(it.value), relres=float(rr.value))
        if hist:
            info["hist"] = h[: it.value]
        return x, info

    def ir(self, b, x0=None, tol: float = 1e-10, inner_tol: float = 1e-5, max_outer: int = 50,
           max_inner: int = 100000, carry: bool = False):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        oi = ctypes.c_int(0)
        ii = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        hist = np.zeros(max_outer + 1)
        st = self.lib.or_ir(self.h, _d(b), _d(x), tol, inner_tol, max_outer, max_inner, 1 if carry else 0,
                            ctypes.byref(oi), ctypes.byref(ii), ctypes.byref(rr), _d(hist))
        return x, dict(status=int(st), outer=int(oi.value), inner=int(ii.value),
                       relres=float(rr.value), outer_hist=hist[: oi.value])


class Projection:
    """Projection onto previous solutions (Sec. II-B, after Fischer 1998, as
    the paper's solvers use it for pressure and velocity; on the GPUs the space
    is reset when it holds `max_vectors` vectors, every 20 solves in the
    paper's runs).

    The space keeps vectors xt_i that are A-orthonormal in the unique-node
    inner product <a, b> = sum_L a_L b_L / mult_L, and bt_i = A xt_i.  For a
    right-hand side b the projected start is xbar = sum_i <xt_i, b> xt_i,
    the A-orthogonal projection of the solution A^-1 b onto the span (its
    error is A-orthogonal to every xt_i).  After the solve, the new direction
    dx = x - xbar is A-orthogonalised against the space by classical
    Gram-Schmidt run twice (coefficients <bt_i, v> = xt_i^T A v), normalised
    in the A-norm and appended; a direction whose A-norm is below 1e-10 of
    the original's is not appended (it lies in the span numerically).  A full
    space restarts from the latest solution: it is cleared and x itself
    (A-normalised) becomes its first vector, so the next start keeps the
    latest solution's direction (the paper does not say what a reset keeps;
    this is the reading taken)."""

    def __init__(self, P, max_vectors: int = 20):
        self.P = P
        self.L = max_vectors
        self.X = []
        self.BX = []

    def start(self, b):
        b = np.asarray(b, dtype=np.float64)
        xbar = np.zeros_like(b)
        for xt in self.X:
            xbar += self.P.dot(xt, b) * xt
        return xbar

    def update(self, x, xbar):
        P = self.P
        v = np.asarray(x, dtype=np.float64) - xbar
        if len(self.X) >= self.L:
            self.X, self.BX = [], []
            v = np.asarray(x, dtype=np.float64).copy()
        total = 0.0
        for _ in range(2):
            g = [P.dot(bt, v) for bt in self.BX]
            total += sum(c * c for c in g)
            for c, xt in zip(g, self.X):
                v = v - c * xt
        w = P.ax(v)
        nn = P.dot(v, w)
        if not (nn > 1e-20 * (total + nn)):
            return False
        s = 1.0 / np.sqrt(nn)
        self.X.append(v * s)
        self.BX.append(w * s)
        return True


def pipelined_pcg(P, b, x0=None, tol: float = 1e-10, max_iter: int = 100000):
    """Pipelined preconditioned CG (Ghysels and Vanroose 2014), the
    communication-reduced CG the paper's solver work builds on (Sec. II-B,
    reference on reducing communication in CG): the same Krylov iterates as
    Jacobi-PCG in exact arithmetic, with one reduction phase per iteration,
    (r, u), (w, u) and (r, r) together, overlapping the operator application
    n = A m.  Recurrences, with M = diag(Minv) and u = M r, w = A u, m = M w:
        gamma = (r, u), delta = (w, u), n = A m
        beta = gamma / gamma_prev, alpha = gamma / (delta - beta gamma / alpha_prev)
        (first iteration: beta = 0, alpha = gamma / delta)
        z = n + beta z, q = m + beta q, s = w + beta s, p = u + beta p
        x += alpha p, r -= alpha s, u -= alpha q, w -= alpha z
    Stops when the recursive ||r|| / ||b|| <= tol.  Returns (x, info) with
    the iterations, the recursive residual history and the true residual."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    Minv = P.minv()
    r = b - P.ax(x)
    u = Minv * r
    w = P.ax(u)
    bn = np.sqrt(P.dot(b, b))
    z = np.zeros_like(b)
    q = np.zeros_like(b)
    s = np.zeros_like(b)
    p = np.zeros_like(b)
    gamma_prev = alpha_prev = 0.0
    hist = []
    it = 0
    status = 1
    while it < max_iter:
        if bn == 0.0 or np.sqrt(P.dot(r, r)) / bn <= tol:
            status = 0
            break
        gamma = P.dot(r, u)
        delta = P.dot(w, u)
        m = Minv * w
        n = P.ax(m)
        if it == 0:
            beta = 0.0
            alpha = gamma / delta
        else:
            beta = gamma / gamma_prev
            alpha = gamma / (delta - beta * gamma / alpha_prev)
        if not np.isfinite(alpha) or alpha <= 0.0:
            status = 2
            break
        z = n + beta * z
        q = m + beta * q
        s = w + beta * s
        p = u + beta * p
        x = x + alpha * p
        r = r - alpha * s
        u = u - alpha * q
        w = w - alpha * z
        gamma_prev, alpha_prev = gamma, alpha
        it += 1
        hist.append(np.sqrt(P.dot(r, r)) / bn if bn > 0 else 0.0)
    rt = b - P.ax(x)
    return x, dict(status=status, iters=it, hist=np.array(hist),
                   relres=float(np.sqrt(P.dot(rt, rt)) / bn) if bn > 0 else 0.0)


def _ref_derivs(D: np.ndarray, u: np.ndarray, lx: int):
    """(du/dr, du/ds, du/dt) per element: D applied along i, j, k of [e][k][j][i]."""
    ue = u.reshape(-1, lx, lx, lx)
    dr = np.einsum("il,ekjl->ekji", D, ue)
    ds = np.einsum("jl,ekli->ekji", D, ue)
    dt = np.einsum("kl,elji->ekji", D, ue)
    return [d.reshape(-1) for d in (dr, ds, dt)]


def metrics(mesh) -> np.ndarray:
    """dr_s/dx_l at every local point, [n_local][s][l]: the inverse of the
    Jacobian matrix dx/dr, whose entries are the reference derivatives of the
    node coordinates (the isoparametric map of Sec. II-A)."""
    D = dmat(mesh.N)
    J = np.zeros((mesh.n_local, 3, 3))
    for m in range(3):
        d = _ref_derivs(D, np.ascontiguousarray(mesh.coords[m].reshape(-1)), mesh.lx)
        for s_ in range(3):
            J[:, m, s_] = d[s_]
    return np.linalg.inv(J)


def grad(mesh, u):
    """Collocation gradient du/dx_l = sum_s (dr_s/dx_l) du/dr_s, element by
    element (Sec. II-A: nodal GLL basis and D).  Returns [3][n_local]."""
    D = dmat(mesh.N)
    d = np.array(_ref_derivs(D, np.asarray(u, dtype=np.float64), mesh.lx))  # [s][n]
    M = metrics(mesh)                                                        # [n][s][l]
    return np.einsum("nsl,sn->ln", M, d)


def div(mesh, vx, vy, vz):
    return grad(mesh, vx)[0] + grad(mesh, vy)[1] + grad(mesh, vz)[2]


def curl(mesh, vx, vy, vz):
    gx, gy, gz = grad(mesh, vx), grad(mesh, vy), grad(mesh, vz)
    return np.array([gz[1] - gy[2], gx[2] - gz[0], gy[0] - gx[1]])


def pressure_rhs(P, mesh, vhat, omega, dt: float, Re: float):
    """Weak right-hand side of the pressure equation (Sec. II-A, eq.
    "pressure"): f = -div(vhat) / dt + (1/Re) div(curl(omega)) at the nodes,
    b = mask QQ^T (B f) (omega None: the term is dropped)."""
    f = -div(mesh, *vhat) / dt
    if omega is not None:
        f = f + div(mesh, *curl(mesh, *omega)) / Re
    return P.mass(f, assemble=True)


def _corner_index(lx: int) -> np.ndarray:
    """Local indices of an element's 8 corner nodes in the [k][j][i] order of
    an lx = 2 element (i fastest)."""
    return np.array([(k * lx + j) * lx + i for k in (0, lx - 1) for j in (0, lx - 1) for i in (0, lx - 1)])


class _CoarseMesh:
    def __init__(self, mesh):
        c = _corner_index(mesh.lx)
        n3 = mesh.lx ** 3
        sel = (np.arange(mesh.E)[:, None] * n3 + c[None, :]).reshape(-1)
        self.E, self.lx = mesh.E, 2
        self.coords = np.ascontiguousarray(mesh.coords.reshape(3, -1)[:, sel].reshape(3, mesh.E, 8))
        self.gid = np.ascontiguousarray(mesh.gid[sel])
        self.mask = np.ascontiguousarray(mesh.mask[sel])
        self.sel = sel


class SchwarzPrecond:
    """Two-level additive Schwarz preconditioner of the pressure solve (Sec.
    II-B: overlapping additive Schwarz with a coarse-grid solve of 10 P-CG
    iterations, after Lottes and Fischer 2005).  The paper gives no further
    detail; this is the reading taken, applied to an assembled residual r:
      z = Minv r                             (point Jacobi, every node)
      z_e,interior = A_box,e^-1 r_e,interior (each element's interior nodes,
          homogeneous Dirichlet on its boundary, by fast diagonalisation of
          the element approximated by a box with the mean lengths of its four
          edges per direction and its mean h1: separable 1-D stiffness K and
          mass W on [-1, 1], K S = W S Lambda, S^T W S = I, scaled to the box)
      z += P A_c^-1 R r                      (coarse grid: the same elements
          with N = 1 on their corner nodes; R r = QQ_c^T sum_L P^T r / mult,
          P the trilinear interpolation to the GLL nodes; A_c^-1 approximated
          by 10 Jacobi-PCG iterations from zero)
      z <- mask z.
    The subdomains do not overlap beyond the shared nodes (the coarse space
    and the Jacobi part on inter-element nodes couple them); the exact
    extended-element overlap of Lottes and Fischer is not reproduced."""

    def __init__(self, P, mesh, h1=None, coarse_iters: int = 10):
        lx, N = mesh.lx, mesh.lx - 1
        n3 = lx ** 3
        self.P, self.mesh, self.lx, self.E = P, mesh, lx, mesh.E
        self.Minv = P.minv()
        self.mult = P.mult()
        self.mask = np.asarray(mesh.mask, dtype=np.float64)
        self.coarse_iters = coarse_iters
        xi, rho = gll(N)
        D = dmat(N)
        K = D.T @ np.diag(rho) @ D
        self.ni = N - 1
        if self.ni > 0:
            Ki, Wi = K[1:N, 1:N], rho[1:N]
            C = Ki / np.sqrt(Wi)[:, None] / np.sqrt(Wi)[None, :]
            lam, V = np.linalg.eigh(C)
            self.lam = lam
            self.S = V / np.sqrt(Wi)[:, None]
        X = mesh.coords.reshape(3, mesh.E, n3)
        c = _corner_index(lx)
        Xc = X[:, :, c]  # [3][E][8], corner (i, j, k) bits = (q & 1, q >> 1 & 1, q >> 2)
        L = np.zeros((mesh.E, 3))
        for d in range(3):
            pairs = [(q, q | (1 << d)) for q in range(8) if not (q >> d) & 1]
            L[:, d] = np.mean([np.linalg.norm(Xc[:, :, b] - Xc[:, :, a], axis=0) for a, b in pairs], axis=0)
        self.L = L
        hh = np.ones(mesh.n_local) if h1 is None else np.asarray(h1, dtype=np.float64)
        self.h1m = hh.reshape(mesh.E, n3).mean(axis=1)
        self.cm = _CoarseMesh(mesh)
        self.Pc = Problem(self.cm, None if h1 is None else np.ascontiguousarray(hh[self.cm.sel]))
        phi = np.array([(1.0 - xi) / 2.0, (1.0 + xi) / 2.0])  # [c][i]
        i, j, k = np.meshgrid(np.arange(lx), np.arange(lx), np.arange(lx), indexing="xy")
        kk, jj, ii = np.meshgrid(np.arange(lx), np.arange(lx), np.arange(lx), indexing="ij")
        ii, jj, kk = ii.reshape(-1), jj.reshape(-1), kk.reshape(-1)
        self.Pw = np.array([phi[q & 1][ii] * phi[(q >> 1) & 1][jj] * phi[(q >> 2) & 1][kk] for q in range(8)]).T

    def local_solve(self, r):
        """The fast-diagonalisation part alone: interior nodes of every element."""
        lx, ni = self.lx, self.ni
        out = np.zeros_like(r)
        if ni <= 0:
            return out
        re = np.asarray(r).reshape(self.E, lx, lx, lx)
        ri = re[:, 1:lx - 1, 1:lx - 1, 1:lx - 1]  # [e][k][j][i]
        sc = np.sqrt(2.0 / self.L)                 # S_d = S sqrt(2 / L_d)
        lam = self.lam[None, :] * (4.0 / self.L[:, :, None] ** 2)  # [e][d][m]
        t = np.einsum("im,ekji->ekjm", self.S, ri) * sc[:, 0, None, None, None]
        t = np.einsum("jm,ekji->ekmi", self.S, t) * sc[:, 1, None, None, None]
        t = np.einsum("km,ekji->emji", self.S, t) * sc[:, 2, None, None, None]
        den = lam[:, 2, :, None, None] + lam[:, 1, None, :, None] + lam[:, 0, None, None, :]
        t = t / (den * self.h1m[:, None, None, None])
        t = np.einsum("km,emji->ekji", self.S, t) * sc[:, 2, None, None, None]
        t = np.einsum("jm,ekmi->ekji", self.S, t) * sc[:, 1, None, None, None]
        t = np.einsum("im,ekjm->ekji", self.S, t) * sc[:, 0, None, None, None]
        oe = out.reshape(self.E, lx, lx, lx)
        oe[:, 1:lx - 1, 1:lx - 1, 1:lx - 1] = t
        return out

    def restrict(self, r):
        rl = (np.asarray(r) / self.mult).reshape(self.E, -1) @ self.Pw  # [E][8]
        return self.Pc.gs(np.ascontiguousarray(rl.reshape(-1)), mask=True)

    def prolong(self, ec):
        return (np.asarray(ec).reshape(self.E, 8) @ self.Pw.T).reshape(-1)

    def __call__(self, r):
        r = np.asarray(r, dtype=np.float64)
        z = self.Minv * r
        if self.ni > 0:
            lx = self.lx
            zi = self.local_solve(r).reshape(self.E, lx, lx, lx)
            ze = z.reshape(self.E, lx, lx, lx)
            ze[:, 1:lx - 1, 1:lx - 1, 1:lx - 1] = zi[:, 1:lx - 1, 1:lx - 1, 1:lx - 1]
        ec, _ = self.Pc.pcg(self.restrict(r), tol=1e-300, max_iter=self.coarse_iters)
        z = z + self.prolong(ec)
        return z * self.mask


def fgmres(P, b, precond=None, restart: int = 30, tol: float = 1e-10, max_iter: int = 2000, x0=None):
    """Restarted flexible GMRES (Saad 1993) with right preconditioning, the
    Krylov method of the paper's pressure solve (Sec. II-B: restarted GMRES,
    Saad and Schultz 1986; flexible because the preconditioner's coarse solve
    is a fixed number of CG iterations): Arnoldi with classical Gram-Schmidt
    run twice in the unique-node inner product, Givens rotations on the
    Hessenberg matrix, x = x0 + Z y at the end of a cycle.  Stops when the
    rotated residual estimate |g_{j+1}| / ||b|| <= tol (checked against the
    true residual at each restart).  precond None: the identity."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    M = precond if precond is not None else (lambda v: v)
    bn = np.sqrt(P.dot(b, b))
    it, cycles, status = 0, 0, 1
    while True:
        r = b - P.ax(x)
        beta = np.sqrt(P.dot(r, r))
        if bn == 0.0 or beta / bn <= tol:
            status = 0
            break
        if it >= max_iter:
            break
        cycles += 1
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        g = np.zeros(restart + 1)
        g[0] = beta
        cs, sn = np.zeros(restart), np.zeros(restart)
        k = 0
        for j in range(restart):
            z = M(V[j])
            Z.append(z)
            w = P.ax(z)
            h = np.zeros(j + 2)
            for _ in range(2):
                c = np.array([P.dot(w, V[i]) for i in range(j + 1)])
                for i in range(j + 1):
                    w = w - c[i] * V[i]
                h[:j + 1] += c
            h[j + 1] = np.sqrt(P.dot(w, w))
            for i in range(j):
                t = cs[i] * h[i] + sn[i] * h[i + 1]
                h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1]
                h[i] = t
            den = np.hypot(h[j], h[j + 1])
            cs[j], sn[j] = h[j] / den, h[j + 1] / den
            h[j] = den
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            H[:j + 1, j] = h[:j + 1]
            it += 1
            k = j + 1
            if abs(g[j + 1]) / bn <= tol or it >= max_iter or h[j + 1] == 0.0:
                break
            V.append(w / np.sqrt(P.dot(w, w)))
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        for i in range(k):
            x = x + y[i] * Z[i]
    rt = b - P.ax(x)
    return x, dict(status=status, iters=it, cycles=cycles,
                   relres=float(np.sqrt(P.dot(rt, rt)) / bn) if bn > 0 else 0.0)
