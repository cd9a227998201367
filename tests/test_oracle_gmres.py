"""Pins of the oracle's pressure solver of Sec. II-B: restarted flexible
GMRES with the two-level Schwarz preconditioner (fast-diagonalisation
element-interior solves, point Jacobi on inter-element nodes, a coarse grid of
the element corners solved by 10 Jacobi-PCG iterations).  The local solve is
the exact inverse of the interior block on box elements; the prolongation
reproduces trilinear fields; FGMRES with the identity reaches the dense
solution; the preconditioned iteration count does not grow with the mesh,
where Jacobi-PCG's does; planted mistakes fail these pins."""
import numpy as np
import pytest

import oracle
import workloads as W
import dense_ref


@pytest.mark.parametrize("dims,N", [((2, 1, 1), 5), ((1, 3, 2), 4), ((2, 2, 1), 7)])
def test_fast_diagonalisation_is_the_interior_inverse_on_boxes(dims, N):
    m = W.box_mesh(*dims, N)
    P = oracle.Problem(m)
    M = oracle.SchwarzPrecond(P, m)
    Ae, _ = dense_ref.element_matrices(m)
    lx = N + 1
    idx = np.arange(lx ** 3).reshape(lx, lx, lx)[1:-1, 1:-1, 1:-1].reshape(-1)
    rng = np.random.default_rng(N)
    for e in range(m.E):
        r = np.zeros(m.n_local)
        r[e * lx ** 3 + idx] = rng.standard_normal(idx.size)
        z = M.local_solve(r)
        ref = np.linalg.solve(Ae[e][np.ix_(idx, idx)], r[e * lx ** 3 + idx])
        assert np.max(np.abs(z[e * lx ** 3 + idx] - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_prolongation_reproduces_trilinear_fields():
    m = W.box_mesh(3, 2, 2, 6)
    P = oracle.Problem(m)
    M = oracle.SchwarzPrecond(P, m)
    f = lambda x, y, z: 1.0 + 2.0 * x - y + 0.5 * z + 3.0 * x * y - x * z + 0.7 * y * z + 2.0 * x * y * z
    cx, cy, cz = M.cm.coords[0].reshape(-1), M.cm.coords[1].reshape(-1), M.cm.coords[2].reshape(-1)
    x, y, z = m.xyz()
    assert np.max(np.abs(M.prolong(f(cx, cy, cz)) - f(x, y, z))) <= 1e-13 * 10


def test_fgmres_identity_reaches_dense_solution():
    m = W.box_mesh(2, 2, 2, 3, amp=0.08)
    P = oracle.Problem(m)
    b = W.random_global_rhs(m, 5)
    K, Q, mask_g, _, _ = dense_ref.assembled(m)
    _, first = np.unique(m.gid, return_index=True)
    F = mask_g > 0
    xg = np.zeros(K.shape[0])
    xg[F] = np.linalg.solve(K[np.ix_(F, F)], b[first][F])
    x, info = oracle.fgmres(P, b, None, restart=10, tol=1e-12)
    assert info["status"] == 0 and info["cycles"] > 1
    assert np.linalg.norm(x - Q @ xg) <= 1e-9 * np.linalg.norm(xg)


def _iters(n, precond_cls=oracle.SchwarzPrecond):
    m = W.box_mesh(n, n, n, 5, amp=0.05)
    h1 = W.h1_wavy(m)
    P = oracle.Problem(m, h1)
    b = W.random_global_rhs(m, 3)
    x, info = oracle.fgmres(P, b, precond_cls(P, m, h1), tol=1e-10)
    _, i64 = P.pcg(b, tol=1e-10)
    assert info["status"] == 0 and info["relres"] <= 1e-10
    xo, _ = P.pcg(b, tol=1e-12)
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
    return info["iters"], i64["iters"]


def test_two_level_preconditioner_is_mesh_independent():
    g3, p3 = _iters(3)
    g6, p6 = _iters(6)
    assert g6 <= 1.15 * g3 and g6 < 80, (g3, g6)
    assert p6 >= 1.8 * p3, (p3, p6)
    assert g6 < 0.5 * p6


class _NoCoarse(oracle.SchwarzPrecond):
    """Planted mistake: the coarse correction is dropped."""

    def prolong(self, ec):
        return np.zeros(self.mesh.n_local)


class _TransposedModes(oracle.SchwarzPrecond):
    """Planted mistake: the modal matrix is used transposed."""

    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.S = self.S.T.copy()


def test_planted_mistakes_are_caught():
    g3, _ = _iters(3, _NoCoarse)
    g6, _ = _iters(6, _NoCoarse)
    assert g6 > 1.15 * g3, (g3, g6)  # mesh-dependent without the coarse grid
    m = W.box_mesh(2, 1, 1, 5)
    P = oracle.Problem(m)
    M = _TransposedModes(P, m)
    Ae, _ = dense_ref.element_matrices(m)
    idx = np.arange(216).reshape(6, 6, 6)[1:-1, 1:-1, 1:-1].reshape(-1)
    r = np.zeros(m.n_local)
    r[idx] = np.random.default_rng(0).standard_normal(idx.size)
    ref = np.linalg.solve(Ae[0][np.ix_(idx, idx)], r[idx])
    assert np.max(np.abs(M.local_solve(r)[idx] - ref)) > 1e-3 * np.max(np.abs(ref))
