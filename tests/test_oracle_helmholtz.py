"""Pins of the oracle's Helmholtz operator A = QQ^T (h1 K + h2 B): the
velocity equation's implicit viscous term gives a Helmholtz problem (Sec.
II-A), with h1 weighing the stiffness and h2 the GLL-quadrature mass
(v, h2 u) = sum rho rho rho J h2 v u.  Pinned to the dense brute-force
construction, a closed form on constants, positive definiteness without
Dirichlet nodes, and spectral convergence to a manufactured solution."""
import numpy as np

import oracle
import workloads as W
import dense_ref


def _helmholtz_case(seed=3):
    m = W.box_mesh(3, 2, 2, 3, amp=0.1, jitter=0.02, seed=seed)
    h1 = W.h1_wavy(m)
    x, y, z = m.xyz()
    h2 = 2.0 + np.cos(3.0 * x) * np.sin(2.0 * y) + z
    return m, h1, h2


def test_constants_give_the_assembled_mass_term():
    """Stiffness annihilates constants (K 1 = 0), so without Dirichlet nodes
    QQ^T A_L 1 = QQ^T (h2 B): the h2 B term, weighted per point, assembled."""
    m, h1, h2 = _helmholtz_case()
    m.mask[:] = 1
    P = oracle.Problem(m, h1)
    P.set_h2(h2)
    _, B = P.geom()
    ref = P.gs(h2 * B, mask=False)
    got = P.ax(np.ones(m.n_local))
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    P.set_h2(None)
    assert np.max(np.abs(P.ax(np.ones(m.n_local)))) <= 1e-12 * np.max(np.abs(ref))


def test_dense_helmholtz_matrix_and_diagonal():
    """A u = Q (mask (K + Q^T diag(h2 B) Q) u_g) with K, B from numpy
    polynomials, Jacobians and an explicit Q; the Jacobi diagonal is the
    diagonal of that dense matrix."""
    m, h1, h2 = _helmholtz_case()
    P = oracle.Problem(m, h1)
    P.set_h2(h2)
    K, Q, mask_g, Ae, Bm = dense_ref.assembled(m, h1)
    H = K + Q.T @ np.diag(h2 * Bm.reshape(-1)) @ Q
    ug = np.random.default_rng(1).standard_normal(Q.shape[1])
    ref = Q @ (mask_g * (H @ ug))
    assert np.max(np.abs(P.ax(Q @ ug) - ref)) <= 1e-12 * np.max(np.abs(ref))
    _, inv = np.unique(m.gid, return_inverse=True)
    ref_minv = np.where(m.mask > 0, 1.0 / np.diag(H)[inv], 0.0)
    np.testing.assert_allclose(P.minv(), ref_minv, rtol=1e-12)


def test_helmholtz_without_dirichlet_is_spd_and_pcg_matches_dense():
    """With h2 > 0 the operator is SPD even with no Dirichlet node (Neumann
    Helmholtz): Jacobi-PCG reaches the dense solution."""
    m, h1, h2 = _helmholtz_case(4)
    m.mask[:] = 1
    P = oracle.Problem(m, h1)
    P.set_h2(h2)
    K, Q, mask_g, Ae, Bm = dense_ref.assembled(m, h1)
    H = K + Q.T @ np.diag(h2 * Bm.reshape(-1)) @ Q
    assert np.min(np.linalg.eigvalsh(H)) > 0
    b = W.random_global_rhs(m, 7)
    _, first = np.unique(m.gid, return_index=True)
    xg = np.linalg.solve(H, b[first])
    x, info = P.pcg(b, tol=1e-13, max_iter=2000)
    assert info["status"] == 0
    assert np.linalg.norm(x - Q @ xg) <= 1e-10 * np.linalg.norm(xg)


def test_helmholtz_spectral_convergence():
    """-lap u + lambda u = (3 pi^2 + lambda) sin(pi x) sin(pi y) sin(pi z) on the
    unit cube, u = 0 on the boundary (h1 = 1, h2 = lambda): the nodal error
    falls geometrically with N on 2^3 elements."""
    lam = 50.0
    errs = []
    for N in (3, 5, 7, 9):
        m = W.box_mesh(2, 2, 2, N)
        P = oracle.Problem(m)
        P.set_h2(np.full(m.n_local, lam))
        f = (3.0 * np.pi ** 2 + lam) / (3.0 * np.pi ** 2) * W.forcing_sines(m)
        b = P.mass(f, assemble=True)
        x, info = P.pcg(b, tol=1e-13, max_iter=5000)
        assert info["status"] == 0
        errs.append(np.max(np.abs(x - W.exact_sines(m))))
    assert all(errs[q + 1] < 0.1 * errs[q] for q in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-7, errs
