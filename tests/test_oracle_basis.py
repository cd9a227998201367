"""Pins of the oracle's GLL basis and derivative matrix (Sec. II-A) to closed
forms, quadrature exactness and polynomial identities."""
import math
import os

import numpy as np
import pytest

import oracle
import dense_ref

GOLD = os.path.join(os.path.dirname(__file__), "golden", "gll_closed_forms.txt")


def _ev(s: str) -> float:
    return float(eval(s, {"__builtins__": {}}, {"sqrt": math.sqrt}))


def _golden():
    gll, stiff = {}, {}
    with open(GOLD) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "gll":
                gll.setdefault(int(tok[1]), []).append((_ev(tok[2]), _ev(tok[3])))
            elif tok[0] == "stiff":
                stiff.setdefault(int(tok[1]), {})[int(tok[2])] = [_ev(t) for t in tok[3:]]
    return gll, {N: np.array([rows[i] for i in sorted(rows)]) for N, rows in stiff.items()}


GLL_GOLD, STIFF_GOLD = _golden()


@pytest.mark.parametrize("N", sorted(GLL_GOLD))
def test_gll_closed_forms(N):
    xi, rho = oracle.gll(N)
    nodes = np.array([a for a, _ in GLL_GOLD[N]])
    wts = np.array([b for _, b in GLL_GOLD[N]])
    np.testing.assert_allclose(xi, nodes, rtol=0, atol=1e-15)
    np.testing.assert_allclose(rho, wts, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("N", range(1, 16))
def test_gll_weights_sum_and_symmetry(N):
    xi, rho = oracle.gll(N)
    assert abs(rho.sum() - 2.0) < 1e-14
    np.testing.assert_allclose(xi, -xi[::-1], atol=1e-15)
    np.testing.assert_allclose(rho, rho[::-1], rtol=1e-14)
    assert np.all(np.diff(xi) > 0)


@pytest.mark.parametrize("N", range(1, 16))
def test_gll_quadrature_exact_to_degree_2N_minus_1(N):
    xi, rho = oracle.gll(N)
    for k in range(0, 2 * N):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(rho @ xi ** k - exact) < 2e-14, (N, k)
    if N >= 2:
        # GLL is not exact at degree 2N (a known property): the pin is not vacuous
        k = 2 * N
        assert abs(rho @ xi ** k - 2.0 / (k + 1)) > 1e-12


@pytest.mark.parametrize("N", range(1, 16))
def test_gll_matches_independent_construction(N):
    """Nodes vs numpy's Legendre roots; weights vs exact integrals of the Lagrange basis."""
    xi, rho = oracle.gll(N)
    xr, rr, _ = dense_ref.basis_data(N)
    np.testing.assert_allclose(xi, xr, atol=2e-15)
    # monomial-basis integration loses digits at high N; a formula error would be O(1)
    np.testing.assert_allclose(rho, rr, rtol=1e-12 if N < 10 else 1e-8, atol=1e-13)


@pytest.mark.parametrize("N", range(1, 16))
def test_dmat_exact_on_polynomials(N):
    D = oracle.dmat(N)
    xi, _ = oracle.gll(N)
    for m in range(0, N + 1):
        d = D @ xi ** m
        ref = m * xi ** (m - 1) if m > 0 else np.zeros_like(xi)
        assert np.max(np.abs(d - ref)) < 1e-13 * max(1.0, N * N), (N, m)


@pytest.mark.parametrize("N", range(1, 16))
def test_dmat_rows_centro_symmetry(N):
    D = oracle.dmat(N)
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-13 * N * N)
    np.testing.assert_allclose(D[::-1, ::-1], -D, atol=1e-13 * N * N)
    assert D[0, 0] == pytest.approx(-N * (N + 1) / 4.0, rel=1e-15)
    assert D[N, N] == pytest.approx(N * (N + 1) / 4.0, rel=1e-15)


@pytest.mark.parametrize("N", range(1, 12))
def test_dmat_matches_lagrange_derivatives(N):
    D = oracle.dmat(N)
    _, _, Dr = dense_ref.basis_data(N)
    np.testing.assert_allclose(D, Dr, atol=1e-11 * N * N)


@pytest.mark.parametrize("N", range(1, 10))
def test_stiffness_1d(N):
    D = oracle.dmat(N)
    _, rho = oracle.gll(N)
    K = D.T @ np.diag(rho) @ D
    np.testing.assert_allclose(K, dense_ref.stiffness_1d_exact(N), atol=1e-11 * N ** 3)
    if N in STIFF_GOLD:
        np.testing.assert_allclose(K, STIFF_GOLD[N], atol=1e-14)


def test_paper_point_count_convention():
    """n_L = E (N+1)^3 reproduces the paper's quoted point counts."""
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.txt")
    rows = [l.split("#")[0].split() for l in open(path)]
    rows = [r for r in rows if r]
    assert rows
    for r in rows:
        E, N, quoted, tol = int(r[0]), int(r[1]), float(r[2]), float(r[3])
        assert abs(E * (N + 1) ** 3 - quoted) / quoted < tol
