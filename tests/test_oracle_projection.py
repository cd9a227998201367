"""Pins of the oracle's projection onto previous solutions (Sec. II-B, after
Fischer 1998): the basis is A-orthonormal; a right-hand side whose solution
lies in the span is solved by the projection alone; the projected start is
the dense Galerkin (A-orthogonal) projection; on a slowly varying sequence of
right-hand sides the projection shrinks the start residual and the
iterations; the space resets when full."""
import numpy as np

import oracle
import workloads as W
import dense_ref


def _problem():
    m = W.box_mesh(3, 2, 2, 3, amp=0.08)
    h1 = W.h1_wavy(m)
    return m, h1, oracle.Problem(m, h1)


def _sequence(m, P, k, seed=0):
    """b(t_k): a fixed smooth forcing plus a slowly rotating second mode."""
    x, y, z = m.xyz()
    t = 0.05 * k
    f = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z) * (1.0 + 0.3 * np.sin(t)) \
        + 0.5 * np.cos(t) * np.sin(2 * np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z) \
        + 0.2 * np.sin(2 * t) * x * y * z
    return P.mass(f, assemble=True)


def test_basis_is_a_orthonormal_and_solution_in_span_is_exact():
    m, h1, P = _problem()
    pr = oracle.Projection(P, 20)
    for k in range(6):
        b = _sequence(m, P, k)
        xbar = pr.start(b)
        x, info = P.pcg(b, x0=xbar, tol=1e-12)
        pr.update(x, xbar)
    G = np.array([[P.dot(a, bt) for bt in pr.BX] for a in pr.X])
    assert np.max(np.abs(G - np.eye(len(pr.X)))) < 1e-10
    # a solution inside the span: y = 0.3 xt_0 - 1.2 xt_3 + xt_5, b = A y
    y = 0.3 * pr.X[0] - 1.2 * pr.X[3] + pr.X[5]
    b = P.ax(y)
    xbar = pr.start(b)
    assert np.linalg.norm(xbar - y) <= 1e-10 * np.linalg.norm(y)
    r = b - P.ax(xbar)
    assert np.sqrt(P.dot(r, r) / P.dot(b, b)) <= 1e-10


def test_projected_start_is_the_dense_galerkin_projection():
    """xbar = V c with (V^T K V) c = V^T b on the free unique nodes, K the dense
    assembled matrix from numpy polynomials and Jacobians."""
    m, h1, P = _problem()
    pr = oracle.Projection(P, 20)
    for k in range(5):
        b = _sequence(m, P, k)
        xbar = pr.start(b)
        x, _ = P.pcg(b, x0=xbar, tol=1e-12)
        pr.update(x, xbar)
    K, Q, mask_g, _, _ = dense_ref.assembled(m, h1)
    _, first = np.unique(m.gid, return_index=True)
    F = mask_g > 0
    V = np.array([xt[first][F] for xt in pr.X]).T
    b = _sequence(m, P, 9)
    bg = b[first][F]
    Kf = K[np.ix_(F, F)]
    c = np.linalg.solve(V.T @ Kf @ V, V.T @ bg)
    xbar = pr.start(b)
    assert np.linalg.norm(xbar[first][F] - V @ c) <= 1e-10 * np.linalg.norm(V @ c)


def test_projection_cuts_iterations_and_resets_when_full():
    m, h1, P = _problem()
    pr = oracle.Projection(P, 4)
    its, starts = [], []
    for k in range(9):
        b = _sequence(m, P, k)
        xbar = pr.start(b)
        r = b - P.ax(xbar)
        starts.append(np.sqrt(P.dot(r, r) / P.dot(b, b)))
        x, info = P.pcg(b, x0=xbar, tol=1e-10)
        its.append(info["iters"])
        xo, _ = P.pcg(b, tol=1e-12)
        assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
        pr.update(x, xbar)
        assert len(pr.X) == (k % 4) + 1
    assert starts[0] == 1.0
    # with three or more vectors the start residual of this smooth sequence is small
    assert max(starts[3], starts[7]) < 1e-3, starts
    assert its[3] < 0.5 * its[0], its


class _StartWithWrongCoefficients(oracle.Projection):
    """Planted mistake: coefficients <A xt_i, b> instead of <xt_i, b>."""

    def start(self, b):
        xbar = np.zeros_like(b)
        for xt, bt in zip(self.X, self.BX):
            xbar += self.P.dot(bt, b) * xt
        return xbar


def test_reset_restarts_from_the_latest_solution():
    """A full space is cleared and restarts from the latest solution x: right
    after the reset it holds x / ||x||_A, so a right-hand side that is a
    multiple of the latest one is solved by the projection alone."""
    m, h1, P = _problem()
    pr = oracle.Projection(P, 3)
    for k in range(4):
        b = _sequence(m, P, k)
        xbar = pr.start(b)
        x, _ = P.pcg(b, x0=xbar, tol=1e-12)
        pr.update(x, xbar)
    assert len(pr.X) == 1
    xn = x / np.sqrt(P.dot(x, P.ax(x)))
    assert np.linalg.norm(pr.X[0] - xn) <= 1e-12 * np.linalg.norm(xn)
    b2 = 3.0 * b
    r = b2 - P.ax(pr.start(b2))
    assert np.sqrt(P.dot(r, r) / P.dot(b2, b2)) <= 1e-10


class _EuclideanGramSchmidt(oracle.Projection):
    """Planted mistake: orthogonalises in the unique-node inner product
    instead of the A inner product."""

    def update(self, x, xbar):
        P = self.P
        v = np.asarray(x, dtype=np.float64) - xbar
        if len(self.X) >= self.L:
            self.X, self.BX = [], []
            v = np.asarray(x, dtype=np.float64).copy()
        for _ in range(2):
            for xt in self.X:
                v = v - P.dot(xt, v) / P.dot(xt, xt) * xt
        w = P.ax(v)
        nn = P.dot(v, w)
        self.X.append(v / np.sqrt(nn))
        self.BX.append(w / np.sqrt(nn))
        return True


def _pins_fail(cls):
    m, h1, P = _problem()
    pr = cls(P, 20)
    for k in range(5):
        b = _sequence(m, P, k)
        xbar = pr.start(b)
        x, _ = P.pcg(b, x0=xbar, tol=1e-12)
        pr.update(x, xbar)
    if len(pr.X) != 5:  # five independent solves give five directions
        return True
    G = np.array([[P.dot(a, bt) for bt in pr.BX] for a in pr.X])
    bad_basis = np.max(np.abs(G - np.eye(len(pr.X)))) >= 1e-10
    y = 0.3 * pr.X[0] - 1.2 * pr.X[3]
    xbar = pr.start(P.ax(y))
    bad_start = np.linalg.norm(xbar - y) > 1e-10 * np.linalg.norm(y)
    return bad_basis or bad_start


def test_pins_catch_planted_mistakes():
    assert not _pins_fail(oracle.Projection)
    assert _pins_fail(_StartWithWrongCoefficients)
    assert _pins_fail(_EuclideanGramSchmidt)
