"""Pins of the oracle's pipelined PCG (Ghysels and Vanroose 2014; the paper's
solver work on reducing communication in CG, Sec. II-B): in exact arithmetic
it produces the iterates of Jacobi-PCG, so on small problems its recursive
residual history and iterates follow the oracle's PCG within rounding, and it
reaches the dense solution."""
import numpy as np

import oracle
import workloads as W
import dense_ref


def test_pipelined_follows_pcg_history():
    m = W.box_mesh(3, 3, 2, 4, amp=0.06)
    h1 = W.h1_wavy(m)
    P = oracle.Problem(m, h1)
    b = W.random_global_rhs(m, 11)
    _, info = P.pcg(b, tol=1e-10, hist=True)
    xp, ip = oracle.pipelined_pcg(P, b, tol=1e-10)
    n = min(30, info["iters"])
    h0, h1_ = info["hist"][:n], ip["hist"][:n]
    assert np.max(np.abs(h1_ - h0) / h0) < 1e-6, np.max(np.abs(h1_ - h0) / h0)
    assert abs(ip["iters"] - info["iters"]) <= 3
    assert ip["status"] == 0 and ip["relres"] <= 2e-10


def test_pipelined_reaches_dense_solution():
    m = W.box_mesh(2, 2, 2, 3, amp=0.08)
    P = oracle.Problem(m)
    b = W.random_global_rhs(m, 5)
    K, Q, mask_g, _, _ = dense_ref.assembled(m)
    _, first = np.unique(m.gid, return_index=True)
    F = mask_g > 0
    xg = np.zeros(K.shape[0])
    xg[F] = np.linalg.solve(K[np.ix_(F, F)], b[first][F])
    x, info = oracle.pipelined_pcg(P, b, tol=1e-12)
    assert info["status"] == 0
    assert np.linalg.norm(x - Q @ xg) <= 1e-9 * np.linalg.norm(xg)


def test_planted_mistake_in_alpha_is_caught():
    """The pin above fails for the plausible slip alpha = gamma / delta at
    every iteration (dropping the beta gamma / alpha_prev correction)."""
    m = W.box_mesh(3, 3, 2, 4, amp=0.06)
    P = oracle.Problem(m, W.h1_wavy(m))
    b = W.random_global_rhs(m, 11)
    _, info = P.pcg(b, tol=1e-10, hist=True)
    Minv = P.minv()
    r = b.copy()
    u = Minv * r
    w = P.ax(u)
    z = q = s = p = np.zeros_like(b)
    hist = []
    bn = np.sqrt(P.dot(b, b))
    for it in range(30):
        gamma, delta = P.dot(r, u), P.dot(w, u)
        mm = Minv * w
        n = P.ax(mm)
        beta = 0.0 if it == 0 else gamma / gprev
        alpha = gamma / delta  # the planted slip
        z, q, s, p = n + beta * z, mm + beta * q, w + beta * s, u + beta * p
        r, u, w = r - alpha * s, u - alpha * q, w - alpha * z
        gprev = gamma
        hist.append(np.sqrt(P.dot(r, r)) / bn)
    h0 = info["hist"][:30]
    assert np.max(np.abs(np.array(hist) - h0) / h0) > 1e-3
