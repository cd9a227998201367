"""GPU parity of the projection onto previous solutions (Sec. II-B, after
Fischer 1998) against the oracle's restatement (oracle.Projection), through
the C ABI: on a slowly varying sequence of right-hand sides the projected
start residuals, iteration counts and solutions follow the oracle's; a
solution in the span needs no iteration; the space resets when full and on
request; batch handles refuse the option."""
import numpy as np
import pytest

import oracle
import workloads as W
import paper_2207_07098_gb300 as S
from gpu_helpers import Handle, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _sequence(m, P, k):
    """b(t_k) of a forcing that drifts in x (every step brings new content)."""
    x, y, z = m.xyz()
    t = 0.03 * k
    f = np.sin(np.pi * (x + t)) * np.sin(np.pi * y) * np.sin(np.pi * z) * (1.0 + x * y) \
        + 0.3 * np.cos(3 * np.pi * (y - t)) * z
    return P.mass(f, assemble=True)


def _oracle_relres(P, x, b):
    r = b - P.ax(x)
    return np.sqrt(P.dot(r, r) / P.dot(b, b))


@pytest.mark.parametrize("mode", [S.SEM_MODE_FP64, S.SEM_MODE_MIXED_IR])
def test_projection_sequence_follows_oracle(mode):
    m = W.box_mesh(4, 3, 3, 7, amp=0.05)
    h1 = W.h1_wavy(m)
    P = oracle.Problem(m, h1)
    H = Handle(m, h1)
    pr = oracle.Projection(P, 4)
    starts = []
    for k in range(10):
        b = _sequence(m, P, k)
        x, st = H.solve(b, tol=TOL, mode=mode, projection=4)
        xbar = pr.start(b)
        r0 = b - P.ax(xbar)
        start = np.sqrt(P.dot(r0, r0) / P.dot(b, b))
        xo, info = P.pcg(b, x0=xbar, tol=TOL)
        pr.update(xo, xbar)
        assert st["status"] == S.SEM_OK and st["relres"] <= TOL, (k, st)
        assert _oracle_relres(P, x, b) <= 1.05 * TOL, k
        assert rel_err(x, xo)[0] <= 1e-7, k
        assert abs(st["relres_start"] - start) <= 0.05 * start + 1e-9, (k, st["relres_start"], start)
        if mode == S.SEM_MODE_FP64:
            assert abs(st["iterations"] - info["iters"]) <= max(3, info["iters"] // 20), (k, st, info)
        assert S.sem_projection_size(H.h) == len(pr.X) == (k % 4) + 1
        starts.append(st["relres_start"])
    # the projection pays off on this sequence: with three or more vectors the
    # start residual is far below that of x0 = 0
    assert starts[0] == 1.0 and max(starts[3], starts[7]) < 0.05, starts


def test_solution_in_span_and_reset():
    m, h1, b = W.deformed_cube(4, 5, seed=2)
    P = oracle.Problem(m, h1)
    H = Handle(m, h1)
    x1, s1 = H.solve(b, tol=TOL, projection=8)
    assert s1["relres_start"] == 1.0 and S.sem_projection_size(H.h) == 1
    # 2.5 b: its solution 2.5 x1 lies in the span of the first increment
    x2, s2 = H.solve(2.5 * b, tol=TOL, projection=8)
    assert s2["relres_start"] <= 1e-9 and s2["iterations"] == 0, s2
    assert _oracle_relres(P, x2, 2.5 * b) <= 1.05 * TOL
    S.sem_projection_reset(H.h)
    assert S.sem_projection_size(H.h) == 0
    _, s3 = H.solve(b, tol=TOL, projection=8)
    assert s3["relres_start"] == 1.0 and s3["iterations"] == s1["iterations"]


def test_batch_refuses_projection():
    import torch
    ms = [W.box_mesh(2, 2, 2, 3), W.box_mesh(1, 2, 2, 4)]
    h = S.sem_setup_batch([(m.E, m.lx, m.coords, m.gid, m.mask, None) for m in ms])
    try:
        b = torch.zeros(sum(m.n_local for m in ms), dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        with pytest.raises(S.SemError) as ei:
            S.sem_cg_solve_batch(h, x, b, 2, {"projection": 4})
        assert ei.value.status == S.SEM_EINVAL
    finally:
        S.sem_destroy(h)


@pytest.mark.parametrize("prec", [S.SEM_FP64, S.SEM_FP32])
def test_projection_with_the_gmres_pressure_solver(prec):
    """The paper pairs projection with its GMRES pressure solve: the same
    projected start residuals as the oracle's projection, solutions at the
    true 1e-10, and fewer GMRES iterations once the space holds vectors."""
    m = W.box_mesh(4, 3, 3, 7, amp=0.05)
    h1 = W.h1_wavy(m)
    P = oracle.Problem(m, h1)
    H = Handle(m, h1, flags=S.SEM_FLAG_SCHWARZ)
    pr = oracle.Projection(P, 4)
    its = []
    for k in range(6):
        b = _sequence(m, P, k)
        x, st = H.solve(b, tol=TOL, mode=S.SEM_MODE_GMRES, precision=prec, projection=4)
        xbar = pr.start(b)
        r0 = b - P.ax(xbar)
        start = np.sqrt(P.dot(r0, r0) / P.dot(b, b))
        xo, _ = P.pcg(b, x0=xbar, tol=TOL)
        pr.update(xo, xbar)
        assert st["status"] == S.SEM_OK and st["relres"] <= TOL, (k, st)
        assert _oracle_relres(P, x, b) <= 1.05 * TOL, k
        assert abs(st["relres_start"] - start) <= 0.05 * start + 1e-9, (k, st["relres_start"], start)
        its.append(st["iterations"])
    assert max(its[3:]) < its[0], its
