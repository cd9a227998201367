"""GPU parity of the paper's pressure solver (Sec. II-B): restarted flexible
GMRES with the two-level Schwarz preconditioner, through the C ABI, against
the oracle's restatement (oracle.SchwarzPrecond, oracle.fgmres): the
preconditioner application itself, the solve's iteration count and true
residual (by the oracle's operator), and the mesh-independent iteration
count the coarse grid gives."""
import numpy as np
import pytest

import oracle
import workloads as W
import paper_2207_07098_gb300 as S
from gpu_helpers import Handle, dev, host, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _oracle_relres(P, x, b):
    r = b - P.ax(x)
    return np.sqrt(P.dot(r, r) / P.dot(b, b))


CASES = [("deformed", 3, 5), ("deformed", 4, 7), ("jitter", 3, 4), ("annulus", 0, 6)]


def _case(kind, n, N):
    if kind == "deformed":
        m = W.box_mesh(n, n, n, N, amp=0.05)
        return m, W.h1_wavy(m)
    if kind == "jitter":
        m = W.box_mesh(n, n, 2, N, amp=0.08, jitter=0.2 / (N * N), seed=2)
        return m, W.h1_wavy(m)
    m = W.annulus_mesh(n_theta=12, n_r=4, n_z=3, N=N)
    return m, None


@pytest.mark.parametrize("kind,n,N", CASES)
def test_schwarz_preconditioner_matches_oracle(kind, n, N):
    import torch
    m, h1 = _case(kind, n, N)
    P = oracle.Problem(m, h1)
    M = oracle.SchwarzPrecond(P, m, h1)
    H = Handle(m, h1, flags=S.SEM_FLAG_SCHWARZ)
    r = P.gs(W.random_local_field(m, 7), mask=True)  # an assembled, masked residual
    z = torch.empty(m.n_local, dtype=torch.float64, device="cuda")
    S.sem_schwarz_apply(H.h, dev(r, torch.float64), z)
    e2, einf = rel_err(host(z), M(r))
    assert e2 <= 1e-10 and einf <= 1e-9, (e2, einf)


@pytest.mark.parametrize("kind,n,N", CASES)
def test_gmres_schwarz_solve_matches_oracle(kind, n, N):
    m, h1 = _case(kind, n, N)
    P = oracle.Problem(m, h1)
    H = Handle(m, h1, flags=S.SEM_FLAG_SCHWARZ)
    b = W.random_global_rhs(m, 13)
    x, st = H.solve(b, tol=TOL, mode=S.SEM_MODE_GMRES)
    assert st["status"] == S.SEM_OK and st["relres"] <= TOL, st
    assert _oracle_relres(P, x, b) <= 1.05 * TOL
    _, info = oracle.fgmres(P, b, oracle.SchwarzPrecond(P, m, h1), restart=20, tol=TOL)
    assert abs(st["iterations"] - info["iters"]) <= max(3, info["iters"] // 10), (st, info)
    xo, _ = P.pcg(b, tol=1e-12)
    assert rel_err(x, xo)[0] <= 1e-8


def test_gmres_iterations_do_not_grow_with_the_mesh():
    its = []
    for n in (3, 6):
        m = W.box_mesh(n, n, n, 7, amp=0.05)
        h1 = W.h1_wavy(m)
        H = Handle(m, h1, flags=S.SEM_FLAG_SCHWARZ)
        b = W.random_global_rhs(m, 3)
        _, st = H.solve(b, tol=TOL, mode=S.SEM_MODE_GMRES)
        _, sp = H.solve(b, tol=TOL, mode=S.SEM_MODE_FP64)
        assert st["status"] == S.SEM_OK
        its.append((st["iterations"], sp["iterations"]))
    (g3, p3), (g6, p6) = its
    assert g6 <= 1.15 * g3 and p6 >= 1.8 * p3, its


def test_gmres_needs_the_schwarz_setup():
    m, h1 = _case("deformed", 2, 3)
    H = Handle(m, h1)
    with pytest.raises(S.SemError) as ei:
        H.solve(W.random_global_rhs(m, 1), tol=TOL, mode=S.SEM_MODE_GMRES)
    assert ei.value.status == S.SEM_EINVAL


# FP32 arithmetic in the local solves, restriction and prolongation: unit
# roundoff 2^-24 = 6e-8 through six contraction passes of length lx - 2 <= 5,
# the Jacobi product and the 8-term corner sums, and the coarse CG (FP64) fed
# with a rounded right-hand side; 1e-5 relative bounds those by two orders of
# magnitude margin while any indexing or table mistake gives O(1) errors.
TOL_SCHWARZ_F32 = 1e-5


@pytest.mark.parametrize("kind,n,N", CASES)
def test_schwarz_preconditioner_fp32_matches_oracle(kind, n, N):
    import torch
    m, h1 = _case(kind, n, N)
    P = oracle.Problem(m, h1)
    M = oracle.SchwarzPrecond(P, m, h1)
    H = Handle(m, h1, flags=S.SEM_FLAG_SCHWARZ)
    r = P.gs(W.random_local_field(m, 7), mask=True).astype(np.float32).astype(np.float64)
    z = torch.empty(m.n_local, dtype=torch.float32, device="cuda")
    S.sem_schwarz_apply32(H.h, dev(r, torch.float32), z)
    e2, einf = rel_err(host(z).astype(np.float64), M(r))
    assert e2 <= TOL_SCHWARZ_F32 and einf <= 10 * TOL_SCHWARZ_F32, (e2, einf)


@pytest.mark.parametrize("kind,n,N", CASES)
def test_mixed_gmres_reaches_fp64_accuracy(kind, n, N):
    """FP32 restart cycles inside FP64 refinement: the same 1e-10 true residual
    (by the oracle's operator) and solution as the FP64 form, at most a few
    more iterations."""
    m, h1 = _case(kind, n, N)
    P = oracle.Problem(m, h1)
    H = Handle(m, h1, flags=S.SEM_FLAG_SCHWARZ)
    b = W.random_global_rhs(m, 13)
    x64, s64 = H.solve(b, tol=TOL, mode=S.SEM_MODE_GMRES)
    x, st = H.solve(b, tol=TOL, mode=S.SEM_MODE_GMRES, precision=S.SEM_FP32)
    assert st["status"] == S.SEM_OK and st["relres"] <= TOL, st
    assert _oracle_relres(P, x, b) <= 1.05 * TOL
    assert st["iterations"] <= 1.5 * s64["iterations"] + 10, (st, s64)
    xo, _ = P.pcg(b, tol=1e-12)
    assert rel_err(x, xo)[0] <= 1e-8


@pytest.mark.parametrize("prec,pc", [(S.SEM_FP64, S.SEM_FP32), (S.SEM_FP64_PAIR, S.SEM_FP64),
                                     (S.SEM_FP64_PAIR, S.SEM_FP32)])
def test_gmres_fp64_operator_and_preconditioner_forms(prec, pc):
    m, h1 = _case("deformed", 4, 7)
    P = oracle.Problem(m, h1)
    H = Handle(m, h1, flags=S.SEM_FLAG_SCHWARZ)
    b = W.random_global_rhs(m, 5)
    _, ref = H.solve(b, tol=TOL, mode=S.SEM_MODE_GMRES)
    x, st = H.solve(b, tol=TOL, mode=S.SEM_MODE_GMRES, precision=prec, precond_precision=pc)
    assert st["status"] == S.SEM_OK and st["relres"] <= TOL, st
    assert _oracle_relres(P, x, b) <= 1.05 * TOL
    assert abs(st["iterations"] - ref["iterations"]) <= max(3, ref["iterations"] // 10), (st, ref)


@pytest.mark.parametrize("restart", [1, 17, 40])
def test_gmres_restart_lengths_match_oracle(restart):
    """Restart 1 (one Arnoldi step per cycle), 17 and 40 (Gram-Schmidt dot
    products over more than one launch of 16)."""
    m, h1 = _case("deformed", 3, 5)
    P = oracle.Problem(m, h1)
    H = Handle(m, h1, flags=S.SEM_FLAG_SCHWARZ)
    b = W.random_global_rhs(m, 21)
    x, st = H.solve(b, tol=TOL, mode=S.SEM_MODE_GMRES, gmres_restart=restart, max_iter=3000)
    assert st["status"] == S.SEM_OK and st["relres"] <= TOL, st
    assert _oracle_relres(P, x, b) <= 1.05 * TOL
    _, info = oracle.fgmres(P, b, oracle.SchwarzPrecond(P, m, h1), restart=restart, tol=TOL, max_iter=3000)
    assert abs(st["iterations"] - info["iters"]) <= max(3, info["iters"] // 10), (st, info)


def test_gmres_rejects_bad_precision_options():
    m, h1 = _case("deformed", 2, 3)
    H = Handle(m, h1, flags=S.SEM_FLAG_SCHWARZ)
    b = W.random_global_rhs(m, 1)
    for bad in ({"precision": S.SEM_TC_SPLIT}, {"precond_precision": 7}, {"gmres_restart": 201},
                {"precision": S.SEM_FP32, "inner_tol": 1.0}, {"gmres_orth": 4}, {"gmres_orth": 0}):
        with pytest.raises(S.SemError) as ei:
            H.solve(b, tol=TOL, mode=S.SEM_MODE_GMRES, **bad)
        assert ei.value.status == S.SEM_EINVAL, bad


@pytest.mark.parametrize("prec", [S.SEM_FP64, S.SEM_FP32])
def test_gmres_gram_schmidt_forms(prec):
    """gmres_orth = 1 (Gram-Schmidt once) and 3 (twice within each step)
    reach the true 1e-10 within a few iterations of the default (twice, the
    second pass lagged one step); so does the coarse CG as one cooperative
    launch (opts.persistent)."""
    m, h1 = _case("deformed", 4, 7)
    P = oracle.Problem(m, h1)
    H = Handle(m, h1, flags=S.SEM_FLAG_SCHWARZ)
    b = W.random_global_rhs(m, 9)
    _, ref = H.solve(b, tol=TOL, mode=S.SEM_MODE_GMRES, precision=prec)
    for extra in ({"gmres_orth": 1}, {"gmres_orth": 3}, {"persistent": 1}):
        x, st = H.solve(b, tol=TOL, mode=S.SEM_MODE_GMRES, precision=prec, **extra)
        assert st["status"] == S.SEM_OK and st["relres"] <= TOL, (extra, st)
        assert _oracle_relres(P, x, b) <= 1.05 * TOL, extra
        assert abs(st["iterations"] - ref["iterations"]) <= max(3, ref["iterations"] // 10), (extra, st, ref)


def test_schwarz_two_stream_path_is_bit_identical():
    """After a GMRES solve the handle applies the preconditioner with the coarse
    CG on a second stream (restriction, local solves and coarse solve split over
    two streams); the arithmetic is the one-stream path's, so the output is the
    same to the bit, in FP64 and FP32."""
    import torch
    m, h1 = _case("deformed", 3, 7)
    P = oracle.Problem(m, h1)
    r = P.gs(W.random_local_field(m, 11), mask=True)
    outs = {}
    for warm in (False, True):
        H = Handle(m, h1, flags=S.SEM_FLAG_SCHWARZ)
        if warm:
            H.solve(W.random_global_rhs(m, 2), tol=TOL, mode=S.SEM_MODE_GMRES, precision=S.SEM_FP32)
        z64 = torch.empty(m.n_local, dtype=torch.float64, device="cuda")
        z32 = torch.empty(m.n_local, dtype=torch.float32, device="cuda")
        S.sem_schwarz_apply(H.h, dev(r, torch.float64), z64)
        S.sem_schwarz_apply32(H.h, dev(r, torch.float32), z32)
        torch.cuda.synchronize()
        outs[warm] = (host(z64), host(z32))
    assert np.array_equal(outs[False][0], outs[True][0])
    assert np.array_equal(outs[False][1], outs[True][1])


@pytest.mark.parametrize("prec", [S.SEM_FP64, S.SEM_FP32])
def test_gmres_edge_cases(prec):
    """Zero right-hand side: SEM_OK at once, x = 0.  Right-hand sides scaled by
    1e-30 and 1e30: the same 1e-10 by the oracle's operator (the Krylov
    vectors are normalised, so the FP32 cycles see unit-sized data).  A NaN in
    b: SEM_EBREAKDOWN.  max_iter too small: SEM_ENOTCONV with the true
    residual above the tolerance."""
    m, h1 = _case("deformed", 3, 5)
    P = oracle.Problem(m, h1)
    H = Handle(m, h1, flags=S.SEM_FLAG_SCHWARZ)
    zero = np.zeros(m.n_local)
    x, st = H.solve(zero, tol=TOL, mode=S.SEM_MODE_GMRES, precision=prec)
    assert st["status"] == S.SEM_OK and st["iterations"] == 0 and not np.any(x), st
    b = W.random_global_rhs(m, 17)
    for scale in (1e-30, 1e30):
        x, st = H.solve(b * scale, tol=TOL, mode=S.SEM_MODE_GMRES, precision=prec)
        assert st["status"] == S.SEM_OK and st["relres"] <= TOL, (scale, st)
        assert _oracle_relres(P, x, b * scale) <= 1.05 * TOL, scale
    bad = b.copy()
    bad[np.flatnonzero(m.mask)[4]] = np.nan
    x, st = H.solve(bad, tol=TOL, mode=S.SEM_MODE_GMRES, precision=prec)
    assert st["status"] == S.SEM_EBREAKDOWN, st
    x, st = H.solve(b, tol=TOL, mode=S.SEM_MODE_GMRES, precision=prec, max_iter=5)
    assert st["status"] == S.SEM_ENOTCONV and st["relres"] > TOL and st["iterations"] <= 5, st


def test_gmres_bounded_wait_expiry_reports_timeout():
    """Failure detection without a fault: with SEM_FLAG_TEST_STALL the
    bulk-staged operator kernels announce more bytes than they copy, their
    bounded waits expire (~50 ms), and the GMRES solve reports SEM_ETIMEOUT at
    its next check; the context stays usable."""
    m, h1 = _case("deformed", 3, 7)
    P = oracle.Problem(m, h1)
    b = W.random_global_rhs(m, 4)
    H = Handle(m, h1, flags=S.SEM_FLAG_SCHWARZ | S.SEM_FLAG_VARIANT(2) | S.SEM_FLAG_TEST_STALL)
    for prec in (S.SEM_FP64, S.SEM_FP32):
        with pytest.raises(S.SemError) as ei:
            H.solve(b, tol=TOL, mode=S.SEM_MODE_GMRES, precision=prec, gmres_restart=4, max_iter=8)
        assert ei.value.status == S.SEM_ETIMEOUT, prec
    H.close()
    H2 = Handle(m, h1, flags=S.SEM_FLAG_SCHWARZ)
    x, st = H2.solve(b, tol=TOL, mode=S.SEM_MODE_GMRES, precision=S.SEM_FP32)
    assert st["status"] == S.SEM_OK and _oracle_relres(P, x, b) <= 1.05 * TOL
