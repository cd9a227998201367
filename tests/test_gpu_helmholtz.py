"""GPU parity of the Helmholtz operator of the velocity solve (Sec. II-A:
the implicit viscous term gives A = QQ^T (h1 K + h2 B); Sec. II-B solves it
with P-CG and a Jacobi-type preconditioner) against the FP64 oracle, through
the C ABI: operator applications in FP64 (1e-12) and FP32, the Jacobi
diagonal with the h2 B term, FP64 and mixed solves (true residual 1e-10 by
the oracle's operator) with and without Dirichlet nodes, batches, and the
return to the Poisson operator."""
import numpy as np
import pytest

import oracle
import workloads as W
import paper_2207_07098_gb300 as S
from gpu_helpers import Handle, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _h2(m, scale=1.0):
    x, y, z = m.xyz()
    return scale * (2.0 + np.cos(3.0 * x) * np.sin(2.0 * y) + z)


def _oracle_relres(P, x, b):
    r = b - P.ax(x)
    return np.sqrt(P.dot(r, r) / P.dot(b, b))


CASES = [("deformed", (3, 2, 2), 3), ("jitter", (3, 3, 2), 5), ("deformed", (4, 3, 3), 7), ("deformed", (2, 2, 2), 9)]


def _case(kind, dims, N):
    if kind == "deformed":
        m = W.box_mesh(*dims, N, amp=0.05)
    else:
        m = W.box_mesh(*dims, N, amp=0.1, jitter=0.25 / (N * N), seed=1)
    return m, W.h1_wavy(m)


@pytest.mark.parametrize("variant", [0, 2])
@pytest.mark.parametrize("kind,dims,N", CASES)
def test_helmholtz_operator_and_jacobi(kind, dims, N, variant):
    m, h1 = _case(kind, dims, N)
    h2 = _h2(m)
    P = oracle.Problem(m, h1)
    P.set_h2(h2)
    H = Handle(m, h1, flags=S.SEM_FLAG_VARIANT(variant))
    S.sem_set_helmholtz(H.h, h2)
    u = W.random_local_field(m, 31)
    for prec in (S.SEM_FP64, S.SEM_FP64_NATIVE):
        e2, einf = rel_err(H.ax(u, prec, assemble=0), P.ax_local(u))
        assert e2 <= 1e-12 and einf <= 1e-12, (prec, e2, einf)
    # the pair kernels carry no mass term: SEM_FP64_PAIR takes the native operator
    assert np.array_equal(H.ax(u, S.SEM_FP64_PAIR, assemble=0), H.ax(u, S.SEM_FP64, assemble=0))
    uc = W.random_local_field(m, 32, continuous=True)
    e2, einf = rel_err(H.ax(uc, S.SEM_FP64, assemble=1), P.ax(uc))
    assert e2 <= 1e-12 and einf <= 1e-12, (e2, einf)
    e2, _ = rel_err(H.ax(uc, S.SEM_FP32, assemble=1), P.ax(uc))
    assert e2 <= 5e-6 * N, e2
    np.testing.assert_allclose(H.jacobi(), P.minv(), rtol=1e-12)


@pytest.mark.parametrize("neumann", [False, True])
def test_helmholtz_solves(neumann):
    """FP64 and mixed Jacobi-PCG on the Helmholtz operator reach 1e-10 by the
    oracle's residual and agree with the oracle's solution; with h2 > 0 the
    problem is SPD without any Dirichlet node."""
    m, h1 = _case("deformed", (4, 3, 3), 7)
    if neumann:
        m.mask[:] = 1
    h2 = _h2(m, 30.0)
    P = oracle.Problem(m, h1)
    P.set_h2(h2)
    H = Handle(m, h1)
    S.sem_set_helmholtz(H.h, h2)
    b = P.mass(W.forcing_sines(m) + 1.0, assemble=True)
    xo, info = P.pcg(b, tol=1e-12)
    for mode, prec, pers in ((S.SEM_MODE_FP64, S.SEM_FP64, 0), (S.SEM_MODE_FP64, S.SEM_FP64_PAIR, 0),
                             (S.SEM_MODE_MIXED_IR, S.SEM_FP64, 0), (S.SEM_MODE_MIXED_IR, S.SEM_FP64, 1)):
        x, st = H.solve(b, tol=TOL, mode=mode, precision=prec, persistent=pers)
        assert st["status"] == S.SEM_OK and st["relres"] <= TOL, (mode, prec, st)
        assert _oracle_relres(P, x, b) <= 1.05 * TOL, (mode, prec)
        assert rel_err(x, xo)[0] <= 1e-8, (mode, prec)
        if mode == S.SEM_MODE_FP64:
            _, i64 = P.pcg(b, tol=TOL)
            assert abs(st["iterations"] - i64["iters"]) <= max(2, i64["iters"] // 50), (st, i64)


def test_helmholtz_batch_and_return_to_poisson():
    """A batch handle with one concatenated h2 for all members: every member's
    solve matches its own oracle Helmholtz problem; sem_set_helmholtz(NULL)
    restores the Poisson operator and preconditioner."""
    import torch
    members = []
    for q, (dims, N) in enumerate((((2, 2, 1), 5), ((3, 2, 2), 7), ((1, 2, 2), 9))):
        m = W.box_mesh(*dims, N, amp=0.04)
        members.append((m, W.random_global_rhs(m, 40 + q)))
    h = S.sem_setup_batch([(m.E, m.lx, m.coords, m.gid, m.mask, None) for m, _ in members])
    try:
        h2s = [_h2(m, 10.0) for m, _ in members]
        S.sem_set_helmholtz(h, np.concatenate(h2s))
        b = torch.from_numpy(np.concatenate([bb for _, bb in members])).cuda()
        for mode in (S.SEM_MODE_FP64, S.SEM_MODE_MIXED_IR):
            x = torch.zeros_like(b)
            sts = S.sem_cg_solve_batch(h, x, b, len(members), {"tol": TOL, "mode": mode})
            xs = x.cpu().numpy()
            off = np.cumsum([0] + [m.n_local for m, _ in members])
            for q, ((m, bb), h2) in enumerate(zip(members, h2s)):
                assert sts[q]["status"] == S.SEM_OK, (mode, q, sts[q])
                P = oracle.Problem(m)
                P.set_h2(h2)
                assert _oracle_relres(P, xs[off[q]:off[q + 1]], bb) <= 1.05 * TOL, (mode, q)
        S.sem_set_helmholtz(h, None)
        x = torch.zeros_like(b)
        sts = S.sem_cg_solve_batch(h, x, b, len(members), {"tol": TOL})
        xs = x.cpu().numpy()
        for q, (m, bb) in enumerate(members):
            P = oracle.Problem(m)
            assert _oracle_relres(P, xs[off[q]:off[q + 1]], bb) <= 1.05 * TOL, q
    finally:
        S.sem_destroy(h)


def test_helmholtz_rejects_bad_coefficients():
    m, h1 = _case("deformed", (2, 2, 1), 3)
    H = Handle(m, h1)
    bad = _h2(m)
    bad[5] = -1.0
    with pytest.raises(S.SemError) as ei:
        S.sem_set_helmholtz(H.h, bad)
    assert ei.value.status == S.SEM_EINVAL
    bad[5] = np.nan
    with pytest.raises(S.SemError) as ei:
        S.sem_set_helmholtz(H.h, bad)
    assert ei.value.status == S.SEM_EINVAL
