"""GPU parity of the batched solve (sem_setup_batch + sem_cg_solve_batch)
against the FP64 oracle: every member of a batch of meshes with different
sizes and orders reaches a TRUE relative residual of 1e-10 (checked with the
oracle's own operator), agrees with the single-mesh solve, and batches are
bit-reproducible."""
import numpy as np
import pytest

import oracle
import workloads as W
import paper_2207_07098_gb300 as S
from gpu_helpers import rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _members(seed=0, count=9):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        nx, ny, nz = (int(v) for v in rng.integers(1, 5, size=3))
        N = int(rng.choice([1, 2, 3, 4, 5, 7, 9]))
        amp = float(rng.uniform(0.0, 0.08))
        m = W.box_mesh(nx, ny, nz, N, amp=amp)
        h1 = W.h1_wavy(m) if q % 2 else None
        b = W.random_global_rhs(m, 100 + q)
        out.append((m, h1, b))
    return out


def _setup(members):
    return S.sem_setup_batch([(m.E, m.lx, m.coords, m.gid, m.mask, h1) for m, h1, _ in members])


def _solve(h, members, **opts):
    import torch
    b = torch.from_numpy(np.concatenate([bb for _, _, bb in members])).cuda()
    x = torch.zeros_like(b)
    st = S.sem_cg_solve_batch(h, x, b, len(members), {"tol": TOL, **opts})
    torch.cuda.synchronize()
    xs = x.cpu().numpy()
    off = np.cumsum([0] + [m.n_local for m, _, _ in members])
    return [xs[off[q]:off[q + 1]] for q in range(len(members))], st


def _oracle_relres(P, x, b):
    r = b - P.ax(x)
    bb = P.dot(b, b)
    return np.sqrt(P.dot(r, r) / bb) if bb > 0 else 0.0


@pytest.mark.parametrize("mode", [S.SEM_MODE_FP64, S.SEM_MODE_MIXED_IR])
def test_batch_members_converge(mode):
    members = _members(1)
    h = _setup(members)
    try:
        info = S.sem_get_info(h)
        assert info["nsolve"] == len(members)
        off = S.sem_get_offsets(h, len(members))
        assert off[-1] == sum(m.n_local for m, _, _ in members)
        xs, st = _solve(h, members, mode=mode)
        for q, ((m, h1, b), x, s) in enumerate(zip(members, xs, st)):
            assert s["status"] == S.SEM_OK, (q, s)
            assert s["relres"] <= TOL, (q, s)
            P = oracle.Problem(m, h1)
            assert _oracle_relres(P, x, b) <= 1.05 * TOL, q
            xo, _ = P.pcg(b, tol=1e-12)
            if np.linalg.norm(xo) > 0:
                assert rel_err(x, xo)[0] <= 1e-7, q
    finally:
        S.sem_destroy(h)


@pytest.mark.parametrize("carry", [0, 1])
def test_batch_mixed_restart_and_carried_direction(carry):
    """Batched refinement with every member restarting its inner CG (ir_carry
    = 0, the tight inner tolerance it is made for) and with every member
    keeping its direction (ir_carry = 1): all members reach 1e-10 by the
    oracle's residual; the carried form takes no more inner iterations in all
    than restarting at the same inner tolerance."""
    members = _members(3)
    h = _setup(members)
    try:
        xs, st = _solve(h, members, mode=S.SEM_MODE_MIXED_IR, inner_tol=1e-2 if carry else 1e-5, ir_carry=carry)
        for q, ((m, h1, b), x, s) in enumerate(zip(members, xs, st)):
            assert s["status"] == S.SEM_OK and s["relres"] <= TOL, (q, s)
            P = oracle.Problem(m, h1)
            assert _oracle_relres(P, x, b) <= 1.05 * TOL, q
        if carry:
            _, st_r = _solve(h, members, mode=S.SEM_MODE_MIXED_IR, inner_tol=1e-2, ir_carry=0)
            assert sum(s["iterations"] for s in st) <= sum(s["iterations"] for s in st_r)
    finally:
        S.sem_destroy(h)


def test_batch_matches_single_and_is_reproducible():
    import torch
    members = _members(2, count=5)
    h = _setup(members)
    try:
        x1, s1 = _solve(h, members)
        x2, s2 = _solve(h, members)
        for a, b in zip(x1, x2):
            assert np.array_equal(a, b)
        x3, s3 = _solve(h, members, use_graph=0, graph_chunk=5)
        for a, b in zip(x1, x3):
            assert np.array_equal(a, b)
        for q, (m, h1, b) in enumerate(members):
            hs = S.sem_setup(m.E, m.lx, m.coords, m.gid, m.mask, h1)
            try:
                xd = torch.zeros(m.n_local, dtype=torch.float64, device="cuda")
                st = S.sem_cg_solve(hs, xd, torch.from_numpy(b).cuda(), {"tol": TOL})
                assert abs(st["iterations"] - s1[q]["iterations"]) <= 2
                assert rel_err(x1[q], xd.cpu().numpy())[0] <= 1e-7
            finally:
                S.sem_destroy(hs)
    finally:
        S.sem_destroy(h)


def test_batch_statuses_are_per_member():
    members = _members(3, count=4)
    m, h1, _ = members[1]
    members[1] = (m, h1, np.zeros(m.n_local))  # zero right-hand side
    h = _setup(members)
    try:
        xs, st = _solve(h, members)
        assert st[1]["status"] == S.SEM_OK and st[1]["iterations"] == 0 and not np.any(xs[1])
        xs, st = _solve(h, members, max_iter=2, tol=1e-14)
        assert all(s["status"] in (S.SEM_ENOTCONV, S.SEM_OK) for s in st)
        assert any(s["status"] == S.SEM_ENOTCONV for s in st)
    finally:
        S.sem_destroy(h)


def test_batch_256_member_workload_sampled():
    """The 256-member batch (nx, ny, nz ~ U{2..16}, N ~ U{5,7,9}): the FP64
    solve (native and FP32-pair operator) and the mixed refinement converge
    for every member; the oracle checks the true residual of a sample of
    members."""
    import torch
    params = W.batch_params()
    members = []
    for p in params:
        m, b = W.batch_member_case(p)
        members.append((m, None, b))
    h = _setup(members)
    try:
        rng = np.random.default_rng(7)
        sample = sorted(set(rng.choice(len(members), size=6, replace=False).tolist()))
        small = sorted(range(len(members)), key=lambda q: members[q][0].n_local)[:2]
        for mode, prec in ((S.SEM_MODE_FP64, S.SEM_FP64), (S.SEM_MODE_FP64, S.SEM_FP64_PAIR),
                           (S.SEM_MODE_MIXED_IR, S.SEM_FP64)):
            xs, st = _solve(h, members, mode=mode, precision=prec)
            assert all(s["status"] == S.SEM_OK and s["relres"] <= TOL for s in st)
            for q in sorted(set(sample) | set(small)):
                m, h1, b = members[q]
                if m.n_local > 3_000_000:
                    continue
                P = oracle.Problem(m, h1)
                assert _oracle_relres(P, xs[q], b) <= 1.05 * TOL, (mode, prec, q)
    finally:
        S.sem_destroy(h)
        torch.cuda.empty_cache()


def _even_members(seed, count, orders=(3, 5, 7, 9, 11)):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        nx, ny, nz = (int(v) for v in rng.integers(1, 5, size=3))
        N = int(rng.choice(np.asarray(orders)))
        m = W.box_mesh(nx, ny, nz, N, amp=float(rng.uniform(0.0, 0.08)))
        h1 = W.h1_wavy(m) if q % 2 else None
        out.append((m, h1, W.random_global_rhs(m, 300 + q)))
    return out


@pytest.mark.parametrize("flags", [S.SEM_FLAG_VARIANT(1), S.SEM_FLAG_VARIANT(2), S.SEM_FLAG_VARIANT(4)])
def test_batch_even_orders_bulk_operator(flags):
    """Every order even (lx 4..12) and a bulk variant pinned: the FP32 inner
    solves run the bulk-staged batched operator where the variant fits; the
    mixed solve reaches 1e-10 by the oracle's residual and agrees with the
    slab operator (variant 0) to solver accuracy."""
    members = _even_members(11, 7)
    h = _setup_flags(members, flags)
    h0 = _setup_flags(members, S.SEM_FLAG_VARIANT(0))
    try:
        xs, st = _solve(h, members, mode=S.SEM_MODE_MIXED_IR)
        x0, s0 = _solve(h0, members, mode=S.SEM_MODE_MIXED_IR)
        xr, _ = _solve(h, members, mode=S.SEM_MODE_MIXED_IR)
        for q, (m, h1, b) in enumerate(members):
            assert st[q]["status"] == S.SEM_OK and st[q]["relres"] <= TOL, (q, st[q])
            assert np.array_equal(xs[q], xr[q]), q
            P = oracle.Problem(m, h1)
            assert _oracle_relres(P, xs[q], b) <= 1.05 * TOL, q
            assert rel_err(xs[q], x0[q])[0] <= 1e-7, q
    finally:
        S.sem_destroy(h)
        S.sem_destroy(h0)


def test_batch_misaligned_even_order_falls_back():
    """A solve of odd lx (lx = 3, 27 nodes per element) ahead of even-order
    solves shifts their first local index off a 16-byte boundary; with a bulk
    variant pinned, those orders still take the slab operator and the mixed
    solve converges."""
    m3 = W.box_mesh(1, 1, 3, 2, amp=0.05)
    members = [(m3, None, W.random_global_rhs(m3, 299))] + _even_members(13, 4)
    h = _setup_flags(members, S.SEM_FLAG_VARIANT(2))
    try:
        off = S.sem_get_offsets(h, len(members))
        assert any(o % 4 for o in off[1:-1])
        xs, st = _solve(h, members, mode=S.SEM_MODE_MIXED_IR)
        for q, (m, h1, b) in enumerate(members):
            assert st[q]["status"] == S.SEM_OK, (q, st[q])
            P = oracle.Problem(m, h1)
            assert _oracle_relres(P, xs[q], b) <= 1.05 * TOL, q
    finally:
        S.sem_destroy(h)


def _setup_flags(members, flags):
    return S.sem_setup_batch([(m.E, m.lx, m.coords, m.gid, m.mask, h1) for m, h1, _ in members], flags)



def test_batch_multi_order_launch_matches_per_order():
    """One operator launch over the element groups of every order (variant 7,
    taken without autotuning where every order is at most lx = 10) against
    one slab launch per order (variant 0 pinned): the same arithmetic in the
    same order, so every member's solution is bit-identical, in FP64 and in
    the mixed refinement; the stats report the launches of one iteration."""
    members = _members(5, count=10)
    orders = {m.lx for m, _, _ in members}
    assert max(orders) <= 10 and len(orders) >= 3
    hm = _setup(members)
    hp = _setup_flags(members, S.SEM_FLAG_VARIANT(0))
    try:
        for mode in (S.SEM_MODE_FP64, S.SEM_MODE_MIXED_IR):
            xm, sm = _solve(hm, members, mode=mode, autotune=0)
            xp, sp = _solve(hp, members, mode=mode)
            assert all(s["ax_variant"] == 7 and s["launches_per_iteration"] == 3 for s in sm), sm[0]
            assert all(s["launches_per_iteration"] == len(orders) + 2 for s in sp), sp[0]
            for q, (m, h1, b) in enumerate(members):
                assert sm[q]["status"] == S.SEM_OK and sm[q]["relres"] <= TOL, (mode, q, sm[q])
                assert np.array_equal(xm[q], xp[q]), (mode, q)
                assert sm[q]["iterations"] == sp[q]["iterations"], (mode, q)
            P = oracle.Problem(*members[3][:2])
            assert _oracle_relres(P, xm[3], members[3][2]) <= 1.05 * TOL
    finally:
        S.sem_destroy(hm)
        S.sem_destroy(hp)


def test_batch_autotuned_configuration_is_reported():
    """With autotuning (the default) the batch times its operator
    configurations at the first solve and reports the one it keeps: the
    multi-order launch (variant 7, 3 launches per iteration) or one launch
    per order with a slab or bulk-staged variant; either way every member
    converges by the oracle's residual."""
    members = _even_members(17, 6, orders=(5, 7, 9))
    h = _setup(members)
    try:
        xs, st = _solve(h, members, mode=S.SEM_MODE_MIXED_IR)
        for q, (m, h1, b) in enumerate(members):
            s = st[q]
            assert s["status"] == S.SEM_OK and s["relres"] <= TOL, (q, s)
            assert (s["ax_variant"] == 7 and s["launches_per_iteration"] == 3) or \
                (0 <= s["ax_variant"] <= 4 and s["launches_per_iteration"] == 5), s
            P = oracle.Problem(m, h1)
            assert _oracle_relres(P, xs[q], b) <= 1.05 * TOL, q
    finally:
        S.sem_destroy(h)
