"""GPU parity of the Poisson solves (through the C ABI) against the FP64 oracle:
FP64 Jacobi-PCG and mixed-precision refinement reach a TRUE relative residual
of 1e-10, checked independently by the oracle's own operator; iterates agree
with the oracle's solution; solves are bit-reproducible; edge cases return the
documented statuses."""
import numpy as np
import pytest

import oracle
import workloads as W
import paper_2207_07098_gb300 as S
from gpu_helpers import Handle, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _oracle_relres(P, x, b):
    r = b - P.ax(x)
    return np.sqrt(P.dot(r, r) / P.dot(b, b))


def _cube_case():
    m, f = W.cube_sines(4, 7)
    P = oracle.Problem(m)
    return m, None, P, P.mass(f, assemble=True)


def _deformed_case(n=6, N=7):
    m, h1, b = W.deformed_cube(n, N, seed=2)
    return m, h1, oracle.Problem(m, h1), b


@pytest.mark.parametrize("case", ["cube", "deformed"])
@pytest.mark.parametrize("precision", [S.SEM_FP64, S.SEM_FP64_NATIVE, S.SEM_FP64_PAIR])
def test_fp64_pcg(case, precision):
    m, h1, P, b = _cube_case() if case == "cube" else _deformed_case()
    H = Handle(m, h1)
    x, st = H.solve(b, mode=S.SEM_MODE_FP64, precision=precision, tol=TOL)
    assert st["status"] == S.SEM_OK, st
    assert st["relres"] <= TOL
    assert _oracle_relres(P, x, b) <= 1.05 * TOL
    xo, info = P.pcg(b, tol=TOL)
    # same method, same preconditioner: iteration counts within rounding effects
    assert abs(st["iterations"] - info["iters"]) <= max(2, info["iters"] // 50), (st, info)
    e2, _ = rel_err(x, xo)
    assert e2 <= 1e-7, e2
    if case == "cube":
        assert np.max(np.abs(x - W.exact_sines(m))) < 1e-7


@pytest.mark.parametrize("case", ["cube", "deformed"])
@pytest.mark.parametrize("inner_tol", [1e-4, 1e-6])
def test_mixed_ir(case, inner_tol):
    m, h1, P, b = _cube_case() if case == "cube" else _deformed_case()
    H = Handle(m, h1)
    x, st = H.solve(b, mode=S.SEM_MODE_MIXED_IR, inner_tol=inner_tol, tol=TOL, ir_carry=0)
    assert st["status"] == S.SEM_OK, st
    assert st["relres"] <= TOL and st["outer_iterations"] >= 1
    assert _oracle_relres(P, x, b) <= 1.05 * TOL
    xo, _ = P.pcg(b, tol=1e-12)
    e2, _ = rel_err(x, xo)
    assert e2 <= 1e-7, e2
    x64, _ = H.solve(b, mode=S.SEM_MODE_FP64, tol=TOL)
    assert rel_err(x, x64)[0] <= 1e-7


@pytest.mark.parametrize("inner_tol", [1e-2, 1e-1])
def test_mixed_ir_carried_direction(inner_tol):
    """ir_carry: the inner FP32 CG keeps its direction across refinement steps
    (residual replacement).  Same true residual and solution as the restarted
    refinement; the inner iterations add up to about the FP64 PCG count, as
    in the oracle's refinement with the same option."""
    m, h1, P, b = _deformed_case()
    H = Handle(m, h1)
    x, st = H.solve(b, mode=S.SEM_MODE_MIXED_IR, inner_tol=inner_tol, tol=TOL, ir_carry=1)
    assert st["status"] == S.SEM_OK, st
    assert st["relres"] <= TOL and st["outer_iterations"] >= 3, st
    assert _oracle_relres(P, x, b) <= 1.05 * TOL
    xo, _ = P.pcg(b, tol=1e-12)
    assert rel_err(x, xo)[0] <= 1e-7
    _, st64 = H.solve(b, mode=S.SEM_MODE_FP64, tol=TOL)
    _, ic = P.ir(b, tol=TOL, inner_tol=inner_tol, carry=True)
    assert 0.9 * st64["iterations"] <= st["iterations"] <= 1.05 * st64["iterations"] + 5, (st, st64)
    assert abs(st["iterations"] - ic["inner"]) <= 0.05 * ic["inner"] + 5, (st, ic)
    _, st_r = H.solve(b, mode=S.SEM_MODE_MIXED_IR, inner_tol=inner_tol, tol=TOL, ir_carry=0)
    assert st_r["iterations"] > st["iterations"], (st_r, st)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 9])
def test_solves_with_each_operator_variant(variant):
    """A pinned variant 0..4 serves the FP64 and FP32 operators, 5 or 6 the
    FP32-pair one (SEM_FP64_PAIR), 9 the FP64 one (native line transforms);
    every solve reaches 1e-10 by the oracle's residual with the variant it
    reports."""
    m, h1, P, b = _deformed_case(5, 7)
    H = Handle(m, h1, flags=S.SEM_FLAG_VARIANT(variant))
    runs = [(S.SEM_MODE_FP64, S.SEM_FP64), (S.SEM_MODE_MIXED_IR, S.SEM_FP64), (S.SEM_MODE_FP64, S.SEM_FP64_PAIR)]
    for mode, prec in runs:
        x, st = H.solve(b, mode=mode, precision=prec, tol=TOL)
        assert st["status"] == S.SEM_OK and st["relres"] <= TOL, st
        if prec == S.SEM_FP64_PAIR:
            # a pinned native variant leaves the pair class on its own default (6 for even lx)
            assert st["ax_variant"] == (variant if variant in (5, 6) else 6)
        elif mode == S.SEM_MODE_FP64:
            # a pinned bulk variant too large for FP64 shared memory falls back to 0
            assert st["ax_variant"] in ((variant, 0) if variant <= 4 else (9,) if variant == 9 else
                                        (0, 1, 2, 3, 4, 9))
        else:
            assert (st["ax_variant"] == variant) if variant <= 4 else (0 <= st["ax_variant"] <= 4)
        assert _oracle_relres(P, x, b) <= 1.05 * TOL


def test_autotuned_solve_reports_variant():
    m, h1, P, b = _deformed_case(6, 7)
    H = Handle(m, h1)
    x, st = H.solve(b, mode=S.SEM_MODE_MIXED_IR, tol=TOL)
    assert st["status"] == S.SEM_OK and 0 <= st["ax_variant"] <= 4
    assert _oracle_relres(P, x, b) <= 1.05 * TOL


def test_solve_bit_reproducible_and_graph_equivalent():
    m, h1, P, b = _deformed_case(4, 5)
    H = Handle(m, h1)
    x1, s1 = H.solve(b, tol=TOL)
    x2, s2 = H.solve(b, tol=TOL)
    assert np.array_equal(x1, x2) and s1["iterations"] == s2["iterations"]
    x3, s3 = H.solve(b, tol=TOL, use_graph=0, graph_chunk=7)
    assert np.array_equal(x1, x3) and s1["iterations"] == s3["iterations"]
    x4, s4 = H.solve(b, tol=TOL, mode=S.SEM_MODE_MIXED_IR)
    x5, _ = H.solve(b, tol=TOL, mode=S.SEM_MODE_MIXED_IR)
    assert np.array_equal(x4, x5)
    # the refinement steps after the first launch graphs sized by the previous
    # step's count (tail graphs of 4 iterations near the predicted end): the
    # same iterations as one launch at a time and as another chunk size
    x6, s6 = H.solve(b, tol=TOL, mode=S.SEM_MODE_MIXED_IR, use_graph=0)
    assert np.array_equal(x4, x6) and s4["iterations"] == s6["iterations"]
    x7, s7 = H.solve(b, tol=TOL, mode=S.SEM_MODE_MIXED_IR, graph_chunk=9)
    assert np.array_equal(x4, x7) and s4["iterations"] == s7["iterations"]
    assert s4["outer_iterations"] >= 2


def test_host_buffers_and_warm_start():
    m, h1, P, b = _deformed_case(3, 6)
    H = Handle(m, h1)
    xh, sh = H.solve(b, on_host=True, tol=TOL)
    xd, sd = H.solve(b, tol=TOL)
    assert np.array_equal(xh, xd)
    x2, s2 = H.solve(b, x0=xd, tol=TOL)
    assert s2["iterations"] <= 1 and s2["relres"] <= TOL


def test_edge_cases():
    m, h1, P, b = _deformed_case(2, 3)
    H = Handle(m, h1)
    # zero right-hand side: no iteration, x = 0
    x, st = H.solve(np.zeros(m.n_local), tol=TOL)
    assert st["status"] == S.SEM_OK and st["iterations"] == 0 and not np.any(x)
    # iteration budget exhausted
    x, st = H.solve(b, tol=1e-14, max_iter=3)
    assert st["status"] == S.SEM_ENOTCONV and st["iterations"] == 3
    # single element, lowest and highest orders
    for N in (1, 15):
        mm = W.box_mesh(1, 1, 1, N, amp=0.05)
        PP = oracle.Problem(mm)
        bb = W.random_global_rhs(mm, 1)
        HH = Handle(mm)
        xx, st = HH.solve(bb, tol=TOL)
        if N == 1:  # no free node: b = 0
            assert st["status"] == S.SEM_OK and st["iterations"] == 0
        else:
            assert st["status"] == S.SEM_OK and _oracle_relres(PP, xx, bb) <= 1.05 * TOL


def test_neumann_problem_does_not_fake_convergence():
    m = W.box_mesh(2, 2, 2, 3)
    m.mask[:] = 1
    P = oracle.Problem(m)
    b = P.mass(np.ones(m.n_local), assemble=True)
    H = Handle(m)
    x, st = H.solve(b, tol=TOL, max_iter=300)
    assert st["status"] in (S.SEM_ENOTCONV, S.SEM_EBREAKDOWN)
    x, st = H.solve(b, tol=TOL, max_iter=300, mode=S.SEM_MODE_MIXED_IR, max_outer=5)
    assert st["status"] in (S.SEM_ENOTCONV, S.SEM_EBREAKDOWN, S.SEM_ESTAGNATE)


def test_annulus_periodic_solve():
    m, f = W.annulus_case(N=5, n_theta=16, n_r=6, n_z=4)
    P = oracle.Problem(m)
    b = P.mass(f, assemble=True)
    H = Handle(m)
    for mode in (S.SEM_MODE_FP64, S.SEM_MODE_MIXED_IR):
        x, st = H.solve(b, tol=TOL, mode=mode)
        assert st["status"] == S.SEM_OK, st
        assert _oracle_relres(P, x, b) <= 1.05 * TOL


def test_full_size_solve_true_residual():
    """The 32^3-element deformed cube (16.8 M points), in the launch
    configuration bench.py times: the mixed-precision solve, the FP64 solve
    (native operator), the FP64 solve with the FP32-pair operator and vectors,
    and the pipelined FP64 solve (whose recurrences need their residual
    replacements at this size: ~1800 iterations) reach 1e-10, checked by the
    oracle's operator on the full mesh, and agree with each other to solver
    accuracy."""
    m, h1, b = W.deformed_cube(32, 7, seed=2)
    H = Handle(m, h1)
    P = oracle.Problem(m, h1)
    xs = {}
    for key, mode, prec, extra in (("mixed", S.SEM_MODE_MIXED_IR, S.SEM_FP64, {}),
                                   ("fp64", S.SEM_MODE_FP64, S.SEM_FP64, {}),
                                   ("pair", S.SEM_MODE_FP64, S.SEM_FP64_PAIR, {}),
                                   ("pipelined", S.SEM_MODE_FP64, S.SEM_FP64, {"pipelined": 1})):
        x, st = H.solve(b, tol=TOL, mode=mode, precision=prec, inner_tol=1e-2, ir_carry=1, **extra)
        assert st["status"] == S.SEM_OK and st["relres"] <= TOL, (key, st)
        assert _oracle_relres(P, x, b) <= 1.05 * TOL, key
        xs[key] = x
    for key in ("mixed", "pair", "pipelined"):
        assert rel_err(xs[key], xs["fp64"])[0] <= 1e-6, key


def test_bounded_wait_expiry_reports_timeout_and_context_survives():
    """Failure detection without a fault: with SEM_FLAG_TEST_STALL the staged
    operator kernels announce more bytes than they copy, so their bounded
    mbarrier waits expire (~50 ms), and the persistent CG kernel's first CTA
    skips a grid barrier, so the other CTAs' bounded barrier waits expire; the
    kernels record the failure and return, and the solve reports
    SEM_ETIMEOUT.  The context stays usable."""
    m, h1, P, b = _deformed_case(3, 7)
    H = Handle(m, h1, flags=S.SEM_FLAG_VARIANT(2) | S.SEM_FLAG_TEST_STALL)
    # graph loop (bulk-staged operator) and persistent launch (grid barrier)
    for mode in (S.SEM_MODE_MIXED_IR, S.SEM_MODE_FP64):
        for persistent in (0, 1):
            with pytest.raises(S.SemError) as ei:
                H.solve(b, mode=mode, tol=TOL, graph_chunk=2, persistent=persistent)
            assert ei.value.status == S.SEM_ETIMEOUT, (mode, persistent)
    H.close()
    H2 = Handle(m, h1, flags=S.SEM_FLAG_VARIANT(2))
    x, st = H2.solve(b, tol=TOL)
    assert st["status"] == S.SEM_OK and _oracle_relres(P, x, b) <= 1.05 * TOL


def test_non_finite_rhs_reports_breakdown():
    m, h1, P, b = _deformed_case(2, 5)
    H = Handle(m, h1)
    bad = b.copy()
    bad[np.flatnonzero(m.mask)[3]] = np.nan
    for mode in (S.SEM_MODE_FP64, S.SEM_MODE_MIXED_IR):
        x, st = H.solve(bad, mode=mode, tol=TOL, max_iter=50)
        assert st["status"] in (S.SEM_EBREAKDOWN, S.SEM_ENOTCONV, S.SEM_ESTAGNATE), st
    x, st = H.solve(b, tol=TOL)
    assert st["status"] == S.SEM_OK


@pytest.mark.parametrize("scale", [1e-30, 1e30])
def test_rhs_far_outside_unit_scale(scale):
    """A right-hand side scaled by 1e-30 or 1e30: the native FP64 solve, the
    FP32-pair solve (whose format reads |u| < 2^-75 as 0; the solver rescales
    x and b by a power of two) and the mixed refinement (which scales every
    inner right-hand side to unit norm) reach the same relative residual and
    the scaled solution, checked by the oracle."""
    m, h1, P, b = _deformed_case(3, 7)
    H = Handle(m, h1)
    x1, s1 = H.solve(b, tol=TOL)
    for mode, prec in ((S.SEM_MODE_FP64, S.SEM_FP64), (S.SEM_MODE_FP64, S.SEM_FP64_PAIR),
                       (S.SEM_MODE_MIXED_IR, S.SEM_FP64)):
        x, st = H.solve(b * scale, tol=TOL, mode=mode, precision=prec)
        assert st["status"] == S.SEM_OK and st["relres"] <= TOL, (mode, prec, st)
        assert _oracle_relres(P, x, b * scale) <= 1.05 * TOL, (mode, prec)
        assert rel_err(x / scale, x1)[0] <= 1e-7, (mode, prec)


def test_non_finite_initial_guess_reports_breakdown():
    """A NaN in x0 makes the true initial residual non-finite: every mode
    reports SEM_EBREAKDOWN with a NaN residual instead of hiding it (the pair
    format alone would read the NaN as 0)."""
    m, h1, P, b = _deformed_case(2, 5)
    H = Handle(m, h1)
    x0 = np.zeros(m.n_local)
    x0[np.flatnonzero(m.mask)[5]] = np.nan
    for mode, prec in ((S.SEM_MODE_FP64, S.SEM_FP64), (S.SEM_MODE_FP64, S.SEM_FP64_PAIR),
                       (S.SEM_MODE_MIXED_IR, S.SEM_FP64)):
        x, st = H.solve(b, x0=x0, tol=TOL, mode=mode, precision=prec)
        assert st["status"] == S.SEM_EBREAKDOWN and not np.isfinite(st["relres"]), (mode, prec, st)


def test_fp64_restarts_exhausted_report_not_converged():
    """A tolerance below what the 48-bit pair arithmetic can reach: the
    recursive residual keeps converging, the true residual does not, the
    residual-replacement restarts run out, and the solve reports
    SEM_ENOTCONV with the true residual above tol (never SEM_OK)."""
    m, h1, P, b = _deformed_case(3, 7)
    H = Handle(m, h1)
    x, st = H.solve(b, tol=1e-16, mode=S.SEM_MODE_FP64, precision=S.SEM_FP64_PAIR, max_iter=5000)
    assert st["status"] == S.SEM_ENOTCONV and st["relres"] > 1e-16, st
    assert _oracle_relres(P, x, b) <= 1e-12


def test_mixed_kept_direction_with_capped_steps_matches_oracle():
    """Kept direction with every refinement step capped at 100 inner
    iterations (ir_carry = 1, max_iter = 100) on a periodic annulus: capped
    steps are not judged for stagnation and keep their direction, as in the
    oracle's refinement with the same cap; the inner iteration count follows
    the oracle's and beats the uncapped kept direction."""
    m, f = W.annulus_case(N=7, n_theta=16, n_r=8, n_z=6)
    P = oracle.Problem(m)
    b = P.mass(f, assemble=True)
    H = Handle(m)
    x, st = H.solve(b, tol=TOL, mode=S.SEM_MODE_MIXED_IR, inner_tol=1e-3, ir_carry=1, max_iter=100,
                    max_outer=60)
    assert st["status"] == S.SEM_OK and st["relres"] <= TOL, st
    assert _oracle_relres(P, x, b) <= 1.05 * TOL
    _, ic = P.ir(b, tol=TOL, inner_tol=1e-3, carry=True, max_inner=100, max_outer=60)
    _, i64 = P.pcg(b, tol=TOL)
    assert abs(st["iterations"] - ic["inner"]) <= 0.15 * ic["inner"] + 10, (st, ic)
    assert st["iterations"] <= 1.3 * i64["iters"], (st, i64)
    _, su = H.solve(b, tol=TOL, mode=S.SEM_MODE_MIXED_IR, inner_tol=1e-3, ir_carry=1, max_outer=60)
    assert su["status"] == S.SEM_OK and st["iterations"] < su["iterations"], (st, su)


@pytest.mark.parametrize("case", ["cube", "annulus5"])
def test_persistent_single_launch_cg(case):
    """The whole CG as one cooperative launch with bounded grid barriers
    (opts.persistent = 1) against the graph loop (0): FP64 and mixed solves
    reach 1e-10 by the oracle's residual with the same iteration counts
    (within rounding effects), report no per-iteration launches, and are
    bit-reproducible."""
    if case == "cube":
        m, h1, P, b = _cube_case()
    else:
        m, f = W.annulus_case(N=4, n_theta=12, n_r=4, n_z=3)
        h1, P = None, oracle.Problem(m)
        b = P.mass(f, assemble=True)
    H = Handle(m, h1)
    for mode, prec in ((S.SEM_MODE_FP64, S.SEM_FP64), (S.SEM_MODE_FP64, S.SEM_FP64_NATIVE),
                       (S.SEM_MODE_MIXED_IR, S.SEM_FP64)):
        xg, sg = H.solve(b, tol=TOL, mode=mode, precision=prec, persistent=0)
        xp, sp = H.solve(b, tol=TOL, mode=mode, precision=prec, persistent=1)
        xq, sq = H.solve(b, tol=TOL, mode=mode, precision=prec, persistent=1)
        assert sp["status"] == S.SEM_OK and sp["relres"] <= TOL, (mode, sp)
        assert sp["launches_per_iteration"] == 0 and sg["launches_per_iteration"] == 3
        assert _oracle_relres(P, xp, b) <= 1.05 * TOL, mode
        assert abs(sp["iterations"] - sg["iterations"]) <= max(2, sg["iterations"] // 50), (mode, sp, sg)
        assert rel_err(xp, xg)[0] <= 1e-7, mode
        assert np.array_equal(xp, xq) and sp["iterations"] == sq["iterations"], mode


@pytest.mark.parametrize("case", ["cube", "deformed"])
def test_pipelined_pcg_matches_oracle(case):
    """Pipelined PCG (opts.pipelined = 1, Ghysels and Vanroose): the PCG
    iterates with one reduction phase per iteration; the iteration count
    follows the oracle's pipelined PCG and PCG, and the true residual reaches
    1e-10 by the oracle's operator (residual replacement restarts included)."""
    m, h1, P, b = _cube_case() if case == "cube" else _deformed_case()
    H = Handle(m, h1)
    x, st = H.solve(b, tol=TOL, mode=S.SEM_MODE_FP64, pipelined=1)
    assert st["status"] == S.SEM_OK and st["relres"] <= TOL, st
    assert _oracle_relres(P, x, b) <= 1.05 * TOL
    _, ip = oracle.pipelined_pcg(P, b, tol=TOL)
    _, i64 = P.pcg(b, tol=TOL)
    assert abs(st["iterations"] - ip["iters"]) <= max(3, ip["iters"] // 20), (st, ip)
    assert abs(st["iterations"] - i64["iters"]) <= max(3, i64["iters"] // 20), (st, i64)
    xg, _ = H.solve(b, tol=TOL, mode=S.SEM_MODE_FP64, pipelined=1, use_graph=0, graph_chunk=5)
    assert np.array_equal(x, xg)
