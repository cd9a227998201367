"""Pins of the oracle's Jacobi-PCG and FP64 iterative refinement (Sec. II-B)
to dense direct solves, finite termination and spectral convergence to a
manufactured solution."""
import numpy as np
import pytest

import oracle
import workloads as W
import dense_ref


def _dense_solution(m, h1, b):
    """Solve the masked assembled system densely: K_FF x_F = b_F with b given
    as an assembled local vector (all copies equal)."""
    K, Q, mask_g, _, _ = dense_ref.assembled(m, h1)
    _, first = np.unique(m.gid, return_index=True)
    bg = b[first]
    F = mask_g > 0
    xg = np.zeros(K.shape[0])
    xg[F] = np.linalg.solve(K[np.ix_(F, F)], bg[F])
    return Q @ xg, int(F.sum())


@pytest.mark.parametrize("dims,N,amp", [((2, 2, 2), 3, 0.05), ((2, 1, 3), 4, 0.1), ((1, 1, 1), 6, 0.1)])
def test_pcg_matches_dense_solve(dims, N, amp):
    m = W.box_mesh(*dims, N, amp=amp)
    h1 = W.h1_wavy(m)
    P = oracle.Problem(m, h1)
    b = W.random_global_rhs(m, 7)
    x, info = P.pcg(b, tol=1e-13)
    assert info["status"] == 0
    xd, nfree = _dense_solution(m, h1, b)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    # CG terminates in at most n_free steps (exact arithmetic); with rounding allow 2x
    assert info["iters"] <= 2 * nfree
    assert info["relres"] <= 1e-12


def test_pcg_true_residual_and_history():
    m = W.box_mesh(3, 3, 3, 5, amp=0.05)
    h1 = W.h1_wavy(m)
    P = oracle.Problem(m, h1)
    b = W.random_global_rhs(m, 3)
    x, info = P.pcg(b, tol=1e-10, hist=True)
    assert info["status"] == 0
    assert info["relres"] <= 2e-10
    assert info["hist"][-1] <= 1e-10 and np.all(info["hist"][:-1] > 1e-10)
    r = b - P.ax(x)
    assert np.sqrt(P.dot(r, r) / P.dot(b, b)) == pytest.approx(info["relres"], rel=1e-6)


def test_pcg_zero_rhs_and_warm_start():
    m = W.box_mesh(2, 2, 2, 3)
    P = oracle.Problem(m)
    x, info = P.pcg(np.zeros(m.n_local))
    assert info["status"] == 0 and info["iters"] == 0 and not np.any(x)
    b = W.random_global_rhs(m, 1)
    xs, _ = P.pcg(b, tol=1e-13)
    x2, info2 = P.pcg(b, x0=xs, tol=1e-10)
    assert info2["iters"] <= 1


def test_pcg_breakdown_on_neumann():
    """Without Dirichlet nodes A is singular: a right-hand side with a
    constant component leaves CG without convergence, never with a false one."""
    m = W.box_mesh(2, 2, 2, 2)
    m.mask[:] = 1
    P = oracle.Problem(m)
    b = P.mass(np.ones(m.n_local), assemble=True)
    x, info = P.pcg(b, tol=1e-10, max_iter=200)
    assert info["status"] in (1, 2)


def test_spectral_convergence_in_N():
    """Manufactured solution sin(pi x) sin(pi y) sin(pi z) on 2^3 elements:
    the max nodal error falls geometrically with N."""
    errs = []
    for N in range(3, 11):
        m, f = W.cube_sines(2, N)
        P = oracle.Problem(m)
        b = P.mass(f, assemble=True)
        x, info = P.pcg(b, tol=1e-13)
        errs.append(np.max(np.abs(x - W.exact_sines(m))))
    errs = np.array(errs)
    # overall: at least 6 orders of magnitude from N=3 to N=10
    assert errs[-1] < 1e-6 * errs[0]
    # each even step of 2 in N gains at least a factor 10
    assert np.all(errs[2::2] < 0.1 * errs[0:-2:2])


def test_h_convergence_at_fixed_N():
    """At N = 3, halving h reduces the max nodal error by at least 2^(N+1)/2."""
    N = 3
    errs = []
    for n in (2, 4, 8):
        m, f = W.cube_sines(n, N)
        P = oracle.Problem(m)
        x, _ = P.pcg(P.mass(f, assemble=True), tol=1e-13)
        errs.append(np.max(np.abs(x - W.exact_sines(m))))
    for a, b in zip(errs[:-1], errs[1:]):
        assert a / b > 2 ** (N + 1) / 2


def test_cube_sines_workload():
    """The 4^3-element, N = 7 cube with the manufactured forcing."""
    m, f = W.cube_sines(4, 7)
    P = oracle.Problem(m)
    x, info = P.pcg(P.mass(f, assemble=True), tol=1e-10)
    assert info["status"] == 0 and info["relres"] <= 1e-10
    assert np.max(np.abs(x - W.exact_sines(m))) < 1e-7


@pytest.mark.parametrize("inner_tol", [1e-3, 1e-5])
def test_ir_reaches_fp64_solution(inner_tol):
    m = W.box_mesh(3, 3, 3, 5, amp=0.05)
    h1 = W.h1_wavy(m)
    P = oracle.Problem(m, h1)
    b = W.random_global_rhs(m, 9)
    x64, _ = P.pcg(b, tol=1e-13)
    x, info = P.ir(b, tol=1e-10, inner_tol=inner_tol)
    assert info["status"] == 0, info
    assert info["relres"] <= 1e-10
    h = info["outer_hist"]
    assert np.all(np.diff(h) < 0)
    assert np.linalg.norm(x - x64) <= 1e-7 * np.linalg.norm(x64)


@pytest.mark.parametrize("inner_tol", [1e-2, 1e-1])
def test_ir_carry_continues_one_cg(inner_tol):
    """Refinement with the inner direction carried across steps, rescaled by
    ||r_prev|| / ||r|| (CG with residual replacement): the inner iterations add
    up to about the FP64 PCG count (one continued Krylov space), while
    restarting at every step costs well over it.  A wrong rescaling (c^2 or
    1/c instead of c) gives 1.35x the FP64 count, or no convergence at all."""
    m, h1, b = W.deformed_cube(4, 7, seed=2)
    P = oracle.Problem(m, h1)
    _, i64 = P.pcg(b, tol=1e-10)
    xref, _ = P.pcg(b, tol=1e-13)
    _, ir = P.ir(b, tol=1e-10, inner_tol=inner_tol)
    xc, ic = P.ir(b, tol=1e-10, inner_tol=inner_tol, carry=True)
    assert ic["status"] == 0 and ic["relres"] <= 1e-10, ic
    assert ic["outer"] >= 3
    assert ic["inner"] <= 1.05 * i64["iters"], (ic["inner"], i64["iters"])
    assert ir["inner"] >= 1.2 * i64["iters"], (ir["inner"], i64["iters"])
    assert np.linalg.norm(xc - xref) <= 1e-7 * np.linalg.norm(xref)


def test_ir_kept_direction_with_capped_steps():
    """Kept direction with every refinement step stopped after at most 100
    inner iterations (a replacement at least every 100 iterations): on the
    periodic annulus, where letting the FP32 CG run to 1e-3 between
    replacements drifts too far, the capped form stays near the FP64 PCG
    count.  The stagnation test skips capped steps (their residual can grow)."""
    m, f = W.annulus_case(N=7, n_theta=16, n_r=8, n_z=6)
    P = oracle.Problem(m)
    b = P.mass(f, assemble=True)
    xref, i64 = P.pcg(b, tol=1e-10)
    _, iu = P.ir(b, tol=1e-10, inner_tol=1e-3, carry=True)
    xc, ic = P.ir(b, tol=1e-10, inner_tol=1e-3, carry=True, max_inner=100, max_outer=60)
    assert ic["status"] == 0 and ic["relres"] <= 1e-10, ic
    assert ic["inner"] <= 1.25 * i64["iters"], (ic["inner"], i64["iters"])
    assert ic["inner"] <= 0.85 * iu["inner"], (ic["inner"], iu["inner"])
    assert np.linalg.norm(xc - xref) <= 1e-7 * np.linalg.norm(xref)


def test_ir_matches_dense_solution_small():
    m = W.box_mesh(2, 2, 2, 3, amp=0.05)
    P = oracle.Problem(m)
    b = W.random_global_rhs(m, 4)
    x, info = P.ir(b, tol=1e-11, inner_tol=1e-4)
    xd, _ = _dense_solution(m, None, b)
    assert info["status"] == 0
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
