"""GPU parity of the split-precision tensor-core operator (SEM_TC_SPLIT:
BF16 slices of u, D and the weighted derivatives, six slice products per
contraction on mma.sync, FP32 accumulation) against the FP64 oracle, through
the C ABI: the FP32 accuracy class on lx = 8 meshes (deformed, jittered,
annulus), the fused CG kernel inside the mixed refinement (true residual
1e-10 by the oracle's operator), the Helmholtz mass term, and the fallback
to the FP32 kernels for other orders."""
import numpy as np
import pytest

import oracle
import workloads as W
import paper_2207_07098_gb300 as S
from gpu_helpers import Handle, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-10

CASES = [("deformed", (3, 2, 2)), ("jitter", (3, 3, 2)), ("deformed", (5, 4, 3)), ("annulus", (8, 3, 2))]


def _case(kind, dims):
    if kind == "deformed":
        m = W.box_mesh(*dims, 7, amp=0.05)
        return m, W.h1_wavy(m)
    if kind == "jitter":
        m = W.box_mesh(*dims, 7, amp=0.1, jitter=0.25 / 49, seed=3)
        return m, W.h1_wavy(m)
    m = W.annulus_mesh(n_theta=dims[0], n_r=dims[1], n_z=dims[2], N=7)
    return m, None


def _oracle_relres(P, x, b):
    r = b - P.ax(x)
    return np.sqrt(P.dot(r, r) / P.dot(b, b))


@pytest.mark.parametrize("kind,dims", CASES)
def test_tc_operator_fp32_class(kind, dims):
    """Local and assembled applications within the FP32 class: relative
    errors of the order of the CUDA-core FP32 kernel's (at most 3x, plus
    1e-7), both far below the inner solve's tolerance."""
    m, h1 = _case(kind, dims)
    P = oracle.Problem(m, h1)
    H = Handle(m, h1)
    u = W.random_local_field(m, 41)
    ref = P.ax_local(u)
    e_tc, _ = rel_err(H.ax(u.astype(np.float32), S.SEM_TC_SPLIT, assemble=0), ref)
    e_32, _ = rel_err(H.ax(u.astype(np.float32), S.SEM_FP32, assemble=0), ref)
    assert e_tc <= 3 * e_32 + 1e-7, (e_tc, e_32)
    uc = W.random_local_field(m, 42, continuous=True)
    e_tc, _ = rel_err(H.ax(uc.astype(np.float32), S.SEM_TC_SPLIT, assemble=1), P.ax(uc))
    assert e_tc <= 5e-6 * 7, e_tc
    us = W.forcing_sines(m) if kind != "annulus" else W.random_local_field(m, 43, continuous=True)
    e_tc, _ = rel_err(H.ax(us.astype(np.float32), S.SEM_TC_SPLIT, assemble=1), P.ax(us))
    e_32, _ = rel_err(H.ax(us.astype(np.float32), S.SEM_FP32, assemble=1), P.ax(us))
    assert e_tc <= 3 * e_32 + 1e-7, (e_tc, e_32)


def test_tc_mixed_refinement_and_helmholtz():
    m, h1, b = W.deformed_cube(6, 7, seed=2)
    P = oracle.Problem(m, h1)
    H = Handle(m, h1)
    x, st = H.solve(b, tol=TOL, mode=S.SEM_MODE_MIXED_IR, tc_split=1)
    assert st["status"] == S.SEM_OK and st["relres"] <= TOL and st["ax_variant"] == 8, st
    assert _oracle_relres(P, x, b) <= 1.05 * TOL
    _, s32 = H.solve(b, tol=TOL, mode=S.SEM_MODE_MIXED_IR, tc_split=0)
    assert abs(st["iterations"] - s32["iterations"]) <= 0.1 * s32["iterations"] + 5, (st, s32)
    # Helmholtz mass term in the tensor-core kernel
    x_, y_, z_ = m.xyz()
    h2 = 20.0 * (1.5 + np.sin(2 * x_) * np.cos(y_))
    S.sem_set_helmholtz(H.h, h2)
    P.set_h2(h2)
    u = W.random_local_field(m, 44, continuous=True)
    e_tc, _ = rel_err(H.ax(u.astype(np.float32), S.SEM_TC_SPLIT, assemble=1), P.ax(u))
    assert e_tc <= 5e-5, e_tc
    x, st = H.solve(b, tol=TOL, mode=S.SEM_MODE_MIXED_IR, tc_split=1)
    assert st["status"] == S.SEM_OK and _oracle_relres(P, x, b) <= 1.05 * TOL, st


def test_tc_pinned_variant_and_other_orders_fall_back():
    m, h1 = _case("deformed", (3, 2, 2))
    H8 = Handle(m, h1, flags=S.SEM_FLAG_VARIANT(8))
    H = Handle(m, h1)
    u = W.random_local_field(m, 45).astype(np.float32)
    # variant 8 pinned: SEM_FP32 applications take the tensor-core kernel
    assert np.array_equal(H8.ax(u, S.SEM_FP32, assemble=0), H.ax(u, S.SEM_TC_SPLIT, assemble=0))
    m5 = W.box_mesh(3, 2, 2, 5, amp=0.05)
    H5 = Handle(m5)
    u5 = W.random_local_field(m5, 46).astype(np.float32)
    assert np.array_equal(H5.ax(u5, S.SEM_TC_SPLIT, assemble=0), H5.ax(u5, S.SEM_FP32, assemble=0))
