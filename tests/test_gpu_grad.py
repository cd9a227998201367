"""GPU parity of the collocation gradient, divergence and curl and of the
pressure right-hand side (Sec. II-A, eq. "pressure") against the oracle's
numpy restatement (metric terms from its own Jacobians), through the C ABI,
on sheared affine, deformed and annulus meshes of several orders."""
import numpy as np
import pytest

import oracle
import workloads as W
import paper_2207_07098_gb300 as S
from gpu_helpers import dev, host, rel_err

pytestmark = pytest.mark.gpu

SHEAR = np.array([[1.0, 0.3, -0.2], [0.1, 0.9, 0.25], [-0.15, 0.2, 1.1]])


def _mesh(kind, N):
    if kind == "sheared":
        m = W.box_mesh(3, 2, 2, N)
        m.coords = (SHEAR @ m.coords.reshape(3, -1)).reshape(m.coords.shape)
        return m
    if kind == "deformed":
        return W.box_mesh(3, 3, 2, N, amp=0.06)
    return W.annulus_mesh(n_theta=8, n_r=3, n_z=2, N=N)


def _fields(m, seed):
    rng = np.random.default_rng(seed)
    x, y, z = m.xyz()
    a = rng.uniform(0.5, 2.0, size=6)
    return [np.sin(a[0] * x + a[1] * y) * np.cos(a[2] * z), np.cos(a[3] * x * y) + z * z,
            np.sin(a[4] * z) * x + np.cos(a[5] * y)]


def _close(got, ref):
    scale = np.max(np.abs(ref)) if np.max(np.abs(ref)) > 0 else 1.0
    return np.max(np.abs(got - ref)) <= 1e-12 * scale * 8


@pytest.mark.parametrize("kind,N", [("sheared", 3), ("deformed", 5), ("deformed", 7), ("annulus", 6)])
def test_grad_div_curl_match_oracle(kind, N):
    import torch
    m = _mesh(kind, N)
    h = S.sem_setup(m.E, m.lx, m.coords, m.gid, m.mask, None, S.SEM_FLAG_METRICS)
    try:
        v = _fields(m, N)
        vd = [dev(f, torch.float64) for f in v]
        out = [torch.empty_like(vd[0]) for _ in range(3)]
        S.sem_grad(h, vd[0], *out)
        ref = oracle.grad(m, v[0])
        for q in range(3):
            assert _close(host(out[q]), ref[q]), ("grad", q)
        d = torch.empty_like(vd[0])
        S.sem_div(h, *vd, d)
        assert _close(host(d), oracle.div(m, *v)), "div"
        S.sem_curl(h, *vd, *out)
        ref = oracle.curl(m, *v)
        for q in range(3):
            assert _close(host(out[q]), ref[q]), ("curl", q)
    finally:
        S.sem_destroy(h)


@pytest.mark.parametrize("kind,N", [("deformed", 7), ("annulus", 5)])
def test_pressure_rhs_matches_oracle(kind, N):
    import torch
    m = _mesh(kind, N)
    P = oracle.Problem(m)
    h = S.sem_setup(m.E, m.lx, m.coords, m.gid, m.mask, None, S.SEM_FLAG_METRICS)
    try:
        v, w = _fields(m, 1), _fields(m, 2)
        dt, Re = 2e-3, 500.0
        b = torch.empty(m.n_local, dtype=torch.float64, device="cuda")
        S.sem_pressure_rhs(h, *[dev(f, torch.float64) for f in v], *[dev(f, torch.float64) for f in w], dt, Re, b)
        e2, _ = rel_err(host(b), oracle.pressure_rhs(P, m, v, w, dt, Re))
        assert e2 <= 1e-12, e2
        S.sem_pressure_rhs(h, *[dev(f, torch.float64) for f in v], None, None, None, dt, Re, b)
        e2, _ = rel_err(host(b), oracle.pressure_rhs(P, m, v, None, dt, Re))
        assert e2 <= 1e-12, e2
    finally:
        S.sem_destroy(h)


def test_operators_need_metrics():
    import torch
    m = W.box_mesh(2, 2, 2, 3)
    h = S.sem_setup(m.E, m.lx, m.coords, m.gid, m.mask, None)
    try:
        u = torch.zeros(m.n_local, dtype=torch.float64, device="cuda")
        with pytest.raises(S.SemError) as ei:
            S.sem_grad(h, u, u.clone(), u.clone(), u.clone())
        assert ei.value.status == S.SEM_EINVAL
    finally:
        S.sem_destroy(h)
