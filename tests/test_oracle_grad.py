"""Pins of the oracle's collocation gradient, divergence, curl and pressure
right-hand side (Sec. II-A): on affine meshes (sheared, so the metric terms
are not diagonal) the collocation derivative of a polynomial of degree <= N
is exact, so curl(grad) and div(curl) vanish to rounding; on deformed meshes
the gradient of a smooth field converges spectrally; the pressure
right-hand side of a gradient field vhat = grad(phi) is -B lap(phi) / dt,
assembled."""
import numpy as np
import pytest

import oracle
import workloads as W

SHEAR = np.array([[1.0, 0.3, -0.2], [0.1, 0.9, 0.25], [-0.15, 0.2, 1.1]])


def sheared(nx, ny, nz, N):
    m = W.box_mesh(nx, ny, nz, N)
    c = m.coords.reshape(3, -1)
    m.coords = (SHEAR @ c).reshape(m.coords.shape)
    return m


def _poly(m, N):
    """A polynomial of total degree N with random coefficients, its gradient
    and its Laplacian (exact)."""
    x, y, z = m.xyz()
    rng = np.random.default_rng(N)
    terms = [(a, b, N - a - b) for a in range(N + 1) for b in range(N + 1 - a)]
    terms += [(1, 0, 0), (0, 1, 1), (2, 0, 0)] if N >= 2 else []
    u = np.zeros_like(x)
    g = np.zeros((3,) + x.shape)
    lap = np.zeros_like(x)
    for (a, b, c) in terms:
        co = rng.standard_normal()
        u += co * x ** a * y ** b * z ** c
        g[0] += co * a * x ** max(a - 1, 0) * y ** b * z ** c
        g[1] += co * b * x ** a * y ** max(b - 1, 0) * z ** c
        g[2] += co * c * x ** a * y ** b * z ** max(c - 1, 0)
        lap += co * (a * (a - 1) * x ** max(a - 2, 0) * y ** b * z ** c
                     + b * (b - 1) * x ** a * y ** max(b - 2, 0) * z ** c
                     + c * (c - 1) * x ** a * y ** b * z ** max(c - 2, 0))
    return u, g, lap


@pytest.mark.parametrize("N", [2, 4, 7])
def test_gradient_exact_on_affine_meshes(N):
    m = sheared(3, 2, 2, N)
    u, g, _ = _poly(m, N)
    got = oracle.grad(m, u)
    assert np.max(np.abs(got - g)) <= 1e-10 * np.max(np.abs(g))


@pytest.mark.parametrize("N", [3, 6])
def test_curl_grad_and_div_curl_vanish_on_affine_meshes(N):
    m = sheared(2, 3, 2, N)
    u, g, _ = _poly(m, N)
    cg = oracle.curl(m, *oracle.grad(m, u))
    assert np.max(np.abs(cg)) <= 1e-9 * np.max(np.abs(g))
    v = [_poly(m, N)[0], np.sin(0.0 * u) + _poly(m, N - 1)[0], _poly(m, N)[0] * 0.5]
    dc = oracle.div(m, *oracle.curl(m, *v))
    assert np.max(np.abs(dc)) <= 1e-8 * max(np.max(np.abs(x)) for x in v)


def test_gradient_converges_spectrally_on_deformed_meshes():
    errs = []
    for N in (3, 5, 7, 9):
        m = W.box_mesh(2, 2, 2, N, amp=0.05)
        x, y, z = m.xyz()
        u = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        gx = np.pi * np.cos(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        errs.append(np.max(np.abs(oracle.grad(m, u)[0] - gx)))
    assert all(errs[q + 1] < 0.2 * errs[q] for q in range(3)) and errs[-1] < 1e-4, errs


def test_pressure_rhs_of_a_gradient_field():
    N = 5
    m = sheared(2, 2, 2, N)
    P = oracle.Problem(m)
    phi, g, lap = _poly(m, N)
    dt, Re = 0.01, 300.0
    b = oracle.pressure_rhs(P, m, list(g), None, dt, Re)
    ref = P.mass(-lap / dt, assemble=True)
    assert np.max(np.abs(b - ref)) <= 1e-9 * np.max(np.abs(ref))
    # the vorticity term is div(curl(omega)) = 0 on affine elements
    om = [_poly(m, N)[0], 0.3 * phi, -phi]
    b2 = oracle.pressure_rhs(P, m, list(g), om, dt, Re)
    assert np.max(np.abs(b2 - b)) <= 1e-8 * np.max(np.abs(b))


def test_metric_transposition_is_caught():
    """A plausible slip, du/dx_l = sum_s (dr_l/dx_s) du/dr_s (transposed
    metric), fails the polynomial pin on the sheared mesh."""
    m = sheared(2, 2, 2, 4)
    u, g, _ = _poly(m, 4)
    D = oracle.dmat(4)
    d = np.array(oracle._ref_derivs(D, u, m.lx))
    M = oracle.metrics(m)
    wrong = np.einsum("nls,sn->ln", M, d)
    assert np.max(np.abs(wrong - g)) > 1e-3 * np.max(np.abs(g))
