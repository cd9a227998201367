"""Pins of the oracle's geometric factors, local operator, gather-scatter and
Jacobi diagonal (Sec. II-A, II-B) to closed forms, invariants and a dense
brute-force assembly."""
import numpy as np
import pytest

import oracle
import workloads as W
import dense_ref


def _expected_mult_box(m):
    """Copies of each local node from the box structure: a node on an internal
    element interface in d directions has 2^d copies."""
    N, (nx, ny, nz) = m.N, (m.meta["nx"], m.meta["ny"], m.meta["nz"])
    lx = m.lx
    e = np.arange(m.E)
    k, j, i = np.meshgrid(np.arange(lx), np.arange(lx), np.arange(lx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    gx = (e % nx)[:, None] * N + i[None, :]
    gy = ((e // nx) % ny)[:, None] * N + j[None, :]
    gz = (e // (nx * ny))[:, None] * N + k[None, :]
    c = np.ones(gx.shape)
    for g, n in ((gx, nx), (gy, ny), (gz, nz)):
        c *= np.where((g % N == 0) & (g > 0) & (g < n * N), 2.0, 1.0)
    return c.ravel()


@pytest.mark.parametrize("dims,N", [((2, 2, 2), 3), ((3, 2, 4), 4), ((1, 1, 1), 5), ((2, 3, 1), 1)])
def test_gs_multiplicity_box(dims, N):
    m = W.box_mesh(*dims, N)
    P = oracle.Problem(m)
    np.testing.assert_array_equal(P.mult(), _expected_mult_box(m))
    np.testing.assert_array_equal(P.gs(np.ones(m.n_local), mask=False), _expected_mult_box(m))


def test_gs_multiplicity_annulus_periodic():
    m = W.annulus_mesh(n_theta=4, n_r=2, n_z=3, N=3)
    P = oracle.Problem(m)
    N = m.N
    lx = m.lx
    e = np.arange(m.E)
    k, j, i = np.meshgrid(np.arange(lx), np.arange(lx), np.arange(lx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    gr = (e % 2)[:, None] * N + i[None, :]
    c = np.where((gr % N == 0) & (gr > 0) & (gr < 2 * N), 2.0, 1.0)
    c = c * np.where(j[None, :] % N == 0, 2.0, 1.0) * np.where(k[None, :] % N == 0, 2.0, 1.0)
    np.testing.assert_array_equal(P.mult(), c.ravel())
    assert P.n_unique == (2 * N + 1) * (4 * N) * (3 * N)


def test_gs_sum_invariance_and_projection():
    m = W.box_mesh(3, 2, 2, 4, amp=0.05)
    P = oracle.Problem(m)
    rng = np.random.default_rng(0)
    w = rng.standard_normal(m.n_local)
    s = P.gs(w, mask=False)
    # sum over unique nodes of the assembled vector = sum over local copies
    assert abs(np.sum(s / P.mult()) - np.sum(w)) < 1e-11 * np.abs(w).sum()
    # QQ^T applied to a continuous vector multiplies it by the multiplicity
    ug = W.random_local_field(m, 1, continuous=True)
    np.testing.assert_allclose(P.gs(ug, mask=False), ug * P.mult(), rtol=1e-15)
    # all copies of a node agree after QQ^T
    _, inv = np.unique(m.gid, return_inverse=True)
    first = np.zeros(inv.max() + 1)
    first[inv[::-1]] = s[::-1]
    assert np.array_equal(s, first[inv])


@pytest.mark.parametrize("dims", [(2, 2, 2), (3, 1, 2)])
@pytest.mark.parametrize("N", [1, 3, 6])
def test_geometry_affine_closed_form(dims, N):
    L = (1.0, 2.0, 0.5)
    m = W.box_mesh(*dims, N, lengths=L)
    P = oracle.Problem(m)
    G, B = P.geom()
    _, rho = oracle.gll(N)
    hx, hy, hz = (L[d] / dims[d] for d in range(3))
    w3 = np.kron(rho, np.kron(rho, rho))
    w = np.tile(w3, m.E)
    np.testing.assert_allclose(G[0], w * hy * hz / (2 * hx), rtol=1e-13)
    np.testing.assert_allclose(G[3], w * hx * hz / (2 * hy), rtol=1e-13)
    np.testing.assert_allclose(G[5], w * hx * hy / (2 * hz), rtol=1e-13)
    for q in (1, 2, 4):
        assert np.max(np.abs(G[q])) < 1e-13 * np.max(np.abs(G[0]))
    np.testing.assert_allclose(B, w * hx * hy * hz / 8, rtol=1e-13)


def test_volume_deformed_cube():
    m = W.box_mesh(3, 3, 3, 5, amp=0.05)
    P = oracle.Problem(m)
    _, B = P.geom()
    # each local copy carries its own element's quadrature weight: volume = sum_L B_L
    assert abs(np.sum(B) - 1.0) < 1e-13
    one = np.ones(m.n_local)
    assert abs(P.dot(one, P.gs(B, mask=False)) - 1.0) < 1e-13


def test_volume_annulus():
    m = W.annulus_mesh(n_theta=16, n_r=4, n_z=2, N=7)
    P = oracle.Problem(m)
    _, B = P.geom()
    vol = np.sum(B)
    assert abs(vol - 255.0 * np.pi) / (255.0 * np.pi) < 1e-8


def test_volume_annulus_full_size():
    """The annulus workload (64 x 32 x 24 elements, N = 7): volume 255 pi."""
    m = W.annulus_mesh()
    P = oracle.Problem(m)
    _, B = P.geom()
    assert abs(np.sum(B) - 255.0 * np.pi) / (255.0 * np.pi) < 1e-8


@pytest.mark.parametrize("N", [1, 2, 4, 7])
def test_ax_constant_in_kernel(N):
    m = W.box_mesh(2, 3, 2, N, amp=0.05)
    h1 = W.h1_wavy(m)
    P = oracle.Problem(m, h1)
    w = P.ax_local(np.ones(m.n_local))
    G, _ = P.geom()
    assert np.max(np.abs(w)) < 1e-12 * np.max(np.abs(G))
    w = P.gs(P.ax_local(np.full(m.n_local, 3.0)), mask=False)
    assert np.max(np.abs(w)) < 1e-12 * np.max(np.abs(G))


@pytest.mark.parametrize("N", [1, 3, 5])
def test_ax_affine_kronecker_closed_form(N):
    L = (1.0, 0.5, 2.0)
    dims = (2, 2, 1)
    m = W.box_mesh(*dims, N, lengths=L)
    P = oracle.Problem(m)
    _, rho = oracle.gll(N)
    K = dense_ref.stiffness_1d_exact(N)
    Wd = np.diag(rho)
    hx, hy, hz = (L[d] / dims[d] for d in range(3))
    Ae = (hy * hz / (2 * hx)) * np.kron(Wd, np.kron(Wd, K)) \
        + (hx * hz / (2 * hy)) * np.kron(Wd, np.kron(K, Wd)) \
        + (hx * hy / (2 * hz)) * np.kron(K, np.kron(Wd, Wd))
    rng = np.random.default_rng(1)
    u = rng.standard_normal(m.n_local)
    w = P.ax_local(u)
    n3 = m.lx ** 3
    ref = np.concatenate([Ae @ u[e * n3:(e + 1) * n3] for e in range(m.E)])
    assert np.max(np.abs(w - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("dims,N,jitter", [((1, 1, 1), 4, 0.0), ((2, 2, 2), 2, 0.0), ((2, 1, 2), 3, 0.0),
                                           ((2, 2, 2), 4, 0.0), ((3, 2, 2), 2, 0.03), ((2, 2, 2), 3, 0.02)])
def test_ax_dense_bruteforce_deformed(dims, N, jitter):
    """Oracle A = mask QQ^T A_L against a dense matrix built from explicit
    Kronecker products, numpy Jacobians and an explicit Q (smoothly deformed
    and node-jittered meshes)."""
    m = W.box_mesh(*dims, N, amp=0.1, jitter=jitter, seed=3)
    h1 = W.h1_wavy(m)
    P = oracle.Problem(m, h1)
    K, Q, mask_g, Ae, Bm = dense_ref.assembled(m, h1)
    rng = np.random.default_rng(2)
    # local operator, element by element
    u = rng.standard_normal(m.n_local)
    n3 = m.lx ** 3
    ref_local = np.concatenate([Ae[e] @ u[e * n3:(e + 1) * n3] for e in range(m.E)])
    wl = P.ax_local(u)
    assert np.max(np.abs(wl - ref_local)) < 1e-13 * np.max(np.abs(ref_local)) * 10
    # assembled, masked operator on a continuous vector
    ug = rng.standard_normal(Q.shape[1])
    w = P.ax(Q @ ug)
    ref = Q @ (mask_g * (K @ ug))
    assert np.max(np.abs(w - ref)) < 1e-13 * np.max(np.abs(ref)) * 10
    # geometry: mass matrix
    _, B = P.geom()
    np.testing.assert_allclose(B, Bm.ravel(), rtol=1e-12)
    # Jacobi diagonal = diagonal of the dense assembled matrix (free nodes)
    minv = P.minv()
    dg = np.diag(K)
    ref_minv = np.where(m.mask > 0, 1.0 / dg[np.unique(m.gid, return_inverse=True)[1]], 0.0)
    np.testing.assert_allclose(minv, ref_minv, rtol=1e-12)


def test_ax_symmetric_positive_definite():
    m = W.box_mesh(2, 2, 3, 4, amp=0.05)
    h1 = W.h1_wavy(m)
    P = oracle.Problem(m, h1)
    rng = np.random.default_rng(3)
    for s in range(3):
        u = W.random_local_field(m, 10 + s, continuous=True) * m.mask
        v = W.random_local_field(m, 20 + s, continuous=True) * m.mask
        a = P.dot(v, P.ax(u))
        b = P.dot(u, P.ax(v))
        assert abs(a - b) < 1e-13 * (abs(a) + abs(b))
        assert P.dot(u, P.ax(u)) > 0.0


@pytest.mark.parametrize("dims,N,jitter", [((2, 1, 1), 3, False), ((2, 2, 1), 4, True)])
def test_ax_magnitude_operator(dims, N, jitter):
    """The oracle's |D^T| |h1 G| |D| |u| (the scale of rounding errors of any
    evaluation of A_L u) equals the nonnegative dense matrix built from
    Kronecker products of |D| and numpy Jacobians, bounds |A_L u| pointwise,
    and is absolutely homogeneous."""
    m = W.box_mesh(*dims, N, amp=0.05, jitter=0.25 / N ** 2 if jitter else 0.0, seed=3)
    h1 = W.h1_wavy(m)
    P = oracle.Problem(m, h1)
    u = W.random_local_field(m, 41)
    a = P.ax_local_abs(u)
    M = dense_ref.element_magnitude_matrices(m, h1)
    n3 = m.lx ** 3
    ref = np.concatenate([M[e] @ np.abs(u[e * n3:(e + 1) * n3]) for e in range(m.E)])
    assert np.max(np.abs(a - ref)) <= 1e-13 * np.max(ref)
    assert np.all(a >= np.abs(P.ax_local(u)))
    assert np.allclose(P.ax_local_abs(-3.0 * u), 3.0 * a, rtol=1e-15, atol=0)


def test_mass_integrates_constant():
    m = W.box_mesh(2, 2, 2, 5, amp=0.05)
    P = oracle.Problem(m)
    # assembled unmasked mass of the constant 1 sums (over unique nodes) to the volume
    _, B = P.geom()
    w = P.mass(np.ones(m.n_local), assemble=False)
    np.testing.assert_array_equal(w, B)
    assert abs(w.sum() - 1.0) < 1e-13
