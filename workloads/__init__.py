"""Seeded synthetic inputs for the spectral-element Poisson solve.

This module is shared by the FP64 oracle (``oracle/``), the CUDA path
(``paper_2207_07098_gb300``), the tests and the benchmark.  It holds none of
the method's arithmetic: no derivative matrix, no geometric factor, no
operator, no gather-scatter and no solver.  What it produces is what a mesh
file and a case setup would hand to a solver:

* node coordinates of hexahedral elements placed at Gauss-Lobatto-Legendre
  (GLL) positions in each direction (Sec. II-A: ``(N+1)^3`` GLL points per
  element), element-major ``[3][E][k][j][i]`` with ``i`` fastest;
* global node ids (equal ids <=> same physical node, including periodic
  identification), which define the scatter operator Q of Sec. II-A;
* the homogeneous Dirichlet mask (0 on Dirichlet nodes, 1 elsewhere);
* coefficient fields (``h1``) and forcing fields sampled at the nodes;
* seeded random right-hand sides drawn per global node.

The GLL positions used to place mesh nodes come from numpy's Legendre
routines (roots of P_N'), a library primitive independent of both the
oracle's Newton iteration and the CUDA library's own node computation.
Random numbers come from ``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

import dataclasses
import numpy as np


def gll_positions(N: int) -> np.ndarray:
    """Positions of the N+1 GLL points on [-1, 1] used to place mesh nodes.

    Endpoints are -1 and 1; interior points are the roots of P_N' (numpy's
    companion-matrix root finder on the Legendre series of P_N').
    """
    if N < 1:
        raise ValueError("polynomial order N must be >= 1")
    if N == 1:
        return np.array([-1.0, 1.0])
    from numpy.polynomial import legendre as leg

    c = np.zeros(N + 1)
    c[N] = 1.0
    inner = np.sort(np.real(leg.legroots(leg.legder(c))))
    return np.concatenate([[-1.0], inner, [1.0]])


@dataclasses.dataclass
class Mesh:
    """One hexahedral spectral-element mesh in local (element-major) layout.

    coords: float64 [3, E, lx**3]  (x, y, z of every local node; i fastest)
    gid:    int64   [E * lx**3]    global node id of every local node
    mask:   uint8   [E * lx**3]    0 on homogeneous Dirichlet nodes, else 1
    """

    E: int
    lx: int
    coords: np.ndarray
    gid: np.ndarray
    mask: np.ndarray
    name: str = ""
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.lx - 1

    @property
    def n_local(self) -> int:
        return self.E * self.lx ** 3

    def xyz(self):
        return self.coords[0].reshape(-1), self.coords[1].reshape(-1), self.coords[2].reshape(-1)


def _local_ijk(lx: int):
    """Index arrays (i, j, k) of the lx^3 local points of one element, i fastest."""
    k, j, i = np.meshgrid(np.arange(lx), np.arange(lx), np.arange(lx), indexing="ij")
    return i.reshape(-1), j.reshape(-1), k.reshape(-1)


def box_mesh(nx: int, ny: int, nz: int, N: int, amp: float = 0.0,
             lengths=(1.0, 1.0, 1.0), name: str = "box", jitter: float = 0.0,
             seed: int = 0) -> Mesh:
    """Structured nx*ny*nz hex mesh of the box [0,Lx]x[0,Ly]x[0,Lz].

    Element e = ex + nx*(ey + ny*ez); node (i,j,k) of element e sits at
    x = (ex + (xi_i+1)/2) * Lx/nx (likewise y, z).  With ``amp`` > 0 every
    node is displaced, as a function of its undeformed position (X,Y,Z), by
    ``amp * h_d * sin(2 pi X/Lx) sin(2 pi Y/Ly) sin(2 pi Z/Lz)`` in each
    coordinate d, with h_d the element width in direction d.  The product of
    sines vanishes on every face of the box, so the boundary and the
    coincidence of shared nodes are preserved.  With ``jitter`` > 0 every
    node off the boundary is further moved by an independent U(-1,1) *
    jitter * h_d per coordinate, drawn once per global node (seeded), so
    copies of a node still coincide but the map is only continuous across
    elements.  Homogeneous Dirichlet on all six faces.
    """
    lx = N + 1
    E = nx * ny * nz
    s = (gll_positions(N) + 1.0) / 2.0
    i, j, k = _local_ijk(lx)
    e = np.arange(E)
    ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
    Lx, Ly, Lz = lengths
    X = (ex[:, None] + s[i][None, :]) * (Lx / nx)
    Y = (ey[:, None] + s[j][None, :]) * (Ly / ny)
    Z = (ez[:, None] + s[k][None, :]) * (Lz / nz)
    if amp != 0.0:
        S = (np.sin(2 * np.pi * X / Lx) * np.sin(2 * np.pi * Y / Ly)
             * np.sin(2 * np.pi * Z / Lz))
        x = X + amp * (Lx / nx) * S
        y = Y + amp * (Ly / ny) * S
        z = Z + amp * (Lz / nz) * S
    else:
        x, y, z = X, Y, Z
    gx = ex[:, None] * N + i[None, :]
    gy = ey[:, None] * N + j[None, :]
    gz = ez[:, None] * N + k[None, :]
    mx, my, mz = nx * N, ny * N, nz * N
    gid = (gx + (mx + 1) * (gy + (my + 1) * gz)).astype(np.int64).reshape(-1)
    dirichlet = ((gx == 0) | (gx == mx) | (gy == 0) | (gy == my) | (gz == 0) | (gz == mz))
    if jitter != 0.0:
        n_g = (mx + 1) * (my + 1) * (mz + 1)
        rnd = np.random.default_rng(seed).uniform(-1.0, 1.0, size=(3, n_g))
        free = ~dirichlet.reshape(-1)
        g = gid.reshape(x.shape)
        for d, (c, h) in enumerate(((x, Lx / nx), (y, Ly / ny), (z, Lz / nz))):
            c += np.where(free.reshape(x.shape), jitter * h * rnd[d][g], 0.0)
    coords = np.ascontiguousarray(np.stack([x, y, z]))
    mask = (~dirichlet).astype(np.uint8).reshape(-1)
    return Mesh(E, lx, coords, gid, mask, name=name,
                meta=dict(kind="box", nx=nx, ny=ny, nz=nz, N=N, amp=amp, lengths=tuple(lengths)))


def annulus_mesh(n_theta: int = 64, n_r: int = 32, n_z: int = 24, N: int = 7,
                 r0: float = 0.5, r1: float = 8.0, ratio: float = 1.1,
                 Lz: float = 4.0, name: str = "annulus") -> Mesh:
    """Isoparametric O-grid annulus r0 <= r <= r1, periodic in theta and z.

    Radial element edges r_k = r0 + h0 (ratio^k - 1)/(ratio - 1) with
    h0 chosen so that r_{n_r} = r1.  Local i runs radially, j azimuthally and
    k spanwise; element e = ir + n_r*(it + n_theta*iz).  Every node is placed
    exactly on its circle (x = r cos(theta), y = r sin(theta)).  Global ids
    identify theta = 0 with theta = 2 pi and z = 0 with z = Lz (periodic
    gather-scatter); Dirichlet at r = r0 and r = r1.
    """
    lx = N + 1
    E = n_theta * n_r * n_z
    s = (gll_positions(N) + 1.0) / 2.0
    h0 = (r1 - r0) * (ratio - 1.0) / (ratio ** n_r - 1.0)
    edges = r0 + h0 * (ratio ** np.arange(n_r + 1) - 1.0) / (ratio - 1.0)
    edges[-1] = r1
    i, j, k = _local_ijk(lx)
    e = np.arange(E)
    ir, it, iz = e % n_r, (e // n_r) % n_theta, e // (n_r * n_theta)
    r = edges[ir][:, None] + (edges[ir + 1] - edges[ir])[:, None] * s[i][None, :]
    th = 2.0 * np.pi * (it[:, None] + s[j][None, :]) / n_theta
    z = Lz * (iz[:, None] + s[k][None, :]) / n_z
    coords = np.ascontiguousarray(np.stack([r * np.cos(th), r * np.sin(th), z]))
    gr = ir[:, None] * N + i[None, :]
    gt = (it[:, None] * N + j[None, :]) % (n_theta * N)
    gz = (iz[:, None] * N + k[None, :]) % (n_z * N)
    gid = (gr + (n_r * N + 1) * (gt + n_theta * N * gz)).astype(np.int64).reshape(-1)
    mask = (~((gr == 0) | (gr == n_r * N))).astype(np.uint8).reshape(-1)
    return Mesh(E, lx, coords, gid, mask, name=name,
                meta=dict(kind="annulus", n_theta=n_theta, n_r=n_r, n_z=n_z, N=N, r0=r0,
                          r1=r1, ratio=ratio, Lz=Lz))


# ----------------------------------------------------------------------------
# fields sampled at the nodes
# ----------------------------------------------------------------------------

def forcing_sines(mesh: Mesh) -> np.ndarray:
    """f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z) at every local node (cube case)."""
    x, y, z = mesh.xyz()
    return 3.0 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def exact_sines(mesh: Mesh) -> np.ndarray:
    """u = sin(pi x) sin(pi y) sin(pi z), the solution of -lap u = forcing_sines."""
    x, y, z = mesh.xyz()
    return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def h1_wavy(mesh: Mesh) -> np.ndarray:
    """h1 = 1 + 0.5 sin(4 pi x) cos(2 pi y) at the (deformed) node coordinates."""
    x, y, _ = mesh.xyz()
    return 1.0 + 0.5 * np.sin(4.0 * np.pi * x) * np.cos(2.0 * np.pi * y)


def random_global_rhs(mesh: Mesh, seed: int) -> np.ndarray:
    """b ~ N(0,1) per global node (ordered by ascending id), zero on Dirichlet nodes,
    copied to every local copy of the node."""
    ug, inv = np.unique(mesh.gid, return_inverse=True)
    rng = np.random.default_rng(seed)
    vals = rng.standard_normal(ug.shape[0])
    return vals[inv] * mesh.mask.astype(np.float64)


def fourier_forcing(mesh: Mesh, seed: int, kmax: int = 4, Lxy: float = 16.0,
                    Lz: float = 4.0, chunk: int = 1 << 20) -> np.ndarray:
    """Smooth random field f = sum_{k in Z^3, 0<|k|<=kmax} a_k cos(2 pi (kx x/Lxy +
    ky y/Lxy + kz z/Lz) + phi_k), a_k ~ N(0,1)/|k|^2, phi_k ~ U(0, 2 pi).

    Wave vectors are enumerated lexicographically (kx, ky, kz from -kmax to
    kmax); a_k is drawn for all of them first, then phi_k.  The z wavenumbers
    are multiples of 2 pi / Lz, so f is periodic in z.
    """
    ks = [(a, b, c) for a in range(-kmax, kmax + 1) for b in range(-kmax, kmax + 1)
          for c in range(-kmax, kmax + 1) if 0 < a * a + b * b + c * c <= kmax * kmax]
    ks = np.array(ks, dtype=np.float64)
    rng = np.random.default_rng(seed)
    knorm2 = (ks ** 2).sum(axis=1)
    amp = rng.standard_normal(ks.shape[0]) / knorm2
    phi = rng.uniform(0.0, 2.0 * np.pi, ks.shape[0])
    x, y, z = mesh.xyz()
    out = np.empty_like(x)
    for c0 in range(0, x.shape[0], chunk):
        c1 = min(c0 + chunk, x.shape[0])
        arg = (2.0 * np.pi) * (np.outer(x[c0:c1], ks[:, 0] / Lxy) + np.outer(y[c0:c1], ks[:, 1] / Lxy)
                               + np.outer(z[c0:c1], ks[:, 2] / Lz)) + phi[None, :]
        out[c0:c1] = np.cos(arg) @ amp
    return out


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def cube_sines(n: int = 4, N: int = 7) -> tuple[Mesh, np.ndarray]:
    """Unit cube, n^3 affine elements, order N, Dirichlet on all faces, h1 = 1.
    Returns (mesh, f) with f the manufactured forcing 3 pi^2 sin sin sin;
    the right-hand side is b = mask * QQ^T (B f)."""
    m = box_mesh(n, n, n, N, name=f"cube{n}^3_N{N}")
    return m, forcing_sines(m)


def deformed_cube(n: int = 32, N: int = 7, seed: int = 2):
    """n^3 elements of order N on the unit cube, nodes deformed by
    0.05 h sin sin sin, h1 = 1 + 0.5 sin(4 pi x) cos(2 pi y), random N(0,1)
    right-hand side per global node, masked.  Returns (mesh, h1, b)."""
    m = box_mesh(n, n, n, N, amp=0.05, name=f"deformed{n}^3_N{N}")
    return m, h1_wavy(m), random_global_rhs(m, seed)


def annulus_case(N: int = 7, seed: int = 5, n_theta: int = 64, n_r: int = 32, n_z: int = 24):
    """O-grid annulus (r in [0.5, 8], span 4 periodic) with the smooth random
    Fourier forcing.  Returns (mesh, f); b = mask * QQ^T (B f)."""
    m = annulus_mesh(n_theta=n_theta, n_r=n_r, n_z=n_z, N=N)
    return m, fourier_forcing(m, seed)


@dataclasses.dataclass
class BatchMember:
    nx: int
    ny: int
    nz: int
    N: int
    amp: float
    seed: int


def batch_params(nsolve: int = 256, seed: int = 4, nmin: int = 2, nmax: int = 16,
                 orders=(5, 7, 9), amp_max: float = 0.08) -> list[BatchMember]:
    """Parameters of the batch of independent box solves, drawn from one master
    stream: per solve nx, ny, nz ~ U{nmin..nmax}, N ~ U(orders),
    deformation amplitude ~ U(0, amp_max) (times the element width), and a
    right-hand-side seed."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nsolve):
        nx, ny, nz = (int(v) for v in rng.integers(nmin, nmax + 1, size=3))
        N = int(rng.choice(np.asarray(orders)))
        amp = float(rng.uniform(0.0, amp_max))
        s = int(rng.integers(0, 2 ** 62))
        out.append(BatchMember(nx, ny, nz, N, amp, s))
    return out


def batch_member_case(p: BatchMember):
    """Mesh and random right-hand side of one batch member (h1 = 1)."""
    m = box_mesh(p.nx, p.ny, p.nz, p.N, amp=p.amp, name=f"box{p.nx}x{p.ny}x{p.nz}_N{p.N}")
    return m, random_global_rhs(m, p.seed)


def random_local_field(mesh: Mesh, seed: int, continuous: bool = False) -> np.ndarray:
    """N(0,1) values at every local node (``continuous``: one value per global
    node copied to all its copies)."""
    rng = np.random.default_rng(seed)
    if continuous:
        ug, inv = np.unique(mesh.gid, return_inverse=True)
        return rng.standard_normal(ug.shape[0])[inv]
    return rng.standard_normal(mesh.n_local)


__all__ = [
    "Mesh", "gll_positions", "box_mesh", "annulus_mesh", "forcing_sines", "exact_sines",
    "h1_wavy", "random_global_rhs", "fourier_forcing", "cube_sines", "deformed_cube",
    "annulus_case", "BatchMember", "batch_params", "batch_member_case", "random_local_field",
]
