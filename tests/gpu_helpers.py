"""Helpers of the GPU parity tests: build handles through the C ABI, move
numpy arrays to the device, and measure relative errors."""
from __future__ import annotations

import numpy as np

import paper_2207_07098_gb300 as S


def torch():
    import torch as _t
    return _t


def dev(a, dtype=None):
    t = torch()
    arr = np.ascontiguousarray(a)
    ten = t.from_numpy(arr).cuda()
    return ten if dtype is None else ten.to(dtype)


def host(t_):
    return t_.detach().cpu().numpy()


class Handle:
    """A libsem handle for one workloads.Mesh (destroyed with the object)."""

    def __init__(self, mesh, h1=None, flags=0):
        self.mesh = mesh
        self.h = S.sem_setup(mesh.E, mesh.lx, mesh.coords, mesh.gid, mesh.mask, h1, flags)
        self.info = S.sem_get_info(self.h)
        self.n = self.info["n_local"]

    def close(self):
        if self.h:
            S.sem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ax(self, u, precision=S.SEM_FP64, assemble=1):
        t = torch()
        dt = t.float32 if precision in (S.SEM_FP32, S.SEM_TC_SPLIT) else t.float64
        ud = dev(u, dt)
        w = t.empty_like(ud)
        S.sem_ax(self.h, w, ud, precision, assemble)
        t.cuda.synchronize()
        return host(w).astype(np.float64)

    def gs(self, u, precision=S.SEM_FP64, mask=1):
        t = torch()
        dt = t.float32 if precision in (S.SEM_FP32, S.SEM_TC_SPLIT) else t.float64
        ud = dev(u, dt)
        S.sem_gs(self.h, ud, precision, mask)
        t.cuda.synchronize()
        return host(ud).astype(np.float64)

    def mass(self, u, assemble=1):
        t = torch()
        ud = dev(u, t.float64)
        w = t.empty_like(ud)
        S.sem_mass(self.h, w, ud, S.SEM_FP64, assemble)
        t.cuda.synchronize()
        return host(w)

    def dot(self, a, b):
        t = torch()
        out = t.zeros(self.info["nsolve"], dtype=t.float64, device="cuda")
        S.sem_dot(self.h, dev(a, t.float64), dev(b, t.float64), out)
        t.cuda.synchronize()
        return host(out)

    def geometry(self):
        t = torch()
        G = t.empty(6 * self.n, dtype=t.float64, device="cuda")
        B = t.empty(self.n, dtype=t.float64, device="cuda")
        S.sem_get_geometry(self.h, G, B)
        t.cuda.synchronize()
        lx3 = self.mesh.lx ** 3
        Gh = host(G).reshape(self.mesh.E, 6, lx3).transpose(1, 0, 2).reshape(6, -1)
        return Gh, host(B)

    def jacobi(self):
        t = torch()
        m = t.empty(self.n, dtype=t.float64, device="cuda")
        S.sem_get_jacobi(self.h, m)
        t.cuda.synchronize()
        return host(m)

    def solve(self, b, x0=None, on_host=False, **opts):
        t = torch()
        if on_host:
            bd = t.from_numpy(np.ascontiguousarray(b, dtype=np.float64))
            xd = t.zeros(self.n, dtype=t.float64) if x0 is None else t.from_numpy(np.array(x0, dtype=np.float64))
        else:
            bd = dev(b, t.float64)
            xd = t.zeros(self.n, dtype=t.float64, device="cuda") if x0 is None else dev(x0, t.float64)
        st = S.sem_cg_solve(self.h, xd, bd, opts)
        t.cuda.synchronize()
        return (xd.numpy().copy() if on_host else host(xd)), st


def rel_err(a, ref):
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = a - ref
    n2 = np.linalg.norm(ref)
    ninf = np.max(np.abs(ref)) if ref.size else 0.0
    return (np.linalg.norm(d) / n2 if n2 > 0 else np.linalg.norm(d),
            np.max(np.abs(d)) / ninf if ninf > 0 else (np.max(np.abs(d)) if d.size else 0.0))
