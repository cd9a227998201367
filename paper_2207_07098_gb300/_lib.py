"""ctypes binding of libsem (include/sem.h): argument marshalling only.

Every entry point keeps the C name and argument order.  Device buffers are
passed as torch tensors (their data_ptr()), set-up arrays as numpy arrays,
streams as torch.cuda.Stream (default: the current stream).  The library must
have been built (``__graft_entry__.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsem.so")

SEM_OK, SEM_EINVAL, SEM_ENOMEM, SEM_ECUDA, SEM_ENOTCONV, SEM_EBREAKDOWN, SEM_ESTAGNATE, SEM_ETIMEOUT = range(8)
SEM_FP64, SEM_FP32, SEM_FP64_NATIVE, SEM_FP64_PAIR, SEM_TC_SPLIT = 0, 1, 2, 3, 4
SEM_MODE_FP64, SEM_MODE_MIXED_IR, SEM_MODE_GMRES = 0, 1, 2


SEM_FLAG_TEST_STALL = 0x100
SEM_FLAG_METRICS = 0x200
SEM_FLAG_SCHWARZ = 0x400


def SEM_FLAG_VARIANT(v: int) -> int:
    """Set-up flag pinning operator kernel variant v, as in sem.h: 0..4 for
    SEM_FP64 and SEM_FP32, 5 or 6 for SEM_FP64_PAIR, 8 for SEM_FP32, 9 for
    SEM_FP64."""
    return (v + 1) & 0xF
STATUS_NAMES = {0: "SEM_OK", 1: "SEM_EINVAL", 2: "SEM_ENOMEM", 3: "SEM_ECUDA", 4: "SEM_ENOTCONV",
                5: "SEM_EBREAKDOWN", 6: "SEM_ESTAGNATE", 7: "SEM_ETIMEOUT"}


class SemError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class sem_info(ctypes.Structure):
    _fields_ = [("nsolve", ctypes.c_int), ("E", ctypes.c_int), ("lx", ctypes.c_int),
                ("n_local", ctypes.c_int64), ("n_unique", ctypes.c_int64), ("n_free", ctypes.c_int64),
                ("n_shared", ctypes.c_int64), ("device_bytes", ctypes.c_size_t)]


class sem_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("mode", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int), ("precision", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("graph_chunk", ctypes.c_int), ("autotune", ctypes.c_int),
                ("ir_carry", ctypes.c_int), ("persistent", ctypes.c_int), ("tc_split", ctypes.c_int),
                ("gmres_restart", ctypes.c_int), ("pipelined", ctypes.c_int), ("projection", ctypes.c_int),
                ("precond_precision", ctypes.c_int), ("gmres_orth", ctypes.c_int)]


class sem_solve_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("outer_iterations", ctypes.c_int),
                ("relres", ctypes.c_double), ("relres_recursive", ctypes.c_double), ("time_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("ax_ms", ctypes.c_double), ("ax_samples", ctypes.c_int),
                ("ax_variant", ctypes.c_int), ("relres_start", ctypes.c_double),
                ("launches_per_iteration", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class sem_mesh_desc(ctypes.Structure):
    _fields_ = [("E", ctypes.c_int), ("lx", ctypes.c_int), ("coords", ctypes.c_void_p),
                ("gid", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("h1", ctypes.c_void_p)]


_lib = None

_VP = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "sem_solve_opts_default": (None, [ctypes.POINTER(sem_solve_opts)]),
    "sem_last_error": (ctypes.c_char_p, []),
    "sem_gll": (_I, [_I, _VP, _VP, _VP]),
    "sem_setup": (_I, [ctypes.POINTER(_VP), _I, _I, _VP, _VP, _VP, _VP, _I, _VP]),
    "sem_setup_batch": (_I, [ctypes.POINTER(_VP), _I, ctypes.POINTER(sem_mesh_desc), _I, _VP]),
    "sem_destroy": (_I, [_VP]),
    "sem_get_info": (_I, [_VP, ctypes.POINTER(sem_info)]),
    "sem_get_offsets": (_I, [_VP, _VP]),
    "sem_set_helmholtz": (_I, [_VP, _VP, _VP]),
    "sem_ax": (_I, [_VP, _VP, _VP, _I, _I, _VP]),
    "sem_gs": (_I, [_VP, _VP, _I, _I, _VP]),
    "sem_mass": (_I, [_VP, _VP, _VP, _I, _I, _VP]),
    "sem_dot": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "sem_dot_noalloc": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "sem_get_geometry": (_I, [_VP, _VP, _VP, _VP]),
    "sem_get_jacobi": (_I, [_VP, _VP, _VP]),
    "sem_cg_solve": (_I, [_VP, _VP, _VP, ctypes.POINTER(sem_solve_opts), ctypes.POINTER(sem_solve_stats), _VP]),
    "sem_cg_solve_batch": (_I, [_VP, _VP, _VP, ctypes.POINTER(sem_solve_opts), _VP, _VP]),
    "sem_grad": (_I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "sem_div": (_I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "sem_curl": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "sem_pressure_rhs": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_double, _VP, _VP]),
    "sem_schwarz_apply": (_I, [_VP, _VP, _VP, _VP]),
    "sem_schwarz_apply32": (_I, [_VP, _VP, _VP, _VP]),
    "sem_projection_reset": (_I, [_VP]),
    "sem_projection_size": (_I, [_VP, ctypes.POINTER(_I)]),
}


def load(path: str = LIB_PATH):
    """Load libsem.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def _check(rc: int, allowed=(SEM_OK,)):
    if rc not in allowed:
        msg = load().sem_last_error()
        raise SemError(rc, msg.decode() if msg else "")
    return rc


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# entry points (same names and argument order as include/sem.h)
# ---------------------------------------------------------------------------

def sem_solve_opts_default() -> sem_solve_opts:
    o = sem_solve_opts()
    load().sem_solve_opts_default(ctypes.byref(o))
    return o


def sem_last_error() -> str:
    m = load().sem_last_error()
    return m.decode() if m else ""


def sem_gll(lx: int):
    xi = np.zeros(lx)
    rho = np.zeros(lx)
    D = np.zeros((lx, lx))
    _check(load().sem_gll(lx, _ptr(xi), _ptr(rho), _ptr(D)))
    return xi, rho, D


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def sem_setup(E: int, lx: int, coords, gid, mask, h1=None, flags: int = 0, stream=None):
    """Returns an opaque handle (int).  coords/gid/mask/h1: host arrays."""
    c = _host(coords, np.float64)
    g = _host(gid, np.int64)
    m = _host(mask, np.uint8)
    hh = None if h1 is None else _host(h1, np.float64)
    out = ctypes.c_void_p()
    _check(load().sem_setup(ctypes.byref(out), E, lx, _ptr(c), _ptr(g), _ptr(m), _ptr(hh), flags, _stream(stream)))
    return out.value


def sem_setup_batch(meshes, flags: int = 0, stream=None):
    """meshes: sequence of (E, lx, coords, gid, mask, h1-or-None) host arrays."""
    keep = []
    descs = (sem_mesh_desc * len(meshes))()
    for q, (E, lx, coords, gid, mask, h1) in enumerate(meshes):
        arrs = (_host(coords, np.float64), _host(gid, np.int64), _host(mask, np.uint8),
                None if h1 is None else _host(h1, np.float64))
        keep.append(arrs)
        descs[q].E, descs[q].lx = E, lx
        descs[q].coords = arrs[0].ctypes.data
        descs[q].gid = arrs[1].ctypes.data
        descs[q].mask = arrs[2].ctypes.data
        descs[q].h1 = None if arrs[3] is None else arrs[3].ctypes.data
    out = ctypes.c_void_p()
    _check(load().sem_setup_batch(ctypes.byref(out), len(meshes), descs, flags, _stream(stream)))
    return out.value


def sem_destroy(h) -> None:
    if h:
        _check(load().sem_destroy(ctypes.c_void_p(h)))


def sem_get_info(h) -> dict:
    info = sem_info()
    _check(load().sem_get_info(ctypes.c_void_p(h), ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in info._fields_}


def sem_get_offsets(h, nsolve: int) -> np.ndarray:
    off = np.zeros(nsolve + 1, dtype=np.int64)
    _check(load().sem_get_offsets(ctypes.c_void_p(h), _ptr(off)))
    return off


def sem_set_helmholtz(h, h2=None, stream=None) -> None:
    """h2: host array [n_local] (mass coefficient) or None for Poisson."""
    hh = None if h2 is None else _host(h2, np.float64)
    _check(load().sem_set_helmholtz(ctypes.c_void_p(h), _ptr(hh), _stream(stream)))


def sem_ax(h, w, u, precision: int = SEM_FP64, assemble: int = 1, stream=None) -> None:
    _check(load().sem_ax(ctypes.c_void_p(h), _ptr(w), _ptr(u), precision, assemble, _stream(stream)))


def sem_gs(h, u, precision: int = SEM_FP64, apply_mask: int = 1, stream=None) -> None:
    _check(load().sem_gs(ctypes.c_void_p(h), _ptr(u), precision, apply_mask, _stream(stream)))


def sem_mass(h, w, u, precision: int = SEM_FP64, assemble: int = 1, stream=None) -> None:
    _check(load().sem_mass(ctypes.c_void_p(h), _ptr(w), _ptr(u), precision, assemble, _stream(stream)))


def sem_dot(h, a, b, result, stream=None) -> None:
    _check(load().sem_dot(ctypes.c_void_p(h), _ptr(a), _ptr(b), _ptr(result), _stream(stream)))


def sem_dot_noalloc(h, a, b, result, stream=None) -> None:
    """Like sem_dot, with the scratch in a fixed device array of the library
    (no allocation; see include/sem.h for the limit and the sharing rules)."""
    _check(load().sem_dot_noalloc(ctypes.c_void_p(h), _ptr(a), _ptr(b), _ptr(result), _stream(stream)))


def sem_get_geometry(h, G=None, B=None, stream=None) -> None:
    _check(load().sem_get_geometry(ctypes.c_void_p(h), _ptr(G), _ptr(B), _stream(stream)))


def sem_get_jacobi(h, minv, stream=None) -> None:
    _check(load().sem_get_jacobi(ctypes.c_void_p(h), _ptr(minv), _stream(stream)))


_SOLVE_OK = (SEM_OK, SEM_ENOTCONV, SEM_EBREAKDOWN, SEM_ESTAGNATE)


def _opts(opts):
    o = sem_solve_opts_default()
    if opts:
        for k, v in opts.items():
            setattr(o, k, v)
    return o


def sem_cg_solve(h, x, b, opts: dict | None = None, stream=None) -> dict:
    """x (in: guess, out: solution) and b: torch tensors on the host or device.
    Returns the sem_solve_stats fields as a dict (status included)."""
    o = _opts(opts)
    st = sem_solve_stats()
    _check(load().sem_cg_solve(ctypes.c_void_p(h), _ptr(x), _ptr(b), ctypes.byref(o), ctypes.byref(st),
                               _stream(stream)), _SOLVE_OK)
    return st.as_dict()


def sem_cg_solve_batch(h, x, b, nsolve: int, opts: dict | None = None, stream=None) -> list[dict]:
    o = _opts(opts)
    st = (sem_solve_stats * nsolve)()
    _check(load().sem_cg_solve_batch(ctypes.c_void_p(h), _ptr(x), _ptr(b), ctypes.byref(o),
                                     ctypes.cast(st, ctypes.c_void_p), _stream(stream)), _SOLVE_OK)
    return [st[q].as_dict() for q in range(nsolve)]


def sem_projection_reset(h) -> None:
    _check(load().sem_projection_reset(ctypes.c_void_p(h)))


def sem_projection_size(h) -> int:
    c = ctypes.c_int(0)
    _check(load().sem_projection_size(ctypes.c_void_p(h), ctypes.byref(c)))
    return c.value


def sem_grad(h, u, gx, gy, gz, stream=None) -> None:
    _check(load().sem_grad(ctypes.c_void_p(h), _ptr(u), _ptr(gx), _ptr(gy), _ptr(gz), _stream(stream)))


def sem_div(h, vx, vy, vz, out, stream=None) -> None:
    _check(load().sem_div(ctypes.c_void_p(h), _ptr(vx), _ptr(vy), _ptr(vz), _ptr(out), _stream(stream)))


def sem_curl(h, vx, vy, vz, cx, cy, cz, stream=None) -> None:
    _check(load().sem_curl(ctypes.c_void_p(h), _ptr(vx), _ptr(vy), _ptr(vz), _ptr(cx), _ptr(cy), _ptr(cz),
                           _stream(stream)))


def sem_pressure_rhs(h, vx, vy, vz, wx, wy, wz, dt: float, Re: float, b, stream=None) -> None:
    _check(load().sem_pressure_rhs(ctypes.c_void_p(h), _ptr(vx), _ptr(vy), _ptr(vz), _ptr(wx), _ptr(wy), _ptr(wz),
                                   dt, Re, _ptr(b), _stream(stream)))


def sem_schwarz_apply(h, r, z, stream=None) -> None:
    _check(load().sem_schwarz_apply(ctypes.c_void_p(h), _ptr(r), _ptr(z), _stream(stream)))


def sem_schwarz_apply32(h, r, z, stream=None) -> None:
    _check(load().sem_schwarz_apply32(ctypes.c_void_p(h), _ptr(r), _ptr(z), _stream(stream)))
