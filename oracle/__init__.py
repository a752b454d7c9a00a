"""FP64 CPU oracle for IRN-PICCS (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` and
reference legs of ``bench.py`` may import this package.  It wraps the plain C
library ``piccs_oracle.c`` (compiled with gcc + OpenMP into ``oracle/_build``)
and shares no code with the CUDA library.  Every function is pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "piccs_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

PICCS, PIPLE, TV, CGLS = 0, 1, 2, 3
RULE_R1, RULE_R2 = 0, 1
SOLVER_CGLS, SOLVER_LSQR, SOLVER_LSQR_REORTH = 0, 1, 2


class _Geom(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("vx", C.c_double), ("vy", C.c_double), ("vz", C.c_double),
                ("nu", C.c_int), ("nv", C.c_int),
                ("du", C.c_double), ("dv", C.c_double),
                ("dso", C.c_double), ("dsd", C.c_double),
                ("n_views", C.c_int), ("angles", C.POINTER(C.c_double)),
                ("layout", C.c_int), ("u_offset", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp); returns the .so path."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER
            d, ll, i = C.c_double, C.c_longlong, C.c_int
            pd = P(d)
            pg = P(_Geom)
            lib.og_check.argtypes = [pg]
            lib.og_forward.argtypes = [pg, pd, pd, i]
            lib.og_forward_rays.argtypes = [pg, pd, P(ll), ll, pd, i]
            lib.og_count_nnz.argtypes = [pg, i]
            lib.og_count_nnz.restype = ll
            lib.og_adjoint.argtypes = [pg, pd, pd, i]
            lib.og_adjoint_voxels.argtypes = [pg, pd, P(ll), ll, pd, i]
            lib.og_clip_ray_voxel.argtypes = [pg, ll, ll]
            lib.og_clip_ray_voxel.restype = d
            lib.og_grad.argtypes = [i, i, i, pd, pd]
            lib.og_grad_adj.argtypes = [i, i, i, pd, pd]
            lib.og_weights.argtypes = [ll, pd, d, i, pd]
            lib.og_cgls_fixed.argtypes = [pg, pd, pd, pd, pd, d, d, i, pd, i, pd, i]
            lib.og_lsqr_fixed.argtypes = [pg, pd, pd, pd, pd, d, d, i, pd, i, i, pd, pd, i]
            lib.og_irn.argtypes = [pg, pd, pd, pd, d, d, d, i, i, i, i, i, pd, pd, i]
            _lib = lib
    return _lib


def _pd(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class _GeomHandle:
    def __init__(self, g):
        self.angles = _f64(g.angles)
        self.s = _Geom(g.nx, g.ny, g.nz, g.vx, g.vy, g.vz, g.nu, g.nv, g.du, g.dv,
                       g.dso, g.dsd, self.angles.shape[0], _pd(self.angles), g.layout,
                       float(getattr(g, "u_offset", 0.0)))

    @property
    def ref(self):
        return C.byref(self.s)


def check(g) -> bool:
    return _load().og_check(_GeomHandle(g).ref) == 0


def forward(g, x, nthreads: int = 0) -> np.ndarray:
    """A x in FP64 (Siddon), shaped like g.proj_shape()."""
    lib = _load()
    x = _f64(x).reshape(-1)
    assert x.size == g.M
    y = np.zeros(g.N, dtype=np.float64)
    lib.og_forward(_GeomHandle(g).ref, _pd(x), _pd(y), nthreads)
    return y.reshape(g.proj_shape())


def forward_rays(g, x, rays, nthreads: int = 0) -> np.ndarray:
    lib = _load()
    x = _f64(x).reshape(-1)
    r = np.ascontiguousarray(np.asarray(rays, dtype=np.int64))
    out = np.zeros(r.size, dtype=np.float64)
    lib.og_forward_rays(_GeomHandle(g).ref, _pd(x), r.ctypes.data_as(C.POINTER(C.c_longlong)),
                        r.size, _pd(out), nthreads)
    return out


def count_nnz(g, nthreads: int = 0) -> int:
    return int(_load().og_count_nnz(_GeomHandle(g).ref, nthreads))


def adjoint(g, y, nthreads: int = 0) -> np.ndarray:
    """A^T y in FP64, shaped (nx, ny, nz)."""
    lib = _load()
    y = _f64(y).reshape(-1)
    assert y.size == g.N
    x = np.zeros(g.M, dtype=np.float64)
    lib.og_adjoint(_GeomHandle(g).ref, _pd(y), _pd(x), nthreads)
    return x.reshape(g.vol_shape())


def adjoint_voxels(g, y, voxels, nthreads: int = 0) -> np.ndarray:
    """(A^T y) at the listed flat voxel indices, by per-voxel ray clipping."""
    lib = _load()
    y = _f64(y).reshape(-1)
    v = np.ascontiguousarray(np.asarray(voxels, dtype=np.int64))
    out = np.zeros(v.size, dtype=np.float64)
    lib.og_adjoint_voxels(_GeomHandle(g).ref, _pd(y), v.ctypes.data_as(C.POINTER(C.c_longlong)),
                          v.size, _pd(out), nthreads)
    return out


def clip_ray_voxel(g, ray: int, voxel: int) -> float:
    return float(_load().og_clip_ray_voxel(_GeomHandle(g).ref, int(ray), int(voxel)))


def grad(z) -> np.ndarray:
    """D z stacked as (3, nx, ny, nz)."""
    z = _f64(z)
    nx, ny, nz = z.shape
    g = np.zeros((3,) + z.shape, dtype=np.float64)
    _load().og_grad(nx, ny, nz, _pd(z), _pd(g))
    return g


def grad_adj(f) -> np.ndarray:
    """D^T f for f shaped (3, nx, ny, nz)."""
    f = _f64(f)
    _, nx, ny, nz = f.shape
    out = np.zeros((nx, ny, nz), dtype=np.float64)
    _load().og_grad_adj(nx, ny, nz, _pd(f), _pd(out))
    return out


def weights(g3, tau: float, rule: int = RULE_R1) -> np.ndarray:
    """IRN weight per voxel from a stacked gradient (3, nx, ny, nz)."""
    g3 = _f64(g3)
    M = g3[0].size
    w = np.zeros(g3.shape[1:], dtype=np.float64)
    _load().og_weights(M, _pd(g3), tau, rule, _pd(w))
    return w


def cgls_fixed(g, b, xp, w1, w2, alpha, lam, variant, x0, iters, nthreads: int = 0):
    """CGLS on the augmented system with fixed weights; returns (x, residuals)."""
    lib = _load()
    x = _f64(x0).reshape(-1).copy()
    b = _f64(b).reshape(-1)
    xp = _f64(xp).reshape(-1)
    w1 = _f64(w1).reshape(-1)
    w2 = _f64(w2).reshape(-1)
    res = np.full(iters + 1, np.nan)
    n = lib.og_cgls_fixed(_GeomHandle(g).ref, _pd(b), _pd(xp), _pd(w1), _pd(w2),
                          alpha, lam, variant, _pd(x), iters, _pd(res), nthreads)
    if n < 0:
        raise ValueError("invalid geometry")
    return x.reshape(g.vol_shape()), res[:n + 1]


def lsqr_fixed(g, b, xp, w1, w2, alpha, lam, variant, x0, iters, reorth: bool = False,
               nthreads: int = 0, return_basis: bool = False):
    """LSQR on the augmented system with fixed weights; returns (x, residuals)
    and, with return_basis, the bidiagonalisation's v vectors (rows).
    reorth: re-orthogonalise every new v against all earlier ones."""
    lib = _load()
    x = _f64(x0).reshape(-1).copy()
    b = _f64(b).reshape(-1)
    xp = _f64(xp).reshape(-1)
    w1 = _f64(w1).reshape(-1)
    w2 = _f64(w2).reshape(-1)
    res = np.full(iters + 1, np.nan)
    V = np.zeros((iters + 1, g.M)) if return_basis else None
    n = lib.og_lsqr_fixed(_GeomHandle(g).ref, _pd(b), _pd(xp), _pd(w1), _pd(w2),
                          alpha, lam, variant, _pd(x), iters, int(bool(reorth)), _pd(res),
                          _pd(V) if V is not None else None, nthreads)
    if n < 0:
        raise ValueError("invalid geometry")
    if return_basis:
        return x.reshape(g.vol_shape()), res[:n + 1], V[:n + 1]
    return x.reshape(g.vol_shape()), res[:n + 1]


def irn(g, b, xp, x0, alpha, lam, tau, n_outer, n_inner, variant=PICCS, rule=RULE_R1,
        nthreads: int = 0, solver: int = SOLVER_CGLS):
    """IRN outer loop with CGLS (or LSQR) inner solves; returns (x, residual
    history, last weights (w1, w2))."""
    lib = _load()
    x = _f64(x0).reshape(-1).copy()
    b = _f64(b).reshape(-1)
    xp = _f64(xp).reshape(-1)
    res = np.full(n_outer * (n_inner + 1), np.nan)
    w = np.zeros(2 * g.M)
    rc = lib.og_irn(_GeomHandle(g).ref, _pd(b), _pd(xp), _pd(x), alpha, lam, tau, rule,
                    variant, n_outer, n_inner, int(solver), _pd(res), _pd(w), nthreads)
    if rc != 0:
        raise ValueError("invalid geometry")
    return (x.reshape(g.vol_shape()), res.reshape(n_outer, n_inner + 1),
            (w[:g.M].reshape(g.vol_shape()), w[g.M:].reshape(g.vol_shape())))
