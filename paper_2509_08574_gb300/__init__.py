"""Python binding of libpiccs (GB300 / sm_103a IRN-PICCS cone-beam CT).

Thin ctypes marshalling over the C ABI of ``include/piccs.h``: the functions
keep the C names, take torch CUDA tensors (or raw device pointers) and raise
:class:`PiccsError` on a negative status.  Every step of the reconstruction
runs in the library's CUDA kernels; there is no Python or CPU fallback, and
importing this package fails if ``_lib/libpiccs.so`` has not been built
(``python paper_2509_08574_gb300/build.py``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpiccs.so")

PICCS_OK = 0
PICCS_EINVAL = -1
PICCS_ENOMEM = -2
PICCS_ENONFINITE = -3
PICCS_EBREAKDOWN = -4
PICCS_ETIMEOUT = -5
PICCS_ECUDA = -6
PICCS_ENOTIMPL = -7

LAYOUT_UV, LAYOUT_VU = 0, 1
VARIANT_PICCS, VARIANT_PIPLE, VARIANT_TV, VARIANT_CGLS = 0, 1, 2, 3
WEIGHT_R1, WEIGHT_R2 = 0, 1
X0_PRIOR, X0_ZERO, X0_USER = 0, 1, 2
SOLVER_CGLS, SOLVER_LSQR, SOLVER_LSQR_REORTH = 0, 1, 2
STORAGE_F32, STORAGE_BF16 = 0, 1
ORDER_RESPONSE_RATIO, ORDER_FIFO, ORDER_ADAPTIVE = 0, 1, 2

_NAMES = {0: "PICCS_OK", -1: "PICCS_EINVAL", -2: "PICCS_ENOMEM", -3: "PICCS_ENONFINITE",
          -4: "PICCS_EBREAKDOWN", -5: "PICCS_ETIMEOUT", -6: "PICCS_ECUDA", -7: "PICCS_ENOTIMPL"}


class PiccsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class piccs_geometry(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("vx", C.c_double), ("vy", C.c_double), ("vz", C.c_double),
                ("nu", C.c_int), ("nv", C.c_int),
                ("du", C.c_double), ("dv", C.c_double),
                ("dso", C.c_double), ("dsd", C.c_double),
                ("n_views", C.c_int), ("angles_rad", C.POINTER(C.c_double)),
                ("proj_layout", C.c_int), ("u_offset", C.c_double)]


class piccs_params(C.Structure):
    _fields_ = [("alpha", C.c_float), ("lambda_", C.c_float), ("tau", C.c_float),
                ("n_outer", C.c_int), ("n_inner", C.c_int), ("x0_mode", C.c_int),
                ("variant", C.c_int), ("weight_rule", C.c_int), ("solver", C.c_int),
                ("storage", C.c_int)]


class piccs_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations_run", C.c_int), ("n_history", C.c_int),
                ("gamma_history", C.c_double * 512)]


class piccs_server_config(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_batch", C.c_int), ("max_running", C.c_int),
                ("use_graphs", C.c_int), ("order", C.c_int), ("max_group", C.c_int)]


class piccs_request_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("batch", C.c_int), ("queued_ms", C.c_double),
                ("run_ms", C.c_double), ("total_ms", C.c_double)]


class piccs_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("completed", C.c_longlong), ("failed", C.c_longlong),
                ("batches", C.c_longlong), ("graph_replays", C.c_longlong),
                ("sessions_made", C.c_longlong), ("evictions", C.c_longlong),
                ("hbm_in_use", C.c_size_t), ("group_runs", C.c_longlong)]


KERNEL_CLASSES = ("forward", "adjoint", "reg", "vector", "scalar")


class piccs_profile(C.Structure):
    _fields_ = [("launches", C.c_longlong * 5), ("total_ms", C.c_double * 5),
                ("total_launches", C.c_longlong), ("calls", C.c_longlong * 5)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libpiccs is not built ({LIB_PATH} missing); run "
                          "`python paper_2509_08574_gb300/build.py` (needs nvcc)")
    lib = C.CDLL(LIB_PATH)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    G, P, R = C.POINTER(piccs_geometry), C.POINTER(piccs_params), C.POINTER(piccs_stats)
    sig = {
        "piccs_create": (i, [C.POINTER(vp), G, vp]),
        "piccs_create_batched": (i, [C.POINTER(vp), G, i, vp]),
        "piccs_query_workspace_batched": (i, [G, P, i, C.POINTER(C.c_size_t)]),
        "piccs_report_slot": (i, [vp, i, R]),
        "piccs_set_prior_broadcast": (i, [vp, vp, i]),
        "piccs_stage": (i, [vp, i, vp, i]),
        "piccs_stage_bf16": (i, [vp, i, vp, i]),
        "piccs_run_staged": (i, [vp, i, P, i]),
        "piccs_run_staged_group": (i, [C.POINTER(vp), C.POINTER(i), i, P, i]),
        "piccs_unstage": (i, [vp, i, vp, i]),
        "piccs_server_create": (i, [C.POINTER(vp), C.POINTER(piccs_server_config)]),
        "piccs_server_destroy": (None, [vp]),
        "piccs_server_last_error": (C.c_char_p, [vp]),
        "piccs_server_add_patient": (i, [vp, i, G, vp]),
        "piccs_server_submit": (i, [vp, i, vp, P, vp, C.POINTER(C.c_longlong)]),
        "piccs_server_wait": (i, [vp, C.c_longlong, i, C.POINTER(piccs_request_stats)]),
        "piccs_server_get_stats": (i, [vp, C.POINTER(piccs_server_stats)]),
        "piccs_destroy": (None, [vp]),
        "piccs_last_error": (C.c_char_p, [vp]),
        "piccs_set_stream": (i, [vp, vp]),
        "piccs_query_workspace": (i, [G, P, C.POINTER(C.c_size_t)]),
        "piccs_validate": (i, [G, P]),
        "piccs_set_prior": (i, [vp, vp]),
        "piccs_reconstruct": (i, [vp, vp, P, vp, vp]),
        "piccs_reconstruct_host": (i, [vp, vp, P, vp, vp]),
        "piccs_report": (i, [vp, R]),
        "piccs_forward": (i, [vp, vp, vp]),
        "piccs_adjoint": (i, [vp, vp, vp]),
        "piccs_reg_weights": (i, [vp, vp, P, vp, vp]),
        "piccs_reg_normal": (i, [vp, vp, P, vp, vp, C.POINTER(d)]),
        "piccs_profile_enable": (i, [vp, i]),
        "piccs_profile_read": (i, [vp, C.POINTER(piccs_profile)]),
        "piccs_reg_normal_noalloc": (i, [i, i, i, vp, C.c_float, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
EXPORTED = ("piccs_create", "piccs_destroy", "piccs_last_error", "piccs_set_stream",
            "piccs_query_workspace", "piccs_validate", "piccs_set_prior", "piccs_reconstruct",
            "piccs_reconstruct_host", "piccs_report", "piccs_forward", "piccs_adjoint",
            "piccs_reg_weights", "piccs_reg_normal", "piccs_profile_enable",
            "piccs_profile_read", "piccs_reg_normal_noalloc", "piccs_create_batched",
            "piccs_query_workspace_batched", "piccs_report_slot", "piccs_set_prior_broadcast",
            "piccs_stage", "piccs_stage_bf16", "piccs_run_staged", "piccs_run_staged_group", "piccs_unstage",
            "piccs_server_create",
            "piccs_server_destroy", "piccs_server_last_error", "piccs_server_add_patient",
            "piccs_server_submit", "piccs_server_wait", "piccs_server_get_stats")


def library():
    """The loaded ctypes.CDLL (for callers that marshal arguments themselves)."""
    return _lib


# --------------------------------------------------------------------------
# marshalling helpers
# --------------------------------------------------------------------------
def _ptr(t, n=None, what="buffer"):
    """Device (or host) pointer of a tensor / int; checks float32 contiguity."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        if t.dtype.__repr__() != "torch.float32":
            raise TypeError(f"{what} must be float32, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{what} must be contiguous")
        if n is not None and t.numel() != n:
            raise ValueError(f"{what} must hold {n} elements, got {t.numel()}")
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        if t.dtype != np.float32 or not t.flags.c_contiguous:
            raise TypeError(f"{what} must be a contiguous float32 array")
        if n is not None and t.size != n:
            raise ValueError(f"{what} must hold {n} elements, got {t.size}")
        return t.ctypes.data
    raise TypeError(f"{what}: unsupported type {type(t)}")


def _ptr16(t, n, what="buffer"):
    """Pointer of a contiguous BF16 buffer (torch.bfloat16 / int16 tensor or
    uint16 numpy array of bit patterns) of n elements."""
    if hasattr(t, "data_ptr"):
        if str(t.dtype) not in ("torch.bfloat16", "torch.int16", "torch.uint16"):
            raise TypeError(f"{what} must be bfloat16, got {t.dtype}")
        if not t.is_contiguous() or t.numel() != n:
            raise ValueError(f"{what} must be contiguous with {n} elements")
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        if t.dtype not in (np.uint16, np.int16) or not t.flags.c_contiguous or t.size != n:
            raise TypeError(f"{what} must be a contiguous uint16 array of {n} elements")
        return t.ctypes.data
    raise TypeError(f"{what}: unsupported type {type(t)}")


def _check(rc, ctx=None):
    if rc != PICCS_OK:
        msg = _lib.piccs_last_error(ctx)
        raise PiccsError(rc, msg.decode() if msg else "")


def make_geometry(g):
    """piccs_geometry from any object with nx, ny, nz, vx, vy, vz, nu, nv, du,
    dv, dso, dsd, angles (radians), layout and (optionally) u_offset
    attributes.  The returned structure keeps the angle array alive."""
    ang = np.ascontiguousarray(np.asarray(g.angles, dtype=np.float64))
    s = piccs_geometry(int(g.nx), int(g.ny), int(g.nz), float(g.vx), float(g.vy), float(g.vz),
                       int(g.nu), int(g.nv), float(g.du), float(g.dv), float(g.dso),
                       float(g.dsd), int(ang.shape[0]),
                       ang.ctypes.data_as(C.POINTER(C.c_double)), int(getattr(g, "layout", 0)),
                       float(getattr(g, "u_offset", 0.0)))
    s._angles = ang
    return s


def make_params(alpha=0.5, lam=0.5, tau=1e-2, n_outer=1, n_inner=10, x0_mode=X0_PRIOR,
                variant=VARIANT_PICCS, weight_rule=WEIGHT_R1, solver=SOLVER_CGLS,
                storage=STORAGE_F32):
    return piccs_params(alpha, lam, tau, n_outer, n_inner, x0_mode, variant, weight_rule, solver,
                        storage)


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# --------------------------------------------------------------------------
# the C ABI, one Python function per entry point
# --------------------------------------------------------------------------
def piccs_validate(geometry, params=None):
    gs = geometry if isinstance(geometry, piccs_geometry) else make_geometry(geometry)
    _check(_lib.piccs_validate(C.byref(gs), C.byref(params) if params is not None else None))


def piccs_query_workspace(geometry, params=None) -> int:
    gs = geometry if isinstance(geometry, piccs_geometry) else make_geometry(geometry)
    out = C.c_size_t(0)
    _check(_lib.piccs_query_workspace(C.byref(gs), C.byref(params) if params is not None else None,
                                      C.byref(out)))
    return int(out.value)


def piccs_create(geometry, stream=None) -> int:
    gs = geometry if isinstance(geometry, piccs_geometry) else make_geometry(geometry)
    h = C.c_void_p()
    _check(_lib.piccs_create(C.byref(h), C.byref(gs), _stream_handle(stream)))
    return h.value


def piccs_create_batched(geometry, batch, stream=None) -> int:
    gs = geometry if isinstance(geometry, piccs_geometry) else make_geometry(geometry)
    h = C.c_void_p()
    _check(_lib.piccs_create_batched(C.byref(h), C.byref(gs), int(batch), _stream_handle(stream)))
    return h.value


def piccs_query_workspace_batched(geometry, params, batch) -> int:
    gs = geometry if isinstance(geometry, piccs_geometry) else make_geometry(geometry)
    out = C.c_size_t(0)
    _check(_lib.piccs_query_workspace_batched(C.byref(gs), C.byref(params) if params is not None
                                              else None, int(batch), C.byref(out)))
    return int(out.value)


def piccs_destroy(ctx):
    _lib.piccs_destroy(ctx)


def piccs_last_error(ctx=None) -> str:
    m = _lib.piccs_last_error(ctx)
    return m.decode() if m else ""


def piccs_set_stream(ctx, stream):
    _check(_lib.piccs_set_stream(ctx, _stream_handle(stream)), ctx)


def piccs_set_prior(ctx, d_xprior):
    _check(_lib.piccs_set_prior(ctx, _ptr(d_xprior, what="prior")), ctx)


def piccs_reconstruct(ctx, d_proj, params, d_x0, d_vol_out):
    _check(_lib.piccs_reconstruct(ctx, _ptr(d_proj, what="projections"), C.byref(params),
                                  _ptr(d_x0, what="x0"), _ptr(d_vol_out, what="volume")), ctx)


def piccs_reconstruct_host(ctx, h_proj, params, h_x0, h_vol_out):
    _check(_lib.piccs_reconstruct_host(ctx, _ptr(h_proj, what="projections"), C.byref(params),
                                       _ptr(h_x0, what="x0"), _ptr(h_vol_out, what="volume")), ctx)


def piccs_report(ctx) -> piccs_stats:
    rep = piccs_stats()
    _check(_lib.piccs_report(ctx, C.byref(rep)), ctx)
    return rep


def piccs_report_slot(ctx, slot) -> piccs_stats:
    rep = piccs_stats()
    _check(_lib.piccs_report_slot(ctx, int(slot), C.byref(rep)), ctx)
    return rep


def piccs_forward(ctx, d_vol, d_proj):
    _check(_lib.piccs_forward(ctx, _ptr(d_vol, what="volume"), _ptr(d_proj, what="projections")), ctx)


def piccs_adjoint(ctx, d_proj, d_vol):
    _check(_lib.piccs_adjoint(ctx, _ptr(d_proj, what="projections"), _ptr(d_vol, what="volume")), ctx)


def piccs_reg_weights(ctx, d_x, params, d_omega, d_c):
    _check(_lib.piccs_reg_weights(ctx, _ptr(d_x, what="x"), C.byref(params), _ptr(d_omega, what="omega"),
                                  _ptr(d_c, what="c")), ctx)


def piccs_reg_normal(ctx, d_omega, params, d_z, d_out, want_rho=True):
    rho = C.c_double(0.0)
    _check(_lib.piccs_reg_normal(ctx, _ptr(d_omega, what="omega"), C.byref(params), _ptr(d_z, what="z"),
                                 _ptr(d_out, what="out"), C.byref(rho) if want_rho else None), ctx)
    return float(rho.value) if want_rho else None


def piccs_reg_normal_noalloc(nx, ny, nz, d_omega, lambda2_piple, d_z, d_out, d_rho,
                             stream=None):
    """Context-free, allocation-free D^T diag(omega) D z (+ lambda2_piple z) and
    its energy, for callers that cannot allocate device memory; d_rho is a
    device buffer of one float64.  See include/piccs.h."""
    n = int(nx) * int(ny) * int(nz)
    if hasattr(d_rho, "data_ptr"):
        if str(d_rho.dtype) != "torch.float64" or d_rho.numel() < 1:
            raise TypeError("d_rho must be a float64 device tensor")
        rho_ptr = d_rho.data_ptr()
    else:
        rho_ptr = d_rho
    _check(_lib.piccs_reg_normal_noalloc(int(nx), int(ny), int(nz), _ptr(d_omega, n, "omega"),
                                         float(lambda2_piple), _ptr(d_z, n, "z"),
                                         _ptr(d_out, n, "out"), rho_ptr, _stream_handle(stream)))


def run_staged_group(contexts, nactive, params, graph=True):
    """Staged reconstructions of several contexts (different geometries) run
    together: every projector product one launch for all of them
    (piccs_run_staged_group).  contexts: Context objects; nactive: staged
    slots per context."""
    n = len(contexts)
    hs = (C.c_void_p * n)(*[c.h for c in contexts])
    na = (C.c_int * n)(*[int(k) for k in nactive])
    rc = _lib.piccs_run_staged_group(hs, na, n, C.byref(params), 1 if graph else 0)
    _check(rc, contexts[0].h if n else None)


def piccs_profile_enable(ctx, timing=True):
    _check(_lib.piccs_profile_enable(ctx, 1 if timing else 0), ctx)


def piccs_profile_read(ctx) -> dict:
    p = piccs_profile()
    _check(_lib.piccs_profile_read(ctx, C.byref(p)), ctx)
    return {"launches": {k: int(p.launches[i]) for i, k in enumerate(KERNEL_CLASSES)},
            "calls": {k: int(p.calls[i]) for i, k in enumerate(KERNEL_CLASSES)},
            "total_ms": {k: float(p.total_ms[i]) for i, k in enumerate(KERNEL_CLASSES)},
            "total_launches": int(p.total_launches)}


class Context:
    """Owns one piccs_ctx (one scanner geometry) on the current CUDA device.
    batch > 1: that many scans of the geometry are reconstructed together;
    volumes and projections then carry a leading batch dimension."""

    def __init__(self, geometry, stream=None, batch=1):
        self.gs = make_geometry(geometry)
        self.nx, self.ny, self.nz = self.gs.nx, self.gs.ny, self.gs.nz
        self.M = self.gs.nx * self.gs.ny * self.gs.nz
        self.N = self.gs.n_views * self.gs.nu * self.gs.nv
        if self.gs.proj_layout == LAYOUT_UV:
            self.proj_shape = (self.gs.n_views, self.gs.nu, self.gs.nv)
        else:
            self.proj_shape = (self.gs.n_views, self.gs.nv, self.gs.nu)
        self.vol_shape = (self.gs.nx, self.gs.ny, self.gs.nz)
        self.batch = int(batch)
        if self.batch > 1:
            self.proj_shape = (self.batch,) + self.proj_shape
            self.vol_shape = (self.batch,) + self.vol_shape
            self.h = piccs_create_batched(self.gs, self.batch, stream)
        else:
            self.h = piccs_create(self.gs, stream)
        self.BM, self.BN = self.batch * self.M, self.batch * self.N

    def close(self):
        if self.h:
            piccs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream):
        piccs_set_stream(self.h, stream)

    def set_prior(self, xp):
        _ptr(xp, self.BM, "prior")
        piccs_set_prior(self.h, xp)

    def forward(self, vol, out=None):
        import torch
        if out is None:
            out = torch.empty(self.proj_shape, dtype=torch.float32, device=vol.device)
        _ptr(vol, self.BM, "volume")
        _ptr(out, self.BN, "projections")
        piccs_forward(self.h, vol, out)
        return out

    def adjoint(self, proj, out=None):
        import torch
        if out is None:
            out = torch.empty(self.vol_shape, dtype=torch.float32, device=proj.device)
        _ptr(proj, self.BN, "projections")
        _ptr(out, self.BM, "volume")
        piccs_adjoint(self.h, proj, out)
        return out

    def reconstruct(self, proj, params, x0=None, out=None):
        import torch
        if out is None:
            out = torch.empty(self.vol_shape, dtype=torch.float32, device=proj.device)
        _ptr(proj, self.BN, "projections")
        _ptr(out, self.BM, "volume")
        if x0 is not None:
            _ptr(x0, self.BM, "x0")
        piccs_reconstruct(self.h, proj, params, x0, out)
        return out

    def reconstruct_host(self, proj, params, x0=None, out=None):
        """proj/x0/out are host tensors or arrays (pinned for full bandwidth)."""
        if out is None:
            out = np.empty(self.vol_shape, dtype=np.float32)
        _ptr(proj, self.BN, "projections")
        _ptr(out, self.BM, "volume")
        if x0 is not None:
            _ptr(x0, self.BM, "x0")
        piccs_reconstruct_host(self.h, proj, params, x0, out)
        return out

    def report(self, slot=0):
        return piccs_report_slot(self.h, slot)

    # staged reconstructions (the request server's building blocks)
    def set_prior_broadcast(self, prior_host):
        prior_host = np.ascontiguousarray(prior_host, dtype=np.float32)
        _check(_lib.piccs_set_prior_broadcast(self.h, _ptr(prior_host, self.M, "prior"), 1), self.h)

    def stage(self, slot, proj, host=True):
        _check(_lib.piccs_stage(self.h, int(slot), _ptr(proj, self.N, "projections"),
                                1 if host else 0), self.h)

    def stage_bf16(self, slot, proj_bits, host=True):
        _check(_lib.piccs_stage_bf16(self.h, int(slot), _ptr16(proj_bits, self.N, "projections"),
                                     1 if host else 0), self.h)

    def run_staged(self, nactive, params, graph=True):
        _check(_lib.piccs_run_staged(self.h, int(nactive), C.byref(params), 1 if graph else 0),
               self.h)

    def unstage(self, slot, out, host=True):
        _check(_lib.piccs_unstage(self.h, int(slot), _ptr(out, self.M, "volume"),
                                  1 if host else 0), self.h)

    def profile_enable(self, timing=True):
        piccs_profile_enable(self.h, timing)

    def profile_read(self) -> dict:
        return piccs_profile_read(self.h)

    def reg_weights(self, x, params, omega=None, c=None):
        import torch
        omega = torch.empty_like(x) if omega is None else omega
        c = torch.empty_like(x) if c is None else c
        piccs_reg_weights(self.h, x, params, omega, c)
        return omega, c

    def reg_normal(self, omega, params, z, out=None):
        import torch
        out = torch.empty_like(z) if out is None else out
        rho = piccs_reg_normal(self.h, omega, params, z, out, True)
        return out, rho


# --------------------------------------------------------------------------
# request server (include/piccs_server.h)
# --------------------------------------------------------------------------
def _check_srv(rc, srv):
    if rc != PICCS_OK:
        m = _lib.piccs_server_last_error(srv)
        raise PiccsError(rc, (m.decode() if m else "") or _NAMES.get(rc, str(rc)))


class Server:
    """A request loop for repeated scans: per-patient device sessions admitted
    by HBM footprint, continuous batching, overlapped batches, groups of
    patients' scans of different sizes run in shared launches (max_group),
    CUDA graphs.  Buffers handed to submit() are kept referenced until wait()
    returns."""

    def __init__(self, hbm_budget=0, max_batch=8, max_running=4, use_graphs=True, order=2,
                 max_group=1):
        cfg = piccs_server_config(int(hbm_budget), int(max_batch), int(max_running),
                                  1 if use_graphs else 0, int(order), int(max_group))
        h = C.c_void_p()
        _check_srv(_lib.piccs_server_create(C.byref(h), C.byref(cfg)), None)
        self.h = h.value
        self._held = {}
        self._shapes = {}

    def close(self):
        if self.h:
            _lib.piccs_server_destroy(self.h)
            self.h = None
            self._held.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_patient(self, patient, geometry, prior):
        gs = geometry if isinstance(geometry, piccs_geometry) else make_geometry(geometry)
        M = gs.nx * gs.ny * gs.nz
        prior = np.ascontiguousarray(prior, dtype=np.float32)
        _check_srv(_lib.piccs_server_add_patient(self.h, int(patient), C.byref(gs),
                                                 _ptr(prior, M, "prior")), self.h)
        self._shapes[int(patient)] = (gs.n_views * gs.nu * gs.nv, (gs.nx, gs.ny, gs.nz))

    def submit(self, patient, proj, params, out=None):
        """proj: host projections (pinned torch tensor or numpy array; BF16 --
        torch.bfloat16 or uint16 bit patterns -- for STORAGE_BF16 params);
        returns (ticket, out)."""
        N, vol_shape = self._shapes[int(patient)]
        if out is None:
            out = np.empty(vol_shape, dtype=np.float32)
        t = C.c_longlong(0)
        pp = _ptr16(proj, N, "projections") if params.storage == STORAGE_BF16 else \
            _ptr(proj, N, "projections")
        _check_srv(_lib.piccs_server_submit(self.h, int(patient), pp,
                                            C.byref(params), _ptr(out, int(np.prod(vol_shape)),
                                                                  "volume"), C.byref(t)), self.h)
        self._held[t.value] = (proj, out, params)
        return t.value, out

    def wait(self, ticket, timeout_ms=-1) -> dict:
        st = piccs_request_stats()
        rc = _lib.piccs_server_wait(self.h, int(ticket), int(timeout_ms), C.byref(st))
        if rc == PICCS_ETIMEOUT:
            return None
        _check_srv(rc, self.h)
        self._held.pop(int(ticket), None)
        return {"status": st.status, "batch": st.batch, "queued_ms": st.queued_ms,
                "run_ms": st.run_ms, "total_ms": st.total_ms}

    def stats(self) -> dict:
        st = piccs_server_stats()
        _check_srv(_lib.piccs_server_get_stats(self.h, C.byref(st)), self.h)
        return {k: int(getattr(st, k)) for k, _ in piccs_server_stats._fields_}
