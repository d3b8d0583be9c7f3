"""GB300 (sm_103a) library for explicit f-x poststack depth migration.

Thin ctypes binding over the C ABI of ``libfxmig.so`` (``include/fxmig.h``):
the functions below carry the C names, check and marshal their arguments
(torch tensors -> raw device pointers, the current torch stream -> cudaStream_t)
and raise ``FxmigError`` on a non-zero return code.  Every step of the method
runs in the library's CUDA kernels; PyTorch only provides device memory and
streams.  There is no CPU fallback: if the library is missing this module
raises on import of any entry point.

Method: Shawahna, Salam, Al-Mouhamed, "Seismic Imaging: An Overview and Parallel
Implementation of Poststack Depth Migration", arXiv 1912.05529 (Algorithm 1,
Eq. 1, Sec. III).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os

__all__ = [
    "FXMIG_OK", "FXMIG_EINVAL", "FXMIG_ENOSPC", "FXMIG_ECUDA", "FXMIG_ETIMEOUT", "FXMIG_EVELOCITY", "FXMIG_ERANGE",
    "FXMIG_WS_T2F", "FXMIG_WS_MIGRATE", "FXMIG_WS_MLP_MIGRATE", "FXMIG_PREC_FP32", "FXMIG_PREC_FP16",
    "FXMIG_PREC_BF16", "FXMIG_PREC_FP16_SPLIT", "FXMIG_PREC_BF16_SPLIT", "FXMIG_MODE_AUTO", "FXMIG_MODE_PERSISTENT", "FXMIG_MODE_PER_DEPTH",
    "FxmigError", "Desc", "Launch", "lib", "library_path",
    "fxmig_version", "fxmig_strerror", "fxmig_workspace_bytes", "fxmig_num_partials", "Shape",
    "fxmig_launch_shape",
    "fxmig_design_operators", "fxmig_t2f", "fxmig_migrate", "fxmig_migrate_ex", "fxmig_image",
    "fxmig_check", "fxmig_migrate_noalloc", "fxmig_selftest_timeout", "desc_for", "migrate_section",
    "fxmig_mlp_param_count", "fxmig_mlp_train_ws_bytes", "fxmig_design_at", "fxmig_mlp_train",
    "fxmig_mlp_grad", "fxmig_mlp_taps", "fxmig_mlp_num_partials", "fxmig_mlp_migrate",
    "Line", "BatchPlan", "line_of", "fxmig_batch_workspace_bytes", "fxmig_batch_num_partials",
    "fxmig_batch_autotune", "fxmig_migrate_batch",
    "Desc3d", "fxmig3d_num_taps", "fxmig3d_design_operators", "fxmig3d_workspace_bytes", "fxmig3d_num_partials",
    "fxmig3d_migrate", "fxmig3d_image", "flat_desc",
]

FXMIG_OK, FXMIG_EINVAL, FXMIG_ENOSPC, FXMIG_ECUDA, FXMIG_ETIMEOUT, FXMIG_EVELOCITY, FXMIG_ERANGE = \
    0, -1, -2, -3, -4, -5, -6
FXMIG_WS_T2F, FXMIG_WS_MIGRATE, FXMIG_WS_MLP_MIGRATE = 1, 2, 3
FXMIG_PREC_FP32, FXMIG_PREC_FP16, FXMIG_PREC_BF16, FXMIG_PREC_FP16_SPLIT, FXMIG_PREC_BF16_SPLIT = 0, 1, 2, 3, 4
FXMIG_MODE_AUTO, FXMIG_MODE_PERSISTENT, FXMIG_MODE_PER_DEPTH = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libfxmig.so")
_lib = None


class FxmigError(RuntimeError):
    def __init__(self, code: int, where: str):
        detail = ""
        if code == FXMIG_ECUDA and _lib is not None:
            detail = ": " + _lib.fxmig_last_error().decode()
        super().__init__(f"{where} failed: {fxmig_strerror(code)} ({code}){detail}")
        self.code = code


class Desc(ctypes.Structure):
    """Mirror of ``fxmig_desc``."""
    _fields_ = [("nx", ctypes.c_int), ("nz", ctypes.c_int), ("nt", ctypes.c_int), ("nw", ctypes.c_int),
                ("i0", ctypes.c_int), ("L", ctypes.c_int), ("nk", ctypes.c_int),
                ("dx", ctypes.c_double), ("dz", ctypes.c_double), ("dt", ctypes.c_double),
                ("theta_max_deg", ctypes.c_double), ("k_max", ctypes.c_double)]

    def __repr__(self):
        return "Desc(" + ", ".join(f"{n}={getattr(self, n)}" for n, _ in self._fields_) + ")"


class Desc3d(ctypes.Structure):
    """Mirror of ``fxmig3d_desc`` (3-D migration with 2-D extrapolators)."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("nt", ctypes.c_int),
                ("nw", ctypes.c_int), ("i0", ctypes.c_int), ("L", ctypes.c_int), ("nk", ctypes.c_int),
                ("dx", ctypes.c_double), ("dz", ctypes.c_double), ("dt", ctypes.c_double),
                ("theta_max_deg", ctypes.c_double), ("k_max", ctypes.c_double)]

    def __repr__(self):
        return "Desc3d(" + ", ".join(f"{n}={getattr(self, n)}" for n, _ in self._fields_) + ")"


class Line(ctypes.Structure):
    """Mirror of ``fxmig_line`` (one line of a batch; device pointers)."""
    _fields_ = [("d", Desc), ("slab", ctypes.c_void_p), ("vel", ctypes.c_void_p), ("table", ctypes.c_void_p),
                ("partials", ctypes.c_void_p), ("z_begin", ctypes.c_int), ("z_end", ctypes.c_int)]


class BatchPlan(ctypes.Structure):
    """Mirror of ``fxmig_batch_plan`` (zeros = defaults)."""
    _fields_ = [("cluster", ctypes.c_int), ("lines_cap", ctypes.c_int)]


class Shape(ctypes.Structure):
    """Mirror of ``fxmig_shape`` (the launch fxmig_migrate_ex makes)."""
    _fields_ = [("mode", ctypes.c_int), ("cluster", ctypes.c_int), ("groups", ctypes.c_int),
                ("ctas", ctypes.c_int), ("warps", ctypes.c_int), ("items_per_lane", ctypes.c_int),
                ("waves", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("smem_bytes", ctypes.c_size_t)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class Launch(ctypes.Structure):
    """Mirror of ``fxmig_launch`` (zeros = automatic)."""
    _fields_ = [("mode", ctypes.c_int), ("cluster", ctypes.c_int), ("groups", ctypes.c_int),
                ("warps", ctypes.c_int), ("precision", ctypes.c_int), ("ctas_per_sm", ctypes.c_int)]


def lib():
    """Load libfxmig.so (built by ``paper_1912_05529_gb300.build``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise ImportError(f"{library_path} is missing: build it with "
                              "`python -m paper_1912_05529_gb300.build` (nvcc, sm_103a)")
        L = ctypes.CDLL(library_path)
        vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        pd, pl = ctypes.POINTER(Desc), ctypes.POINTER(Launch)
        L.fxmig_version.restype = i
        L.fxmig_strerror.argtypes = [i]
        L.fxmig_strerror.restype = ctypes.c_char_p
        L.fxmig_last_error.restype = ctypes.c_char_p
        L.fxmig_workspace_bytes.argtypes = [pd, i]
        L.fxmig_workspace_bytes.restype = sz
        L.fxmig_num_partials.argtypes = [pd, pl]
        L.fxmig_num_partials.restype = i
        L.fxmig_launch_shape.argtypes = [pd, pl, ctypes.POINTER(Shape)]
        L.fxmig_launch_shape.restype = i
        L.fxmig_design_operators.argtypes = [pd, vp, vp, vp]
        L.fxmig_t2f.argtypes = [pd, vp, vp, vp, sz, vp]
        L.fxmig_migrate.argtypes = [pd, vp, vp, vp, vp, i, i, i, vp, sz, vp]
        L.fxmig_migrate_ex.argtypes = [pd, pl, vp, vp, vp, vp, i, i, i, vp, sz, vp]
        L.fxmig_image.argtypes = [pd, vp, i, vp, vp]
        L.fxmig_check.argtypes = [vp, vp]
        L.fxmig_selftest_timeout.argtypes = [vp, i, vp]
        fl = ctypes.c_float
        L.fxmig_mlp_param_count.argtypes = [i]
        L.fxmig_mlp_train_ws_bytes.argtypes = [i, i]
        L.fxmig_mlp_train_ws_bytes.restype = sz
        L.fxmig_design_at.argtypes = [pd, vp, i, vp, vp, vp]
        L.fxmig_mlp_train.argtypes = [pd, vp, vp, vp, i, i, fl, fl, i, vp, vp, i, vp, vp, sz, vp]
        L.fxmig_mlp_grad.argtypes = [pd, vp, vp, vp, i, vp, vp, vp, sz, vp]
        L.fxmig_mlp_taps.argtypes = [pd, vp, vp, i, vp, vp]
        L.fxmig_mlp_num_partials.argtypes = [pd]
        L.fxmig_mlp_migrate.argtypes = [pd, vp, vp, vp, vp, i, i, i, vp, sz, vp]
        p3 = ctypes.POINTER(Desc3d)
        L.fxmig3d_num_taps.argtypes = [i]
        L.fxmig3d_design_operators.argtypes = [p3, vp, vp, vp]
        L.fxmig3d_workspace_bytes.argtypes = [p3]
        L.fxmig3d_workspace_bytes.restype = sz
        L.fxmig3d_num_partials.argtypes = [p3]
        L.fxmig3d_migrate.argtypes = [p3, vp, vp, vp, vp, i, i, i, i, vp, vp]
        L.fxmig3d_image.argtypes = [p3, vp, i, vp, vp]
        pln, pbp = ctypes.POINTER(Line), ctypes.POINTER(BatchPlan)
        L.fxmig_batch_workspace_bytes.argtypes = [pln, i, i]
        L.fxmig_batch_workspace_bytes.restype = sz
        L.fxmig_batch_num_partials.argtypes = [pln, i, pbp, ctypes.POINTER(ctypes.c_int)]
        L.fxmig_batch_autotune.argtypes = [pln, i, pbp, ctypes.POINTER(ctypes.c_float), vp, sz, vp]
        L.fxmig_migrate_batch.argtypes = [pln, i, pbp, vp, sz, vp]
        for f in ("fxmig_design_operators", "fxmig_t2f", "fxmig_migrate", "fxmig_migrate_ex",
                  "fxmig_image", "fxmig_check", "fxmig_mlp_param_count", "fxmig_design_at",
                  "fxmig_mlp_train", "fxmig_mlp_grad", "fxmig_mlp_taps", "fxmig_mlp_num_partials",
                  "fxmig_mlp_migrate", "fxmig_batch_num_partials", "fxmig_batch_autotune",
                  "fxmig_migrate_batch", "fxmig_selftest_timeout", "fxmig3d_num_taps",
                  "fxmig3d_design_operators", "fxmig3d_num_partials", "fxmig3d_migrate", "fxmig3d_image"):
            getattr(L, f).restype = i
        _lib = L
    return _lib


# ------------------------------------------------------------------ helpers
def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev_ptr(t, what, dtype=None, numel=None, complex_ok=False):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what}: expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{what}: must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what}: must be contiguous")
    if dtype is not None:
        ok = t.dtype == dtype or (complex_ok and t.dtype == torch.complex64 and dtype == torch.float32)
        if not ok:
            raise TypeError(f"{what}: dtype {t.dtype}, expected {dtype}")
    if numel is not None:
        n = t.numel() * (2 if t.is_complex() else 1)
        if n < numel:
            raise ValueError(f"{what}: {n} elements, need {numel}")
    return ctypes.c_void_p(t.data_ptr())


def _check(code, where):
    if code != FXMIG_OK:
        raise FxmigError(code, where)


# ---------------------------------------------------------------- C entry points
def fxmig_version() -> int:
    return lib().fxmig_version()


def fxmig_strerror(code: int) -> str:
    return lib().fxmig_strerror(code).decode()


def fxmig_workspace_bytes(d: Desc, kind: int) -> int:
    return int(lib().fxmig_workspace_bytes(ctypes.byref(d), kind))


def fxmig_num_partials(d: Desc, launch: Launch | None = None) -> int:
    n = lib().fxmig_num_partials(ctypes.byref(d), ctypes.byref(launch) if launch else None)
    if n < 0:
        raise FxmigError(n, "fxmig_num_partials")
    return n


def fxmig_launch_shape(d: Desc, launch: Launch | None = None) -> Shape:
    """The launch fxmig_migrate_ex makes for d and launch (None = automatic)."""
    out = Shape()
    _check(lib().fxmig_launch_shape(ctypes.byref(d), ctypes.byref(launch) if launch else None, ctypes.byref(out)),
           "fxmig_launch_shape")
    return out


def fxmig_design_operators(d: Desc, table, table64=None, stream=None) -> None:
    """table: [nk][L+1] complex64 (device); table64: [nk][L+1] complex128 or None."""
    torch = _torch()
    n = d.nk * (d.L + 1)
    tp = _dev_ptr(table, "table", torch.float32, 2 * n, complex_ok=True)
    t64 = None
    if table64 is not None:
        if table64.dtype not in (torch.complex128, torch.float64):
            raise TypeError("table64: expected complex128 or float64")
        t64 = _dev_ptr(table64, "table64", None, 2 * n)
    _check(lib().fxmig_design_operators(ctypes.byref(d), tp, t64, _stream(stream)), "fxmig_design_operators")


def fxmig_t2f(d: Desc, section, slab, ws, stream=None) -> None:
    """section: [nx][nt] float32; slab: [nw][nx] complex64; ws: uint8 scratch."""
    torch = _torch()
    sp = _dev_ptr(section, "section", torch.float32, d.nx * d.nt)
    bp = _dev_ptr(slab, "slab", torch.float32, 2 * d.nw * d.nx, complex_ok=True)
    wp = _dev_ptr(ws, "ws")
    _check(lib().fxmig_t2f(ctypes.byref(d), sp, bp, wp, ws.numel() * ws.element_size(), _stream(stream)),
           "fxmig_t2f")


def fxmig_migrate_ex(d: Desc, launch: Launch | None, slab, vel, table, partials, z_begin, z_end, ws,
                     stream=None) -> None:
    torch = _torch()
    bp = _dev_ptr(slab, "slab", torch.float32, 2 * d.nw * d.nx, complex_ok=True)
    vp = _dev_ptr(vel, "vel", torch.float32, d.nz * d.nx)
    tp = _dev_ptr(table, "table", torch.float32, 2 * d.nk * (d.L + 1), complex_ok=True)
    pp = _dev_ptr(partials, "partials", torch.float32)
    nparts = partials.numel() // max(1, d.nz * d.nx)
    wp = _dev_ptr(ws, "ws")
    rc = lib().fxmig_migrate_ex(ctypes.byref(d), ctypes.byref(launch) if launch else None, bp, vp, tp, pp,
                                int(nparts), int(z_begin), int(z_end), wp, ws.numel() * ws.element_size(),
                                _stream(stream))
    _check(rc, "fxmig_migrate")


def fxmig_migrate(d: Desc, slab, vel, table, partials, z_begin, z_end, ws, stream=None) -> None:
    """slab: [nw][nx] complex64 in/out; vel: [nz][nx] float32; table: [nk][L+1]
    complex64; partials: [nparts][nz][nx] float32, the image accumulator
    (fixed-point rows, read by fxmig_image); ws: uint8 scratch."""
    fxmig_migrate_ex(d, None, slab, vel, table, partials, z_begin, z_end, ws, stream)


def fxmig_image(d: Desc, partials, image, stream=None) -> None:
    torch = _torch()
    pp = _dev_ptr(partials, "partials", torch.float32)
    nparts = partials.numel() // max(1, d.nz * d.nx)
    ip = _dev_ptr(image, "image", torch.float32, d.nz * d.nx)
    _check(lib().fxmig_image(ctypes.byref(d), pp, int(nparts), ip, _stream(stream)), "fxmig_image")


# ------------------------------------------------- 3-D, 2-D extrapolators
def fxmig3d_num_taps(L: int) -> int:
    n = lib().fxmig3d_num_taps(int(L))
    if n < 0:
        raise FxmigError(n, "fxmig3d_num_taps")
    return n


def flat_desc(d: "Desc3d", L: int = 4) -> Desc:
    """The 2-D description of the flattened surface grid (nx ny traces), for
    fxmig_t2f on a section [ny][nx][nt] (the other fields as in d)."""
    return Desc(nx=d.nx * d.ny, nz=d.nz, nt=d.nt, nw=d.nw, i0=d.i0, L=L, nk=d.nk, dx=d.dx, dz=d.dz, dt=d.dt,
                theta_max_deg=d.theta_max_deg, k_max=d.k_max)


def fxmig3d_design_operators(d: "Desc3d", table, table64=None, stream=None) -> None:
    """table: [nk][taps] complex64 (device); table64: [nk][taps] complex128 or None."""
    torch = _torch()
    n = d.nk * fxmig3d_num_taps(d.L)
    tp = _dev_ptr(table, "table", torch.float32, 2 * n, complex_ok=True)
    t64 = None
    if table64 is not None:
        if table64.dtype not in (torch.complex128, torch.float64):
            raise TypeError("table64: expected complex128 or float64")
        t64 = _dev_ptr(table64, "table64", None, 2 * n)
    _check(lib().fxmig3d_design_operators(ctypes.byref(d), tp, t64, _stream(stream)), "fxmig3d_design_operators")


def fxmig3d_workspace_bytes(d: "Desc3d") -> int:
    return int(lib().fxmig3d_workspace_bytes(ctypes.byref(d)))


def fxmig3d_num_partials(d: "Desc3d") -> int:
    n = lib().fxmig3d_num_partials(ctypes.byref(d))
    if n < 0:
        raise FxmigError(n, "fxmig3d_num_partials")
    return n


def fxmig3d_migrate(d: "Desc3d", slab, vel, table, partials, z_begin, z_end, ws, groups: int = 0,
                    stream=None) -> None:
    """slab: [nw][ny][nx] complex64; vel: [nz][ny][nx] float32; table: [nk][taps]
    complex64; partials: [nparts][nz][ny][nx] float32; ws: uint8 scratch of
    fxmig3d_workspace_bytes(d)."""
    torch = _torch()
    npts = d.nx * d.ny
    bp = _dev_ptr(slab, "slab", torch.float32, 2 * d.nw * npts, complex_ok=True)
    vp = _dev_ptr(vel, "vel", torch.float32, d.nz * npts)
    tp = _dev_ptr(table, "table", torch.float32, 2 * d.nk * fxmig3d_num_taps(d.L), complex_ok=True)
    pp = _dev_ptr(partials, "partials", torch.float32)
    nparts = partials.numel() // max(1, d.nz * npts)
    wp = _dev_ptr(ws, "ws", None, fxmig3d_workspace_bytes(d) // max(1, ws.element_size()))
    _check(lib().fxmig3d_migrate(ctypes.byref(d), bp, vp, tp, pp, int(nparts), int(z_begin), int(z_end),
                                 int(groups), wp, _stream(stream)), "fxmig3d_migrate")


def fxmig3d_image(d: "Desc3d", partials, image, stream=None) -> None:
    """image: [nz][ny][nx] float32 from the accumulator of fxmig3d_migrate."""
    torch = _torch()
    npts = d.nx * d.ny
    pp = _dev_ptr(partials, "partials", torch.float32)
    nparts = partials.numel() // max(1, d.nz * npts)
    ip = _dev_ptr(image, "image", torch.float32, d.nz * npts)
    _check(lib().fxmig3d_image(ctypes.byref(d), pp, int(nparts), ip, _stream(stream)), "fxmig3d_image")


def fxmig_check(ws, stream=None) -> int:
    """Synchronise the stream and return the device status code (0 = ok)."""
    return int(lib().fxmig_check(_dev_ptr(ws, "ws"), _stream(stream)))


def fxmig_selftest_timeout(ws, polls: int = 1000, stream=None) -> None:
    """Make the device's bounded wait give up once (nothing arrives at its
    barrier); fxmig_check(ws) then reports FXMIG_ETIMEOUT."""
    _check(lib().fxmig_selftest_timeout(_dev_ptr(ws, "ws"), int(polls), _stream(stream)), "fxmig_selftest_timeout")


def fxmig_migrate_noalloc(d: Desc, slab, vel, table, partials, z_begin, z_end, stream=None) -> None:
    """fxmig_migrate without a workspace argument: the library keeps its scratch
    in a fixed device array (for callers that cannot allocate; see fxmig.h)."""
    torch = _torch()
    L = lib()
    f = L.fxmig_migrate_noalloc
    f.argtypes = [ctypes.POINTER(Desc)] + [ctypes.c_void_p] * 4 + [ctypes.c_int] * 3 + [ctypes.c_void_p]
    f.restype = ctypes.c_int
    bp = _dev_ptr(slab, "slab", torch.float32, 2 * d.nw * d.nx, complex_ok=True)
    vp = _dev_ptr(vel, "vel", torch.float32, d.nz * d.nx)
    tp = _dev_ptr(table, "table", torch.float32, 2 * d.nk * (d.L + 1), complex_ok=True)
    pp = _dev_ptr(partials, "partials", torch.float32)
    nparts = partials.numel() // max(1, d.nz * d.nx)
    _check(f(ctypes.byref(d), bp, vp, tp, pp, int(nparts), int(z_begin), int(z_end), _stream(stream)),
           "fxmig_migrate_noalloc")


# ------------------------------------------------------------ learned operators
def fxmig_mlp_param_count(L: int) -> int:
    n = lib().fxmig_mlp_param_count(int(L))
    if n < 0:
        raise FxmigError(n, "fxmig_mlp_param_count")
    return n


def fxmig_mlp_train_ws_bytes(L: int, n: int) -> int:
    return int(lib().fxmig_mlp_train_ws_bytes(int(L), int(n)))


def _taps_ptr(taps, what, n, L):
    torch = _torch()
    return _dev_ptr(taps, what, torch.float32, 2 * n * (L + 1), complex_ok=True)


def fxmig_design_at(d: Desc, k, taps, taps64=None, stream=None) -> None:
    """k: [n] float64 (device); taps: [n][L+1] complex64; taps64: complex128 or None."""
    torch = _torch()
    n = k.numel()
    kp = _dev_ptr(k, "k", torch.float64)
    tp = _taps_ptr(taps, "taps", n, d.L)
    t64 = None
    if taps64 is not None:
        if taps64.dtype not in (torch.complex128, torch.float64):
            raise TypeError("taps64: expected complex128 or float64")
        t64 = _dev_ptr(taps64, "taps64", None, 2 * n * (d.L + 1))
    _check(lib().fxmig_design_at(ctypes.byref(d), kp, int(n), tp, t64, _stream(stream)), "fxmig_design_at")


def fxmig_mlp_train(d: Desc, params, adam_m, adam_v, step0, nsteps, lr_max, lr_min, schedule_steps, k, taps,
                    ws, loss=None, stream=None) -> None:
    """nsteps Adam steps on samples (k[i], taps[i]); loss: [nsteps] float32 or None."""
    torch = _torch()
    P = fxmig_mlp_param_count(d.L)
    n = k.numel()
    lp = _dev_ptr(loss, "loss", torch.float32, int(nsteps)) if loss is not None else None
    rc = lib().fxmig_mlp_train(ctypes.byref(d), _dev_ptr(params, "params", torch.float32, P),
                               _dev_ptr(adam_m, "adam_m", torch.float32, P),
                               _dev_ptr(adam_v, "adam_v", torch.float32, P), int(step0), int(nsteps),
                               float(lr_max), float(lr_min), int(schedule_steps), _dev_ptr(k, "k", torch.float64),
                               _taps_ptr(taps, "taps", n, d.L), int(n), lp, _dev_ptr(ws, "ws"),
                               ws.numel() * ws.element_size(), _stream(stream))
    _check(rc, "fxmig_mlp_train")


def fxmig_mlp_grad(d: Desc, params, k, taps, grad, ws, loss=None, stream=None) -> None:
    torch = _torch()
    P = fxmig_mlp_param_count(d.L)
    n = k.numel()
    lp = _dev_ptr(loss, "loss", torch.float32, 1) if loss is not None else None
    rc = lib().fxmig_mlp_grad(ctypes.byref(d), _dev_ptr(params, "params", torch.float32, P),
                              _dev_ptr(k, "k", torch.float64), _taps_ptr(taps, "taps", n, d.L), int(n),
                              _dev_ptr(grad, "grad", torch.float32, P), lp, _dev_ptr(ws, "ws"),
                              ws.numel() * ws.element_size(), _stream(stream))
    _check(rc, "fxmig_mlp_grad")


def fxmig_mlp_taps(d: Desc, params, k, taps, stream=None) -> None:
    torch = _torch()
    n = k.numel()
    rc = lib().fxmig_mlp_taps(ctypes.byref(d), _dev_ptr(params, "params", torch.float32,
                                                        fxmig_mlp_param_count(d.L)),
                              _dev_ptr(k, "k", torch.float64), int(n), _taps_ptr(taps, "taps", n, d.L),
                              _stream(stream))
    _check(rc, "fxmig_mlp_taps")


def fxmig_mlp_num_partials(d: Desc) -> int:
    n = lib().fxmig_mlp_num_partials(ctypes.byref(d))
    if n < 0:
        raise FxmigError(n, "fxmig_mlp_num_partials")
    return n


def fxmig_mlp_migrate(d: Desc, slab, vel, params, partials, z_begin, z_end, ws, stream=None) -> None:
    """Depth loop with network operators at the exact slowness of every point."""
    torch = _torch()
    bp = _dev_ptr(slab, "slab", torch.float32, 2 * d.nw * d.nx, complex_ok=True)
    vp = _dev_ptr(vel, "vel", torch.float32, d.nz * d.nx)
    mp = _dev_ptr(params, "params", torch.float32, fxmig_mlp_param_count(d.L))
    pp = _dev_ptr(partials, "partials", torch.float32)
    nparts = partials.numel() // max(1, d.nz * d.nx)
    wp = _dev_ptr(ws, "ws")
    rc = lib().fxmig_mlp_migrate(ctypes.byref(d), bp, vp, mp, pp, int(nparts), int(z_begin), int(z_end), wp,
                                 ws.numel() * ws.element_size(), _stream(stream))
    _check(rc, "fxmig_mlp_migrate")


# ------------------------------------------------------------ batches of lines
def line_of(d: Desc, slab, vel, table, partials, z_begin=0, z_end=None) -> Line:
    """A ``fxmig_line`` for torch tensors (device, contiguous); keep the
    tensors alive while the line is used."""
    torch = _torch()
    return Line(d=d, slab=_dev_ptr(slab, "slab", torch.float32, 2 * d.nw * d.nx, complex_ok=True),
                vel=_dev_ptr(vel, "vel", torch.float32, d.nz * d.nx),
                table=_dev_ptr(table, "table", torch.float32, 2 * d.nk * (d.L + 1), complex_ok=True),
                partials=_dev_ptr(partials, "partials", torch.float32),
                z_begin=int(z_begin), z_end=int(d.nz if z_end is None else z_end))


def _lines_array(lines):
    arr = (Line * len(lines))(*lines)
    return arr, len(lines)


def fxmig_batch_workspace_bytes(lines, autotune: bool = False) -> int:
    arr, n = _lines_array(lines)
    return int(lib().fxmig_batch_workspace_bytes(arr, n, 1 if autotune else 0))


def fxmig_batch_num_partials(lines, plan: BatchPlan | None = None) -> list:
    """Partial images of every line (only the descriptors are read)."""
    arr, n = _lines_array(lines)
    out = (ctypes.c_int * n)()
    _check(lib().fxmig_batch_num_partials(arr, n, ctypes.byref(plan) if plan else None, out),
           "fxmig_batch_num_partials")
    return list(out)


def fxmig_batch_autotune(lines, ws, stream=None):
    """Returns (BatchPlan, best time in ms over the tuning depth rows)."""
    arr, n = _lines_array(lines)
    plan, ms = BatchPlan(), ctypes.c_float(0.0)
    _check(lib().fxmig_batch_autotune(arr, n, ctypes.byref(plan), ctypes.byref(ms), _dev_ptr(ws, "ws"),
                                      ws.numel() * ws.element_size(), _stream(stream)), "fxmig_batch_autotune")
    return plan, float(ms.value)


def fxmig_migrate_batch(lines, plan: BatchPlan | None, ws, stream=None) -> None:
    arr, n = _lines_array(lines)
    _check(lib().fxmig_migrate_batch(arr, n, ctypes.byref(plan) if plan else None, _dev_ptr(ws, "ws"),
                                     ws.numel() * ws.element_size(), _stream(stream)), "fxmig_migrate_batch")


# ------------------------------------------------------------------ conveniences
def desc_for(nx, nz, nt, dx, dz, dt, f_lo, f_hi, L, v_min, nk=1024, theta_deg=65.0) -> Desc:
    """Descriptor of a problem: band bins f_lo <= j/(nt dt) <= f_hi and a table
    spanning k up to w_max / v_min (v_min: smallest migration velocity)."""
    df = 1.0 / (nt * dt)
    i0 = max(1, int(math.ceil(f_lo / df - 1e-9)))
    i1 = min((nt - 1) // 2, int(math.floor(f_hi / df + 1e-9)))
    nw = i1 - i0 + 1
    k_max = 2.0 * math.pi * (i0 + nw - 1) / (nt * dt) / v_min
    return Desc(nx=nx, nz=nz, nt=nt, nw=nw, i0=i0, L=L, nk=nk, dx=dx, dz=dz, dt=dt,
                theta_max_deg=theta_deg, k_max=k_max)


@dataclasses.dataclass
class Buffers:
    """Device buffers of one migration (caller-owned, reusable across calls)."""
    section: object
    slab: object
    vel: object
    table: object
    partials: object
    image: object
    ws_t2f: object
    ws_mig: object


def allocate(d: Desc, launch: Launch | None = None, device="cuda") -> Buffers:
    torch = _torch()
    nparts = fxmig_num_partials(d, launch)
    return Buffers(
        section=torch.empty((d.nx, d.nt), dtype=torch.float32, device=device),
        slab=torch.empty((d.nw, d.nx), dtype=torch.complex64, device=device),
        vel=torch.empty((d.nz, d.nx), dtype=torch.float32, device=device),
        table=torch.empty((d.nk, d.L + 1), dtype=torch.complex64, device=device),
        partials=torch.empty((nparts, d.nz, d.nx), dtype=torch.float32, device=device),
        image=torch.empty((d.nz, d.nx), dtype=torch.float32, device=device),
        ws_t2f=torch.empty(fxmig_workspace_bytes(d, FXMIG_WS_T2F), dtype=torch.uint8, device=device),
        ws_mig=torch.empty(fxmig_workspace_bytes(d, FXMIG_WS_MIGRATE), dtype=torch.uint8, device=device),
    )


def migrate_section(d: Desc, section_host, vel_host, bufs: Buffers | None = None, launch: Launch | None = None,
                    image_host=None, design: bool = True, stream=None):
    """End-to-end migration from host arrays (Algorithm 1): copy the section and
    velocity to the device, t -> f, (design the table), depth loop, imaging,
    copy the image back.  Returns the host image tensor [nz][nx]."""
    torch = _torch()
    b = bufs or allocate(d, launch)
    b.section.copy_(section_host, non_blocking=True)
    b.vel.copy_(vel_host, non_blocking=True)
    if design:
        fxmig_design_operators(d, b.table, None, stream)
    fxmig_t2f(d, b.section, b.slab, b.ws_t2f, stream)
    fxmig_migrate_ex(d, launch, b.slab, b.vel, b.table, b.partials, 0, d.nz, b.ws_mig, stream)
    fxmig_image(d, b.partials, b.image, stream)
    if image_host is None:
        image_host = torch.empty((d.nz, d.nx), dtype=torch.float32, pin_memory=True)
    image_host.copy_(b.image, non_blocking=True)
    return image_host
