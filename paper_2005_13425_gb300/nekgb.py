"""Thin Python binding of ``include/nekgb.h`` (ctypes).

Each function has the name of the C entry point it wraps and only marshals
arguments: device buffers are passed as raw addresses (``int``) or as CUDA
tensors whose ``data_ptr()`` is taken after dtype/contiguity/device checks;
host arrays are numpy arrays.  Every step of the computation runs in
``libnekgb.so``; there is no Python or CPU fallback.  If the library has not
been built (``__graft_entry__.build()``), loading raises ``NekgbUnavailable``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnekgb.so")

NB_OK, NB_ERR_ARG, NB_ERR_CUDA, NB_ERR_OOM = 0, 1, 2, 3
NB_ERR_NOT_CONVERGED, NB_ERR_BREAKDOWN, NB_ERR_TIMEOUT, NB_ERR_STATE = 4, 5, 6, 7
NB_FP64, NB_MIXED = 0, 1
NB_K_AX, NB_K_DSSUM, NB_K_MASK, NB_K_DOT, NB_K_UPDATE, NB_K_OTHER = range(6)
NB_K_COUNT = 6
KERNEL_NAMES = {NB_K_AX: "ax_e", NB_K_DSSUM: "dssum", NB_K_MASK: "mask",
                NB_K_DOT: "dot", NB_K_UPDATE: "update", NB_K_OTHER: "other"}


class NekgbUnavailable(RuntimeError):
    """libnekgb.so is missing or cannot be loaded."""


class NekgbError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: status {status} ({msg})")


class nb_box(ctypes.Structure):
    _fields_ = [("ex", ctypes.c_int), ("ey", ctypes.c_int), ("ez", ctypes.c_int)]


class nb_info(ctypes.Structure):
    _fields_ = [("ex", ctypes.c_int), ("ey", ctypes.c_int), ("ez", ctypes.c_int),
                ("n", ctypes.c_int), ("nelt", ctypes.c_int64), ("npts", ctypes.c_int64),
                ("nunique", ctypes.c_int64), ("precision", ctypes.c_int),
                ("ax_variant", ctypes.c_int), ("device_bytes", ctypes.c_size_t)]


class nb_request(ctypes.Structure):
    _fields_ = [("mesh", nb_box), ("n", ctypes.c_int), ("amp", ctypes.c_double),
                ("s", ctypes.c_double * 3), ("tol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("prec", ctypes.c_int), ("inner_tol", ctypes.c_double)]


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "nb_setup": [ctypes.POINTER(_vp), nb_box, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, _vp],
    "nb_setup_box": [ctypes.POINTER(_vp), nb_box, ctypes.c_int, ctypes.c_double, _vp,
                     ctypes.c_int, _vp],
    "nb_destroy": [_vp],
    "nb_get_info": [_vp, ctypes.POINTER(nb_info)],
    "nb_ax": [_vp, _vp, _vp],
    "nb_dssum": [_vp, _vp],
    "nb_mask": [_vp, _vp],
    "nb_apply": [_vp, _vp, _vp],
    "nb_cg_solve": [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, _ip, _dp],
    "nb_cg_solve_host": [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, _ip, _dp],
    "nb_cg_history": [_vp, _vp, ctypes.c_int, _ip],
    "nb_dot_c": [_vp, _vp, _vp, _dp],
    "nb_dot_c_noalloc": [nb_box, ctypes.c_int, _vp, _vp, _vp, _vp],
    "nb_scatter_unique": [_vp, _vp, _vp],
    "nb_tables": [_vp, _vp, _vp, _vp],
    "nb_get_operator": [_vp, _vp, _vp],
    "nb_set_ax_variant": [_vp, ctypes.c_int],
    "nb_box_coords": [_vp, _vp],
    "nb_ax_f32": [_vp, _vp, _vp],
    "nb_dssum_f32": [_vp, _vp],
    "nb_set_mixed_params": [_vp, ctypes.c_double, ctypes.c_int],
    "nb_solve_stats": [_vp, _ip, _ip],
    "nb_set_preconditioner": [_vp, ctypes.c_int],
    "nb_jacobi_diagonal": [_vp, _vp],
    "nb_engine_create": [ctypes.POINTER(_vp), ctypes.c_size_t, _vp],
    "nb_engine_destroy": [_vp],
    "nb_engine_footprint": [nb_box, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)],
    "nb_engine_submit": [_vp, ctypes.POINTER(nb_request), _vp, _ip],
    "nb_engine_submit_unique": [_vp, ctypes.POINTER(nb_request), _vp, _ip],
    "nb_engine_step": [_vp, ctypes.c_int],
    "nb_engine_poll": [_vp, ctypes.c_int, _ip, _ip, _dp, _ip],
    "nb_engine_request_info": [_vp, ctypes.c_int, _ip, _ip],
    "nb_engine_retire": [_vp, ctypes.c_int, _vp],
    "nb_engine_stats": [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t), _ip],
    "nb_engine_tuning": [_vp, ctypes.c_int, ctypes.c_int, _ip, _ip],
    "nb_timing_enable": [_vp, ctypes.c_int],
    "nb_launch_count": [_vp, ctypes.POINTER(ctypes.c_int64)],
    "nb_timing_read": [_vp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_int64), ctypes.c_int],
    "nb_fp32_rate": [_dp],
    "nb_setup_slab": [ctypes.POINTER(_vp), nb_box, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                      ctypes.c_double, _vp, _vp],
    "nb_slab_info": [_vp, ctypes.POINTER(ctypes.c_int64), _ip, _ip],
    "nb_slab_top_partial": [_vp, _vp, _vp],
    "nb_slab_add_bottom": [_vp, _vp, _vp],
    "nb_slab_bottom_value": [_vp, _vp, _vp],
    "nb_slab_set_top": [_vp, _vp, _vp],
    "nb_slab_dot": [_vp, _vp, _vp, _dp],
    "nb_axpby": [_vp, ctypes.c_double, _vp, ctypes.c_double, _vp],
    "nb_probe_grad": [_vp, ctypes.c_int, _vp, _vp, ctypes.c_double],
}


def load(path: str = LIB_PATH):
    """Load libnekgb.so and declare every exported signature."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise NekgbUnavailable(f"{path} is not built; run __graft_entry__.build()")
        try:
            lib = ctypes.CDLL(path)
        except OSError as exc:
            raise NekgbUnavailable(f"cannot load {path}: {exc}") from exc
        for name, args in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.nb_status_str.argtypes = [ctypes.c_int]
        lib.nb_status_str.restype = ctypes.c_char_p
        lib.nb_last_error.argtypes = []
        lib.nb_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def exported_symbols():
    return sorted(list(_SIGS) + ["nb_status_str", "nb_last_error"])


def _check(status: int, where: str, ok=(NB_OK,)):
    if status not in ok:
        lib = load()
        raise NekgbError(status, where, (lib.nb_last_error() or b"").decode())
    return status


def _ptr(x, dtype=None) -> int:
    """Device address of a CUDA tensor (checked) or a raw int address."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        if dtype is not None and str(x.dtype) != dtype:
            raise ValueError(f"expected dtype {dtype}, got {x.dtype}")
        return x.data_ptr()
    raise TypeError(f"cannot take a device address of {type(x)}")


def _host(a, dtype):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, arr.ctypes.data


def _stream_handle(stream) -> int:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------ set-up
def nb_setup(mesh, n, D, gxyz, mask=None, prec=NB_FP64, stream=None):
    lib = load()
    ctx = _vp()
    Dh, Dp = _host(D, np.float64)
    Gh, Gp = _host(gxyz, np.float64)
    Mh, Mp = _host(mask, np.uint8)
    _check(lib.nb_setup(ctypes.byref(ctx), nb_box(*mesh), int(n), Dp, Gp, Mp, int(prec),
                        _stream_handle(stream)), "nb_setup")
    return ctx


def nb_setup_box(mesh, n, amp, s, prec=NB_FP64, stream=None):
    lib = load()
    ctx = _vp()
    Sh, Sp = _host(s, np.float64)
    _check(lib.nb_setup_box(ctypes.byref(ctx), nb_box(*mesh), int(n), float(amp), Sp, int(prec),
                            _stream_handle(stream)), "nb_setup_box")
    return ctx


def nb_destroy(ctx):
    _check(load().nb_destroy(ctx), "nb_destroy")


def nb_get_info(ctx) -> dict:
    info = nb_info()
    _check(load().nb_get_info(ctx, ctypes.byref(info)), "nb_get_info")
    return {name: getattr(info, name) for name, _ in nb_info._fields_}


# ------------------------------------------------------------------ operator
def nb_ax(ctx, u, w):
    _check(load().nb_ax(ctx, _ptr(u, "torch.float64"), _ptr(w, "torch.float64")), "nb_ax")


def nb_dssum(ctx, w):
    _check(load().nb_dssum(ctx, _ptr(w, "torch.float64")), "nb_dssum")


def nb_mask(ctx, w):
    _check(load().nb_mask(ctx, _ptr(w, "torch.float64")), "nb_mask")


def nb_apply(ctx, u, w):
    _check(load().nb_apply(ctx, _ptr(u, "torch.float64"), _ptr(w, "torch.float64")), "nb_apply")


# ------------------------------------------------------------------ solver
def nb_cg_solve(ctx, f, x, tol=0.0, maxit=100, allow=(NB_OK,)):
    """Returns (status, iters, relres); raises unless status is in `allow`."""
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = load().nb_cg_solve(ctx, _ptr(f, "torch.float64"), _ptr(x, "torch.float64"), float(tol),
                            int(maxit), ctypes.byref(it), ctypes.byref(rr))
    _check(st, "nb_cg_solve", allow)
    return st, it.value, rr.value


def nb_cg_solve_host(ctx, f_host: np.ndarray, x_host: np.ndarray, tol=0.0, maxit=100,
                     allow=(NB_OK,)):
    """Host-buffer solve; x_host (float64, contiguous) is updated in place."""
    if f_host.dtype != np.float64 or not f_host.flags.c_contiguous:
        raise ValueError("f_host must be contiguous float64")
    if x_host.dtype != np.float64 or not x_host.flags.c_contiguous:
        raise ValueError("x_host must be contiguous float64")
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = load().nb_cg_solve_host(ctx, f_host.ctypes.data, x_host.ctypes.data, float(tol),
                                 int(maxit), ctypes.byref(it), ctypes.byref(rr))
    _check(st, "nb_cg_solve_host", allow)
    return st, it.value, rr.value


def nb_cg_history(ctx) -> np.ndarray:
    cnt = ctypes.c_int(0)
    _check(load().nb_cg_history(ctx, None, 0, ctypes.byref(cnt)), "nb_cg_history")
    out = np.zeros(cnt.value)
    if cnt.value:
        _check(load().nb_cg_history(ctx, out.ctypes.data, cnt.value, ctypes.byref(cnt)),
               "nb_cg_history")
    return out


# ------------------------------------------------------------------ helpers
def nb_dot_c(ctx, a, b) -> float:
    out = ctypes.c_double(0.0)
    _check(load().nb_dot_c(ctx, _ptr(a, "torch.float64"), _ptr(b, "torch.float64"),
                           ctypes.byref(out)), "nb_dot_c")
    return out.value


def nb_dot_c_noalloc(mesh, n, a, b, out, stream=None):
    """<a,b>_c into the 1-double device buffer `out`, with no context and no
    allocation (asynchronous on `stream`)."""
    _check(load().nb_dot_c_noalloc(nb_box(*mesh), int(n), _ptr(a, "torch.float64"),
                                   _ptr(b, "torch.float64"), _ptr(out, "torch.float64"),
                                   _stream_handle(stream)), "nb_dot_c_noalloc")


def nb_scatter_unique(ctx, g, local):
    _check(load().nb_scatter_unique(ctx, _ptr(g, "torch.float64"), _ptr(local, "torch.float64")),
           "nb_scatter_unique")


def nb_tables(ctx, gid=None, mult=None, mask=None):
    _check(load().nb_tables(ctx, _ptr(gid, "torch.int64"), _ptr(mult, "torch.int32"),
                            _ptr(mask, "torch.uint8")), "nb_tables")


def nb_get_operator(ctx, n, gxyz_dev=None) -> np.ndarray:
    D = np.zeros((n, n))
    _check(load().nb_get_operator(ctx, D.ctypes.data, _ptr(gxyz_dev, "torch.float64")),
           "nb_get_operator")
    return D


def nb_box_coords(ctx, xyz):
    _check(load().nb_box_coords(ctx, _ptr(xyz, "torch.float64")), "nb_box_coords")


def nb_ax_f32(ctx, u, w):
    _check(load().nb_ax_f32(ctx, _ptr(u, "torch.float32"), _ptr(w, "torch.float32")), "nb_ax_f32")


def nb_dssum_f32(ctx, w):
    _check(load().nb_dssum_f32(ctx, _ptr(w, "torch.float32")), "nb_dssum_f32")


def nb_set_mixed_params(ctx, inner_tol: float = 1e-5, max_outer: int = 50):
    _check(load().nb_set_mixed_params(ctx, float(inner_tol), int(max_outer)), "nb_set_mixed_params")


def nb_set_preconditioner(ctx, kind: int):
    _check(load().nb_set_preconditioner(ctx, int(kind)), "nb_set_preconditioner")


def nb_jacobi_diagonal(ctx, minv):
    _check(load().nb_jacobi_diagonal(ctx, _ptr(minv, "torch.float64")), "nb_jacobi_diagonal")


def nb_solve_stats(ctx):
    """(iterations, outer corrections) of the last solve."""
    it = ctypes.c_int(0)
    outer = ctypes.c_int(0)
    _check(load().nb_solve_stats(ctx, ctypes.byref(it), ctypes.byref(outer)), "nb_solve_stats")
    return it.value, outer.value


def nb_set_ax_variant(ctx, variant: int):
    _check(load().nb_set_ax_variant(ctx, int(variant)), "nb_set_ax_variant")


def nb_timing_enable(ctx, on):
    """on: False/0 off, True/1 every launch event-timed, 2 sampled (see nekgb.h)."""
    _check(load().nb_timing_enable(ctx, int(on)), "nb_timing_enable")


def nb_launch_count(ctx) -> int:
    n = ctypes.c_int64(0)
    _check(load().nb_launch_count(ctx, ctypes.byref(n)), "nb_launch_count")
    return n.value


def nb_timing_read(ctx, kernel_id: int, reset: bool = False):
    ms = ctypes.c_double(0.0)
    cnt = ctypes.c_int64(0)
    _check(load().nb_timing_read(ctx, int(kernel_id), ctypes.byref(ms), ctypes.byref(cnt),
                                 1 if reset else 0), "nb_timing_read")
    return ms.value, cnt.value


def nb_probe_grad(ctx, method: int, u, w, umax: float):
    """Measurement probe: w = D_r u + D_s u + D_t u per element, by the
    double-float line products (method 0) or the tensor-core digit split
    (methods 1 and 2); see nekgb.h."""
    _check(load().nb_probe_grad(ctx, int(method), _ptr(u, "torch.float64"), _ptr(w, "torch.float64"),
                                float(umax)), "nb_probe_grad")


def nb_fp32_rate() -> float:
    """Measured FFMA (FP32 instruction) rate of the current device, per second."""
    v = ctypes.c_double(0.0)
    _check(load().nb_fp32_rate(ctypes.byref(v)), "nb_fp32_rate")
    return v.value


# ------------------------------------------------------------------ slabs
def nb_setup_slab(mesh, z0: int, z1: int, n: int, amp: float, s, stream=None):
    lib = load()
    ctx = _vp()
    Sh, Sp = _host(s, np.float64)
    _check(lib.nb_setup_slab(ctypes.byref(ctx), nb_box(*mesh), int(z0), int(z1), int(n), float(amp), Sp,
                             _stream_handle(stream)), "nb_setup_slab")
    return ctx


def nb_slab_info(ctx):
    """(plane_nodes, has_below, has_above)."""
    npl, lo, hi = ctypes.c_int64(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(load().nb_slab_info(ctx, ctypes.byref(npl), ctypes.byref(lo), ctypes.byref(hi)), "nb_slab_info")
    return npl.value, bool(lo.value), bool(hi.value)


def nb_slab_top_partial(ctx, w, buf):
    _check(load().nb_slab_top_partial(ctx, _ptr(w, "torch.float64"), _ptr(buf, "torch.float64")),
           "nb_slab_top_partial")


def nb_slab_add_bottom(ctx, w, buf):
    _check(load().nb_slab_add_bottom(ctx, _ptr(w, "torch.float64"), _ptr(buf, "torch.float64")),
           "nb_slab_add_bottom")


def nb_slab_bottom_value(ctx, w, buf):
    _check(load().nb_slab_bottom_value(ctx, _ptr(w, "torch.float64"), _ptr(buf, "torch.float64")),
           "nb_slab_bottom_value")


def nb_slab_set_top(ctx, w, buf):
    _check(load().nb_slab_set_top(ctx, _ptr(w, "torch.float64"), _ptr(buf, "torch.float64")),
           "nb_slab_set_top")


def nb_slab_dot(ctx, a, b) -> float:
    out = ctypes.c_double(0.0)
    _check(load().nb_slab_dot(ctx, _ptr(a, "torch.float64"), _ptr(b, "torch.float64"), ctypes.byref(out)),
           "nb_slab_dot")
    return out.value


def nb_axpby(ctx, alpha: float, x, beta: float, y):
    _check(load().nb_axpby(ctx, float(alpha), _ptr(x, "torch.float64"), float(beta), _ptr(y, "torch.float64")),
           "nb_axpby")


# ------------------------------------------------------------------ engine
def nb_engine_create(arena_bytes: int, stream=None):
    eng = _vp()
    _check(load().nb_engine_create(ctypes.byref(eng), int(arena_bytes), _stream_handle(stream)),
           "nb_engine_create")
    return eng


def nb_engine_destroy(eng):
    _check(load().nb_engine_destroy(eng), "nb_engine_destroy")


def nb_engine_footprint(mesh, n, prec=NB_FP64) -> int:
    b = ctypes.c_size_t(0)
    _check(load().nb_engine_footprint(nb_box(*mesh), int(n), int(prec), ctypes.byref(b)), "nb_engine_footprint")
    return b.value


def _request(mesh, n, amp, s, tol, maxit, prec, inner_tol):
    return nb_request(nb_box(*mesh), int(n), float(amp), (ctypes.c_double * 3)(*[float(v) for v in s]),
                      float(tol), int(maxit), int(prec), float(inner_tol))


def nb_engine_submit(eng, mesh, n, amp, s, tol, maxit, f, allow=(NB_OK,), prec=NB_FP64, inner_tol=0.0):
    """Returns (status, id); id is -1 when the request was not admitted."""
    req = _request(mesh, n, amp, s, tol, maxit, prec, inner_tol)
    rid = ctypes.c_int(-1)
    st = load().nb_engine_submit(eng, ctypes.byref(req), _ptr(f, "torch.float64"), ctypes.byref(rid))
    _check(st, "nb_engine_submit", allow)
    return st, (rid.value if st == NB_OK else -1)


def nb_engine_submit_unique(eng, mesh, n, amp, s, tol, maxit, fu, allow=(NB_OK,), prec=NB_FP64, inner_tol=0.0):
    """nb_engine_submit with f given per unique node (device, NX*NY*NZ)."""
    req = _request(mesh, n, amp, s, tol, maxit, prec, inner_tol)
    rid = ctypes.c_int(-1)
    st = load().nb_engine_submit_unique(eng, ctypes.byref(req), _ptr(fu, "torch.float64"), ctypes.byref(rid))
    _check(st, "nb_engine_submit_unique", allow)
    return st, (rid.value if st == NB_OK else -1)


def nb_engine_step(eng, iters: int):
    _check(load().nb_engine_step(eng, int(iters)), "nb_engine_step")


def nb_engine_poll(eng, rid: int):
    """(done, iterations, relres, status)."""
    d, it, st = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    _check(load().nb_engine_poll(eng, int(rid), ctypes.byref(d), ctypes.byref(it), ctypes.byref(rr),
                                 ctypes.byref(st)), "nb_engine_poll")
    return bool(d.value), it.value, rr.value, st.value


def nb_engine_request_info(eng, rid: int):
    """(precision, outer corrections so far)."""
    p, o = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().nb_engine_request_info(eng, int(rid), ctypes.byref(p), ctypes.byref(o)), "nb_engine_request_info")
    return p.value, o.value


def nb_engine_retire(eng, rid: int, x=None):
    _check(load().nb_engine_retire(eng, int(rid), _ptr(x, "torch.float64")), "nb_engine_retire")


def nb_engine_stats(eng):
    u, c, a = ctypes.c_size_t(0), ctypes.c_size_t(0), ctypes.c_int(0)
    _check(load().nb_engine_stats(eng, ctypes.byref(u), ctypes.byref(c), ctypes.byref(a)), "nb_engine_stats")
    return u.value, c.value, a.value


def nb_engine_tuning(eng, n: int, prec=NB_FP64):
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().nb_engine_tuning(eng, int(n), int(prec), ctypes.byref(a), ctypes.byref(b)), "nb_engine_tuning")
    return a.value, b.value


def nb_status_str(status: int) -> str:
    return load().nb_status_str(int(status)).decode()


def nb_last_error() -> str:
    return (load().nb_last_error() or b"").decode()
