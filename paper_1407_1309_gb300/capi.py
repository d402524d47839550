"""Thin ctypes binding of the C ABI in include/mpdata.h.

The functions keep the C names and only marshal arguments: tensors become
device pointers (``data_ptr()``), sequences of advector components become
host arrays of pointers, status codes become exceptions.  Every computation
runs in the CUDA library; if the library cannot be built or loaded this module
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

# element types, option bits and status codes (include/mpdata.h)
F32, F64 = 0, 1
FCT, TOT, IGA, NUG, KAHAN, RHS_EULER_A, RHS_EULER_B, STAGED, ABS, DFL = 1, 2, 4, 8, 16, 32, 64, 128, 256, 512
OPEN0, OPEN1, OPEN2 = 1024, 2048, 4096  # open edges along dimension 0, 1, 2 (Sect. 2.4)
RHS_TRAPEZ = 65536  # trapezoidal source scheme with sources affine in the state (Sect. 4.1)
SW = 131072  # shallow-water system with prognosed velocity (Sect. 5)
OK, EINVAL, EUNSUPPORTED, ECUDA, ECOURANT, ETIMEOUT, ESTOPPED, ENOMEM = range(8)

EXPORTED = (
    "mpdata_create", "mpdata_step", "mpdata_advance", "mpdata_adjoint_step", "mpdata_reduce",
    "mpdata_diff_norms", "mpdata_check_courant", "mpdata_request_stop", "mpdata_clear_stop",
    "mpdata_sync", "mpdata_destroy", "mpdata_strerror", "mpdata_version", "mpdata_tune", "mpdata_set_stream",
    "mpdata_advance_compensated", "mpdata_selftest_division", "mpdata_selftest_fma_rate",
    "mpdata_adjoint_tape_bytes", "mpdata_adjoint_record", "mpdata_adjoint_replay", "mpdata_adjoint_step_rhs",
    "mpdata_set_rhs_linear", "mpdata_step_noalloc", "mpdata_sw_advance", "mpdata_sw_reset",
)
TUNE_TILE_ROWS = 1
TUNE_KERNEL = 2
TUNE_STEPS_PER_LAUNCH = 3


class MpdataError(RuntimeError):
    """A non-OK status code returned by the library."""

    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {mpdata_strerror(code)} (status {code})")


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libmpdata_gb300.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_needed and not _build.up_to_date():
            path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with `python -m paper_1407_1309_gb300.build`")
        lib = ctypes.CDLL(path)
        P, I, U, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_double, ctypes.c_int64
        PP = ctypes.POINTER(ctypes.c_void_p)
        DP = ctypes.POINTER(ctypes.c_double)
        sig = {
            "mpdata_create": ([ctypes.POINTER(ctypes.c_void_p), I, I, ctypes.POINTER(I64), I, I, U, P], I),
            "mpdata_step": ([P, P, PP, P, P, D, I], I),
            "mpdata_advance": ([P, P, P, PP, P, P, D, I, DP], I),
            "mpdata_advance_compensated": ([P, P, P, P, P, PP, P, P, D, I, DP], I),
            "mpdata_selftest_division": ([P, P, P, I64, P], I),
            "mpdata_selftest_fma_rate": ([I, I64, P, ctypes.POINTER(I64), P], I),
            "mpdata_adjoint_step": ([P, P, PP, P, P, PP], I),
            "mpdata_adjoint_step_rhs": ([P, P, PP, P, P, D, P, PP, P], I),
            "mpdata_adjoint_tape_bytes": ([P, ctypes.POINTER(ctypes.c_size_t)], I),
            "mpdata_adjoint_record": ([P, P, PP, P, P, P], I),
            "mpdata_adjoint_replay": ([P, P, PP, P, P, P, PP], I),
            "mpdata_reduce": ([P, P, P, DP], I),
            "mpdata_diff_norms": ([P, P, P, DP, DP], I),
            "mpdata_check_courant": ([P, PP, P, DP], I),
            "mpdata_tune": ([P, I, I], I),
            "mpdata_set_rhs_linear": ([P, DP, P], I),
            "mpdata_sw_advance": ([P, P, D, D, D, I], I),
            "mpdata_sw_reset": ([P], I),
            "mpdata_set_stream": ([P, P], I),
            "mpdata_request_stop": ([P], I),
            "mpdata_clear_stop": ([P], I),
            "mpdata_sync": ([P], I),
            "mpdata_destroy": ([P], I),
            "mpdata_strerror": ([I], ctypes.c_char_p),
            "mpdata_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _ptr(x):
    """Device pointer of a tensor (or an int address); None stays NULL."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_contiguous") and not x.is_contiguous():
            raise ValueError("tensors passed to the library must be contiguous")
        return x.data_ptr()
    raise TypeError(f"expected a tensor or an address, got {type(x)!r}")


def _ptr_array(xs):
    if xs is None:
        return None
    arr = (ctypes.c_void_p * max(1, len(xs)))(*[_ptr(x) for x in xs])
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), arr


def _check(rc, where):
    if rc != OK:
        raise MpdataError(rc, where)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def mpdata_strerror(code: int) -> str:
    return load().mpdata_strerror(int(code)).decode()


def mpdata_version() -> str:
    return load().mpdata_version().decode()


def mpdata_create(ndims, shapes, dtype, n_iters, opts, stream=None, *, raw=False):
    """shapes: one tuple of ndims extents per field.  Returns the handle (int)."""
    flat = [int(s) for shp in shapes for s in shp]
    arr = (ctypes.c_int64 * max(1, len(flat)))(*flat)
    h = ctypes.c_void_p()
    rc = load().mpdata_create(ctypes.byref(h), int(ndims), len(shapes), arr, int(dtype), int(n_iters),
                              int(opts), _stream_ptr(stream))
    if raw:
        return rc, h.value
    _check(rc, "mpdata_create")
    return h.value


def mpdata_step(h, psi, gc, g=None, r=None, dt=0.0, n_steps=1, *, raw=False):
    gcp, _keep = _ptr_array(gc)
    rc = load().mpdata_step(h, _ptr(psi), gcp, _ptr(g), _ptr(r), float(dt), int(n_steps))
    if raw:
        return rc
    _check(rc, "mpdata_step")


def mpdata_advance(h, psi_in, psi_out, gc, g=None, r=None, dt=0.0, n_steps=1, gc_scale=None, *, raw=False):
    gcp, _keep = _ptr_array(gc)
    sc = None
    if gc_scale is not None:
        sc = (ctypes.c_double * len(gc_scale))(*[float(v) for v in gc_scale])
        if len(gc_scale) < n_steps:
            raise ValueError("gc_scale needs one factor per step")
    rc = load().mpdata_advance(h, _ptr(psi_in), _ptr(psi_out), gcp, _ptr(g), _ptr(r), float(dt), int(n_steps),
                               ctypes.cast(sc, ctypes.POINTER(ctypes.c_double)) if sc is not None else None)
    if raw:
        return rc
    _check(rc, "mpdata_advance")


def mpdata_advance_compensated(h, psi_in, lo_in, psi_out, lo_out, gc, g=None, r=None, dt=0.0, n_steps=1,
                               gc_scale=None, *, raw=False):
    gcp, _keep = _ptr_array(gc)
    sc = None
    if gc_scale is not None:
        if len(gc_scale) < n_steps:
            raise ValueError("gc_scale needs one factor per step")
        sc = (ctypes.c_double * len(gc_scale))(*[float(v) for v in gc_scale])
    rc = load().mpdata_advance_compensated(h, _ptr(psi_in), _ptr(lo_in), _ptr(psi_out), _ptr(lo_out), gcp, _ptr(g),
                                           _ptr(r), float(dt), int(n_steps),
                                           ctypes.cast(sc, ctypes.POINTER(ctypes.c_double)) if sc is not None else None)
    if raw:
        return rc
    _check(rc, "mpdata_advance_compensated")


def mpdata_selftest_division(n, d, q, stream=None):
    """q = n / d elementwise with the kernels' FP64 division (device float64 tensors)."""
    _check(load().mpdata_selftest_division(_ptr(n), _ptr(d), _ptr(q), int(q.numel()), _ptr(stream)),
           "mpdata_selftest_division")


def mpdata_set_rhs_linear(h, A, b=None):
    """Sources R = A psi + b of the trapezoidal scheme; A: n_fields x n_fields (anything numpy
    turns into that many doubles, row-major), b: device tensor of the handle's total size or None."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(A, dtype=np.float64)).ravel()
    arr = (ctypes.c_double * max(1, a.size))(*a.tolist())
    _check(load().mpdata_set_rhs_linear(h, arr, _ptr(b)), "mpdata_set_rhs_linear")


def mpdata_sw_advance(h, state, dt, dx, eps=1e-8, n_steps=1, *, raw=False):
    """Shallow-water steps of a MPDATA_SW handle on state = [h, q_0, ..] (one device tensor)."""
    rc = load().mpdata_sw_advance(h, _ptr(state), float(dt), float(dx), float(eps), int(n_steps))
    if raw:
        return rc
    _check(rc, "mpdata_sw_advance")


def mpdata_sw_reset(h):
    _check(load().mpdata_sw_reset(h), "mpdata_sw_reset")


def mpdata_selftest_fma_rate(dtype, iters, sink, stream=None):
    """Launch the FMA-rate kernel (F32 or F64) on `stream`; returns the FMA lane operations it
    issues.  sink: a one-element device tensor of that dtype."""
    n = ctypes.c_int64(0)
    _check(load().mpdata_selftest_fma_rate(int(dtype), int(iters), _ptr(sink), ctypes.byref(n), _stream_ptr(stream)),
           "mpdata_selftest_fma_rate")
    return n.value


def prepare_advance(h, psi_in, psi_out, gc, g=None, r=None, dt=0.0, n_steps=1):
    """mpdata_advance with its arguments marshalled once: returns a callable that issues
    the same call (same buffers) again with no per-call argument conversion, for loops
    whose host-side cost must stay below the device time of a step.  The caller keeps
    the tensors alive while the callable is in use."""
    gcp, keep = _ptr_array(gc)
    fn = load().mpdata_advance
    args = (h, _ptr(psi_in), _ptr(psi_out), gcp, _ptr(g), _ptr(r), float(dt), int(n_steps), None)

    def call():
        rc = fn(*args)
        if rc != 0:
            _check(rc, "mpdata_advance")
    call._keep = keep
    return call


def prepare_advance_compensated(h, psi_in, lo_in, psi_out, lo_out, gc, g=None, r=None, dt=0.0, n_steps=1):
    """mpdata_advance_compensated with its arguments marshalled once (as prepare_advance)."""
    gcp, keep = _ptr_array(gc)
    fn = load().mpdata_advance_compensated
    args = (h, _ptr(psi_in), _ptr(lo_in), _ptr(psi_out), _ptr(lo_out), gcp, _ptr(g), _ptr(r), float(dt),
            int(n_steps), None)

    def call():
        rc = fn(*args)
        if rc != 0:
            _check(rc, "mpdata_advance_compensated")
    call._keep = keep
    return call


def mpdata_adjoint_step(h, psi_n, gc, g, psi_bar, gc_bar=None, *, raw=False):
    gcp, _k1 = _ptr_array(gc)
    gbp = None
    if gc_bar is not None:
        gbp, _k2 = _ptr_array(gc_bar)
    rc = load().mpdata_adjoint_step(h, _ptr(psi_n), gcp, _ptr(g), _ptr(psi_bar), gbp)
    if raw:
        return rc
    _check(rc, "mpdata_adjoint_step")


def mpdata_adjoint_step_rhs(h, psi_n, gc, g, r, dt, psi_bar, gc_bar=None, r_bar=None, *, raw=False):
    gcp, _k1 = _ptr_array(gc)
    gbp = None
    if gc_bar is not None:
        gbp, _k2 = _ptr_array(gc_bar)
    rc = load().mpdata_adjoint_step_rhs(h, _ptr(psi_n), gcp, _ptr(g), _ptr(r), float(dt), _ptr(psi_bar), gbp,
                                        _ptr(r_bar))
    if raw:
        return rc
    _check(rc, "mpdata_adjoint_step_rhs")


def mpdata_adjoint_tape_bytes(h):
    out = ctypes.c_size_t(0)
    _check(load().mpdata_adjoint_tape_bytes(h, ctypes.byref(out)), "mpdata_adjoint_tape_bytes")
    return out.value


def mpdata_adjoint_record(h, psi_n, gc, g, tape, psi_next=None, *, raw=False):
    gcp, _k1 = _ptr_array(gc)
    rc = load().mpdata_adjoint_record(h, _ptr(psi_n), gcp, _ptr(g), _ptr(tape), _ptr(psi_next))
    if raw:
        return rc
    _check(rc, "mpdata_adjoint_record")


def mpdata_adjoint_replay(h, psi_n, gc, g, tape, psi_bar, gc_bar=None, *, raw=False):
    gcp, _k1 = _ptr_array(gc)
    gbp = None
    if gc_bar is not None:
        gbp, _k2 = _ptr_array(gc_bar)
    rc = load().mpdata_adjoint_replay(h, _ptr(psi_n), gcp, _ptr(g), _ptr(tape), _ptr(psi_bar), gbp)
    if raw:
        return rc
    _check(rc, "mpdata_adjoint_replay")


def mpdata_reduce(h, psi, g=None, n_fields=1):
    out = (ctypes.c_double * n_fields)()
    _check(load().mpdata_reduce(h, _ptr(psi), _ptr(g), out), "mpdata_reduce")
    return list(out)


def mpdata_diff_norms(h, a, b, n_fields=1):
    l2 = (ctypes.c_double * n_fields)()
    li = (ctypes.c_double * n_fields)()
    _check(load().mpdata_diff_norms(h, _ptr(a), _ptr(b), l2, li), "mpdata_diff_norms")
    return list(l2), list(li)


def mpdata_check_courant(h, gc, g=None):
    """Returns (status, max outflow sum); status is OK or ECOURANT."""
    gcp, _keep = _ptr_array(gc)
    m = ctypes.c_double(0.0)
    rc = load().mpdata_check_courant(h, gcp, _ptr(g), ctypes.byref(m))
    if rc not in (OK, ECOURANT):
        _check(rc, "mpdata_check_courant")
    return rc, m.value


def mpdata_tune(h, knob, value):
    _check(load().mpdata_tune(h, int(knob), int(value)), "mpdata_tune")


def mpdata_set_stream(h, stream):
    _check(load().mpdata_set_stream(h, _stream_ptr(stream)), "mpdata_set_stream")


def mpdata_request_stop(h):
    _check(load().mpdata_request_stop(h), "mpdata_request_stop")


def mpdata_clear_stop(h):
    _check(load().mpdata_clear_stop(h), "mpdata_clear_stop")


def mpdata_sync(h, *, raw=False):
    rc = load().mpdata_sync(h)
    if raw:
        return rc
    _check(rc, "mpdata_sync")


def mpdata_destroy(h):
    _check(load().mpdata_destroy(h), "mpdata_destroy")


def mpdata_step_noalloc(ndims, shape, dtype, n_iters, opts, psi_in, psi_out, gc, g=None, r=None, dt=0.0,
                        stream=None, *, raw=False):
    """One step of one field without a handle and without any device allocation (the scratch is a
    static device array inside the library); for callers that may not allocate device memory.
    Returns the status code when raw=True, else raises on error."""
    shape = tuple(int(v) for v in shape)
    if int(ndims) != len(shape) or len(gc) != len(shape):
        raise ValueError("mpdata_step_noalloc: ndims, len(shape) and len(gc) must agree")
    n = 1
    for v in shape:
        n *= v
    want = {F32: "torch.float32", F64: "torch.float64"}.get(int(dtype))
    for name, x in [("psi_in", psi_in), ("psi_out", psi_out), ("g", g), ("r", r)] + \
            [(f"gc[{d}]", v) for d, v in enumerate(gc)]:
        if x is None or isinstance(x, int):
            continue  # NULL, or a raw address the caller vouches for
        if not getattr(x, "is_cuda", False) or not x.is_contiguous():
            raise ValueError(f"mpdata_step_noalloc: {name} must be a contiguous CUDA tensor")
        if want is not None and str(x.dtype) != want:
            raise ValueError(f"mpdata_step_noalloc: {name} has dtype {x.dtype}, expected {want}")
        if x.numel() != n:
            raise ValueError(f"mpdata_step_noalloc: {name} has {x.numel()} elements, expected {n}")
    lib = load()
    fn = lib.mpdata_step_noalloc
    fn.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_int, ctypes.c_uint32,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    shp = (ctypes.c_int64 * max(1, len(shape)))(*[int(v) for v in shape])
    gcp, _keep = _ptr_array(gc)
    rc = fn(int(ndims), shp, int(dtype), int(n_iters), int(opts), _ptr(psi_in), _ptr(psi_out), gcp, _ptr(g),
            _ptr(r), float(dt), _stream_ptr(stream))
    if raw:
        return rc
    _check(rc, "mpdata_step_noalloc")
