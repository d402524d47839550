"""Host-side checks of the C ABI that need no GPU: the library loads, exports every
symbol include/mpdata.h declares, and rejects invalid arguments before any CUDA call."""
import ctypes
import os
import re

import pytest

from paper_1407_1309_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "mpdata.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mpdata_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = capi.load()
    names = declared_symbols()
    assert "mpdata_create" in names and "mpdata_adjoint_step" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(capi.EXPORTED) <= set(names)


def test_status_strings_and_version():
    for code in range(8):
        assert capi.mpdata_strerror(code) and capi.mpdata_strerror(code) != "unknown status"
    assert capi.mpdata_strerror(99) == "unknown status"
    assert "sm_103a" in capi.mpdata_version()


@pytest.mark.parametrize("args", [
    dict(ndims=0, shapes=[()], dtype=0, n_iters=2, opts=0),
    dict(ndims=4, shapes=[(2, 2, 2, 2)], dtype=0, n_iters=2, opts=0),
    dict(ndims=2, shapes=[(4, 4)], dtype=2, n_iters=2, opts=0),
    dict(ndims=2, shapes=[(4, 4)], dtype=0, n_iters=0, opts=0),
    dict(ndims=2, shapes=[(4, 0)], dtype=0, n_iters=2, opts=0),
    dict(ndims=2, shapes=[(4, -3)], dtype=0, n_iters=2, opts=0),
    dict(ndims=2, shapes=[(4, 4)], dtype=0, n_iters=3, opts=capi.IGA),
    dict(ndims=2, shapes=[(4, 4)], dtype=0, n_iters=2, opts=capi.RHS_EULER_A | capi.RHS_EULER_B),
    dict(ndims=2, shapes=[(4, 4)], dtype=0, n_iters=2, opts=1 << 14),
    dict(ndims=2, shapes=[(4, 4)], dtype=0, n_iters=2, opts=capi.OPEN2),
    dict(ndims=2, shapes=[(4, 1)], dtype=0, n_iters=2, opts=capi.OPEN1),
    dict(ndims=1, shapes=[(4,)], dtype=0, n_iters=2, opts=capi.RHS_TRAPEZ | capi.RHS_EULER_B),
    dict(ndims=1, shapes=[(4,)], dtype=0, n_iters=2, opts=capi.SW),
    dict(ndims=1, shapes=[(4,), (5,)], dtype=0, n_iters=2, opts=capi.SW),
    dict(ndims=1, shapes=[(4,), (4,)], dtype=0, n_iters=2, opts=capi.SW | capi.NUG),
    dict(ndims=2, shapes=[(4, 4)], dtype=0, n_iters=2, opts=capi.DFL | capi.IGA),
    dict(ndims=2, shapes=[(4, 4)], dtype=0, n_iters=2, opts=capi.ABS | capi.IGA),
])
def test_create_rejects_invalid_arguments(args):
    rc, h = capi.mpdata_create(args["ndims"], args["shapes"], args["dtype"], args["n_iters"], args["opts"], raw=True)
    assert rc == capi.EINVAL and not h


def test_null_handle_is_rejected():
    lib = capi.load()
    assert lib.mpdata_step(None, None, None, None, None, 0.0, 1) == capi.EINVAL
    assert lib.mpdata_destroy(None) == capi.EINVAL
    assert lib.mpdata_request_stop(None) == capi.EINVAL
    assert lib.mpdata_sync(None) == capi.EINVAL
    out = ctypes.c_void_p()
    assert lib.mpdata_create(None, 2, 1, None, 0, 2, 0, None) == capi.EINVAL


def test_python_and_oracle_constants_match_the_header():
    """The option bits, element types, status codes and tuning knobs the binding (and the
    oracle, for its options) use are the values include/mpdata.h declares."""
    import oracle
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "mpdata.h")).read()
    enums = {m.group(1): int(m.group(2)) for m in re.finditer(r"\bMPDATA_([A-Z0-9_]+)\s*=\s*(\d+)u?\b", hdr)}
    for name in ("FCT", "TOT", "IGA", "NUG", "KAHAN", "RHS_EULER_A", "RHS_EULER_B", "STAGED", "ABS", "DFL",
                 "F32", "F64", "OK", "EINVAL", "EUNSUPPORTED", "ECUDA", "ECOURANT", "ETIMEOUT", "ESTOPPED", "ENOMEM",
                 "TUNE_TILE_ROWS", "TUNE_KERNEL", "TUNE_STEPS_PER_LAUNCH", "OPEN0", "OPEN1", "OPEN2", "RHS_TRAPEZ", "SW"):
        assert getattr(capi, name) == enums[name], name
    for name in ("FCT", "TOT", "IGA", "NUG", "KAHAN", "RHS_EULER_A", "RHS_EULER_B", "ABS", "DFL",
                 "OPEN0", "OPEN1", "OPEN2"):
        assert getattr(oracle, name) == enums[name], name
