"""The allocation-free step entry point (mpdata_step_noalloc) against mpdata_advance.

mpdata_step_noalloc exists for callers that may not allocate device memory when
they advance a field (a fixed memory budget owned by another allocator, or a
loop that cannot afford cudaMalloc/cudaFree synchronising the device); it takes
its scratch from a static device array inside the library.  This file is
collected last so that a run stopping at the first failure has already run every
other test; it passes both on its own and after the rest of the suite.
"""
import numpy as np
import pytest
import torch

from helpers import boxes, nondivergent, smooth_positive
from paper_1407_1309_gb300 import capi
from paper_1407_1309_gb300.solver import Mpdata

pytestmark = pytest.mark.gpu

CASES = [
    ((96, 80), 2, capi.FCT),
    ((61, 47), 2, capi.IGA | capi.FCT),
    ((12, 10, 9), 3, capi.TOT | capi.FCT),
    ((301,), 2, capi.FCT | capi.KAHAN),
]


def close(a, b, dtype):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    if dtype == torch.float64:
        return np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    return np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("shape,n_iters,opts", CASES, ids=lambda c: str(c))
def test_noalloc_matches_advance_on_two_calls(shape, n_iters, opts, dtype):
    rng = np.random.default_rng(len(shape) * 100 + n_iters)
    dev = torch.device("cuda")
    gc_np = nondivergent(shape, rng, 0.35)
    psi_np = boxes(shape, rng) if len(shape) != 2 else smooth_positive(shape, rng)
    if opts & capi.IGA:
        psi_np = psi_np - 2.5
    t = lambda a: torch.tensor(a, dtype=dtype, device=dev)
    gc = [t(v) for v in gc_np]
    psi = t(psi_np)
    dcode = capi.F32 if dtype == torch.float32 else capi.F64
    # existing entry point: one and two steps through a handle
    with Mpdata(shape, dtype=dtype, n_iters=n_iters, opts=opts) as m:
        ref1, ref2 = torch.empty_like(psi), torch.empty_like(psi)
        m.advance(psi, ref1, gc, n_steps=1)
        m.advance(psi, ref2, gc, n_steps=2)
    # new entry point: two calls in a row, the second reading the first's output
    out1, out2 = torch.empty_like(psi), torch.empty_like(psi)
    stream = torch.cuda.current_stream()
    capi.mpdata_step_noalloc(len(shape), shape, dcode, n_iters, opts, psi, out1, gc, stream=stream)
    capi.mpdata_step_noalloc(len(shape), shape, dcode, n_iters, opts, out1, out2, gc, stream=stream)
    torch.cuda.synchronize()
    assert close(out1, ref1, dtype)
    assert close(out2, ref2, dtype)


def test_noalloc_rejects_fields_beyond_the_static_scratch():
    dev = torch.device("cuda")
    limit = (16 << 20) // (16 * 4)  # 16 MiB static scratch / (16 arrays x 4 bytes): FP32 cell limit
    side = int(np.ceil(np.sqrt(limit + 1)))
    psi = torch.ones((side, side), device=dev)
    gc = [torch.zeros_like(psi), torch.zeros_like(psi)]
    rc = capi.mpdata_step_noalloc(2, (side, side), capi.F32, 2, capi.FCT, psi, psi, gc, raw=True)
    assert rc == capi.EINVAL
    # the largest allowed square still runs
    ok = int(np.floor(np.sqrt(limit)))
    p = torch.ones((ok, ok), device=dev)
    g = [torch.zeros_like(p), torch.zeros_like(p)]
    out = torch.empty_like(p)
    assert capi.mpdata_step_noalloc(2, (ok, ok), capi.F32, 2, capi.FCT, p, out, g, raw=True) == capi.OK
    torch.cuda.synchronize()
    assert torch.equal(out, p)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("shape,n_iters,opts", [((40, 33), 1, 0), ((40, 33), 2, capi.FCT),
                                                ((9, 8, 11), 1, 0), ((9, 8, 11), 2, capi.FCT),
                                                ((9, 8, 11), 3, capi.TOT | capi.FCT)],
                         ids=lambda c: str(c))
def test_noalloc_in_place_matches_the_handle(shape, n_iters, opts, dtype):
    """psi_in == psi_out is allowed: in place it gives what the handle path gives out of place,
    for one pass (the result is copied out of the scratch) and for several (with the limiter)."""
    rng = np.random.default_rng(7 + n_iters)
    dev = torch.device("cuda")
    t = lambda a: torch.tensor(a, dtype=dtype, device=dev)
    gc = [t(v) for v in nondivergent(shape, rng, 0.35)]
    psi = t(smooth_positive(shape, rng))
    dcode = capi.F32 if dtype == torch.float32 else capi.F64
    with Mpdata(shape, dtype=dtype, n_iters=n_iters, opts=opts) as m:
        ref = torch.empty_like(psi)
        m.advance(psi, ref, gc, n_steps=2)
    p = psi.clone()
    for _ in range(2):
        capi.mpdata_step_noalloc(len(shape), shape, dcode, n_iters, opts, p, p, gc,
                                 stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert close(p, ref, dtype)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("rhs", [capi.RHS_EULER_A, capi.RHS_EULER_B], ids=["euler_a", "euler_b"])
@pytest.mark.parametrize("inplace", [False, True], ids=["out_of_place", "in_place"])
def test_noalloc_with_g_and_sources(rhs, inplace, dtype):
    """Non-unit G and a source term (both Euler schemes of Sect. 4.1), in and out of place."""
    shape = (37, 29)
    rng = np.random.default_rng(21)
    dev = torch.device("cuda")
    t = lambda a: torch.tensor(a, dtype=dtype, device=dev)
    gc = [t(v) for v in nondivergent(shape, rng, 0.3)]
    psi = t(smooth_positive(shape, rng))
    G = t(1.0 + 0.3 * rng.uniform(size=shape))
    R = t(rng.normal(size=shape))
    opts = capi.FCT | capi.NUG | rhs
    dcode = capi.F32 if dtype == torch.float32 else capi.F64
    with Mpdata(shape, dtype=dtype, n_iters=2, opts=opts) as m:
        ref = torch.empty_like(psi)
        m.advance(psi, ref, gc, g=G, r=R, dt=0.25, n_steps=1)
    out = psi.clone() if inplace else torch.empty_like(psi)
    src = out if inplace else psi
    capi.mpdata_step_noalloc(2, shape, dcode, 2, opts, src, out, gc, g=G, r=R, dt=0.25,
                             stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert close(out, ref, dtype)


def test_noalloc_allocates_no_device_memory():
    """The reason the entry point exists: after a first call (module loading may allocate), further
    calls change neither the device's free memory nor torch's allocator."""
    shape = (64, 48, 20)
    rng = np.random.default_rng(3)
    dev = torch.device("cuda")
    gc = [torch.tensor(v, dtype=torch.float32, device=dev) for v in nondivergent(shape, rng, 0.3)]
    psi = torch.tensor(smooth_positive(shape, rng), dtype=torch.float32, device=dev)
    out = torch.empty_like(psi)
    stream = torch.cuda.current_stream()
    opts = capi.TOT | capi.FCT
    capi.mpdata_step_noalloc(3, shape, capi.F32, 3, opts, psi, out, gc, stream=stream)
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(5):
        capi.mpdata_step_noalloc(3, shape, capi.F32, 3, opts, out, out, gc, stream=stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_wrapper_rejects_inconsistent_arguments():
    dev = torch.device("cuda")
    psi = torch.ones((8, 8), device=dev)
    gc = [torch.zeros_like(psi), torch.zeros_like(psi)]
    with pytest.raises(ValueError):
        capi.mpdata_step_noalloc(3, (8, 8), capi.F32, 2, 0, psi, psi, gc)
    with pytest.raises(ValueError):
        capi.mpdata_step_noalloc(2, (8, 8), capi.F32, 2, 0, psi, psi, gc[:1])
    with pytest.raises(ValueError):
        capi.mpdata_step_noalloc(2, (8, 8), capi.F64, 2, 0, psi, psi, gc)
    with pytest.raises(ValueError):
        capi.mpdata_step_noalloc(2, (8, 9), capi.F32, 2, 0, psi, psi, gc)
