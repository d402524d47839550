"""The fused 2D kernels (warp march and band march) against the staged kernels
and the oracle.

Sizes span several strips (120 output columns in FP32, 56 in FP64) and row
tiles or bands, ragged edges, odd widths (scalar copies) and even widths (vector
copies), fields shorter than one band, and band heights from 5 rows (many
bands, a ragged last one) to 64; the full 1024^2 rotation workload runs a short
sequence in the bench's launch configuration.
"""
import zlib

import numpy as np
import pytest
import torch

import oracle
from helpers import boxes, nondivergent, smooth_positive
from paper_1407_1309_gb300 import capi, workloads
from paper_1407_1309_gb300.solver import Mpdata

pytestmark = pytest.mark.gpu

FUSED_OPTS = {
    "basic": 0,
    "fct": capi.FCT,
    "iga_fct": capi.IGA | capi.FCT,
    "kahan_fct": capi.KAHAN | capi.FCT,
    "iga": capi.IGA,
}


# kernel family (MPDATA_TUNE_KERNEL) and tile / band rows (MPDATA_TUNE_TILE_ROWS)
KERNELS = {"warp": (1, 0), "band": (2, 0), "band_h5": (2, 5), "band_h64": (2, 64), "warp2": (3, 0),
           "warp2_h12": (3, 12)}
_ORACLE = {}


def gpu_run(psi, gc, G, R, dt, opts, n_steps, dtype, staged, kernel="band", gc_scale=None):
    dev = torch.device("cuda")
    t = lambda a: None if a is None else torch.tensor(a, dtype=dtype, device=dev)
    o = opts | (capi.NUG if G is not None else 0) | (capi.STAGED if staged else 0)
    with Mpdata(psi.shape, dtype=dtype, n_iters=2, opts=o) as m:
        fam, rows = KERNELS[kernel]
        m.tune(capi.TUNE_KERNEL, fam)
        m.tune(capi.TUNE_TILE_ROWS, rows)
        a = t(psi)
        b = torch.empty_like(a)
        m.advance(a, b, [t(v) for v in gc], t(G), t(R), dt, n_steps, gc_scale)
        torch.cuda.synchronize()
        return b.cpu().numpy().astype(np.float64)


def r32(a):
    return None if a is None else a.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("shape", [(200, 130), (57, 123), (64, 64), (9, 250), (130, 7)],
                         ids=lambda s: f"{s[0]}x{s[1]}")
@pytest.mark.parametrize("name", sorted(FUSED_OPTS))
@pytest.mark.parametrize("extra", ["plain", "nug", "euler_a", "euler_b"])
@pytest.mark.parametrize("kernel", sorted(KERNELS))
def test_fused_vs_staged_and_oracle(shape, name, extra, kernel):
    opts = FUSED_OPTS[name]
    rng = np.random.default_rng(zlib.crc32(repr((shape, name, extra)).encode()))
    gc = nondivergent(shape, rng, 0.35)
    psi = boxes(shape, rng) if rng.uniform() < 0.5 else smooth_positive(shape, rng)
    if opts & capi.IGA:
        psi = psi - 2.5
    G = 1.0 + 0.3 * rng.uniform(size=shape) if extra == "nug" else None
    R = rng.normal(size=shape) if extra.startswith("euler") else None
    rhs = extra if extra.startswith("euler") else "euler_a"
    o = opts | (capi.RHS_EULER_A if extra == "euler_a" else capi.RHS_EULER_B if extra == "euler_b" else 0)
    n = 5
    key = (shape, name, extra)
    p32, g32, G32, R32 = r32(psi), [r32(v) for v in gc], r32(G), r32(R)
    if key not in _ORACLE:
        _ORACLE[key] = (
            oracle.step(psi, gc, g=G, r=R, dt=0.1, n_iters=2, opts=opts, n_steps=n, rhs=rhs),
            oracle.step(p32, g32, g=G32, r=R32, dt=np.float32(0.1), n_iters=2, opts=opts, n_steps=n, rhs=rhs),
            gpu_run(psi, gc, G, R, 0.1, o, n, torch.float64, True))
    ref, ref32, s64 = _ORACLE[key]
    # FP64: fused == oracle to 1e-12, fused ~ staged to 1e-13
    f64 = gpu_run(psi, gc, G, R, 0.1, o, n, torch.float64, False, kernel)
    scale = np.abs(ref).max()
    assert np.abs(f64 - ref).max() <= 1e-12 * scale
    assert np.abs(f64 - s64).max() <= 1e-13 * scale
    # FP32: relative L2 against the oracle on the same rounded inputs
    f32 = gpu_run(p32, g32, G32, R32, 0.1, o, n, torch.float32, False, kernel)
    assert np.linalg.norm(f32 - ref32) <= 1e-5 * np.linalg.norm(ref32)


@pytest.mark.parametrize("shape", [(3, 130), (1, 64), (300, 250)], ids=lambda s: f"{s[0]}x{s[1]}")
@pytest.mark.parametrize("kernel", sorted(KERNELS))
def test_fused_time_dependent_advector(shape, kernel):
    """Per-step advector multipliers (gc_scale) with FCT: each step against an oracle step
    on gc * scale_s; also fields of 1 and 3 rows (shorter than the stencil's halo)."""
    rng = np.random.default_rng(sum(shape))
    gc = nondivergent(shape, rng, 0.3)
    psi = smooth_positive(shape, rng)
    scales = [1.0, 0.5, -0.75, 1.25]
    ref = psi
    for s in scales:
        ref = oracle.step(ref, [v * s for v in gc], n_iters=2, opts=oracle.FCT)
    f64 = gpu_run(psi, gc, None, None, 0.0, capi.FCT, len(scales), torch.float64, False, kernel,
                  np.array(scales))
    assert np.abs(f64 - ref).max() <= 1e-12 * np.abs(ref).max()
    f32 = gpu_run(r32(psi), [r32(v) for v in gc], None, None, 0.0, capi.FCT, len(scales), torch.float32,
                  False, kernel, np.array(scales))
    assert np.linalg.norm(f32 - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("kernel", ["warp", "band", "warp2"])
def test_rotation_1024_short_run(dtype, kernel):
    """Full-size 2D rotation workload (1024^2, FCT, two passes) for 10 steps in the
    launch configuration the benchmark times, against the oracle element by element."""
    psi, gc, _ = workloads.rotation_2d(1024)
    if dtype == torch.float32:
        psi, gc = r32(psi), [r32(v) for v in gc]
    oracle.set_threads(0)
    ref = oracle.step(psi, gc, n_iters=2, opts=oracle.FCT, n_steps=10)
    out = gpu_run(psi, gc, None, None, 0.0, capi.FCT, 10, dtype, False, kernel)
    if dtype == torch.float64:
        assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()
    else:
        assert np.linalg.norm(out - ref) <= 1e-5 * np.linalg.norm(ref)
        assert abs(out.sum() - ref.sum()) <= 1e-6 * np.abs(ref).sum()


@pytest.mark.parametrize("name", sorted(FUSED_OPTS))
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_kernel_families_agree(name, dtype):
    """Band heights change the band march's schedule, not its arithmetic: bit-equal
    results.  The warp march evaluates the same expressions in the same order, but the
    compiler fuses multiply-adds differently in the two kernels, so across families
    the results agree to rounding (FP64 1e-14 max-norm, FP32 1e-6 relative L2)."""
    shape = (203, 261)
    rng = np.random.default_rng(7)
    gc = nondivergent(shape, rng, 0.4)
    psi = smooth_positive(shape, rng) - (2.5 if FUSED_OPTS[name] & capi.IGA else 0.0)
    run = lambda k: gpu_run(psi, gc, None, None, 0.0, FUSED_OPTS[name], 7, dtype, False, k)
    band = run("band")
    for k in ("band_h5", "band_h64"):
        assert np.array_equal(run(k), band)
    for k in ("warp", "warp2"):  # lanes of 4 (FP64: 2) and of 2 columns
        warp = run(k)
        if dtype == torch.float64:
            assert np.abs(warp - band).max() <= 1e-14 * np.abs(band).max(), k
        else:
            assert np.linalg.norm(warp - band) <= 1e-6 * np.linalg.norm(band), k
