"""The 3D configuration (deformational flow, Sect. 3.7 style: n_iters = 3 with the third-order
terms, FCT and non-unit G; the infinite-gauge variant with n_iters = 2 on a variable-sign field)
on the GPU against the FP64 oracle, element by element.

The shapes cross every seam of the 3D kernels: x extents above the 32-column tile and not a
multiple of it, y extents above the 8-row tile, z extents above the 16-plane chunk and not a
multiple of it.  The deformational workload itself runs at 64^3 for 20 steps and at the full
256^3 for 2 steps, with the per-step advector factor cos(pi t / T) evaluated at n + 1/2.
Bars: FP64 max-norm relative error <= 1e-12; FP32 relative L2 error <= 1e-5 and relative mass
drift <= 1e-6 (inputs rounded to FP32 on both sides).
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import nondivergent, smooth_positive
from paper_1407_1309_gb300 import capi, workloads
from paper_1407_1309_gb300.solver import Mpdata

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")

CASES = {
    "tot3_fct_G": (3, capi.TOT | capi.FCT | capi.NUG),
    "iga_tot_fct_G": (2, capi.IGA | capi.TOT | capi.FCT | capi.NUG),
    "tot3_fct": (3, capi.TOT | capi.FCT),
    "it2_fct": (2, capi.FCT),
}
# (z, y, x): x above 32 and ragged, y above 8, z above 16 and ragged (scalar z-march); x a
# multiple of 4 above the 128-cell tiles of the vectorised z-march, the last tile partial; for
# the vectorised kernels also one plane of one row (every halo row and plane wraps onto the
# cell's own), a chunk shorter than 16 planes with fewer rows than a tile, and three tiles with
# a 4-cell tail
SEAM_SHAPES = [(37, 19, 70), (17, 9, 33), (33, 17, 65), (37, 19, 136), (17, 9, 260), (21, 11, 68), (18, 3, 4),
               (1, 1, 132), (5, 3, 128), (18, 9, 388)]


def rounded(a, dtype):
    if a is None:
        return None
    return a.astype(np.float32).astype(np.float64) if dtype == torch.float32 else a


def gpu_run(psi, gc, G, n_iters, opts, scales, dtype):
    t = lambda a: None if a is None else torch.tensor(a, dtype=dtype, device=DEV)
    with Mpdata(psi.shape, dtype=dtype, n_iters=n_iters, opts=opts) as m:
        p = t(psi)
        out = torch.empty_like(p)
        g = t(G)
        m.advance(p, out, [t(v) for v in gc], n_steps=len(scales), g=g, gc_scale=list(scales))
        torch.cuda.synchronize()
        mass = m.mass(out, g)
        return out.double().cpu().numpy(), mass


def oracle_run(psi, gc, G, n_iters, opts, scales):
    ref = psi
    o = int(opts) & ~capi.NUG
    for s in scales:
        ref = oracle.step(ref, [v * s for v in gc], g=G, n_iters=n_iters, opts=o)
    return ref


def check(out, ref, dtype, m_gpu=None, G=None):
    if dtype == torch.float64:
        err = np.abs(out - ref).max() / np.abs(ref).max()
        assert err <= 1e-12, err
    else:
        l2 = np.linalg.norm(out - ref) / np.linalg.norm(ref)
        assert l2 <= 1e-5, l2
        if m_gpu is not None:
            m0 = oracle.mass(ref, G)
            assert abs(m_gpu - m0) <= 1e-6 * oracle.mass(np.abs(ref), G)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("shape", SEAM_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("name", sorted(CASES))
def test_3d_tile_seams_match_oracle(name, shape, dtype):
    n_iters, opts = CASES[name]
    rng = np.random.default_rng(sum(shape))
    gc = nondivergent(shape, rng, 0.35)
    psi = smooth_positive(shape, rng)
    if opts & capi.IGA:
        psi = psi - 2.0  # variable sign
    G = 1.0 + 0.2 * rng.uniform(size=shape) if opts & capi.NUG else None
    psi, gc, G = rounded(psi, dtype), [rounded(v, dtype) for v in gc], rounded(G, dtype)
    scales = [1.0, 0.75, -0.5, 1.0, 0.875]
    out, m = gpu_run(psi, gc, G, n_iters, opts, scales, dtype)
    ref = oracle_run(psi, gc, G, n_iters, opts, scales)
    check(out, ref, dtype, m, G)


def _deform(n, iga, dtype):
    psi, gc, G = workloads.deformational_3d(n, iga=iga)
    return rounded(psi, dtype), [rounded(v, dtype) for v in gc], rounded(G, dtype)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("iga", [False, True], ids=["tot3_fct", "iga_tot_fct"])
def test_deformational_64_cubed_20_steps_match_oracle(iga, dtype):
    n_iters, opts = (2, capi.IGA | capi.TOT | capi.FCT | capi.NUG) if iga else (3, capi.TOT | capi.FCT | capi.NUG)
    psi, gc, G = _deform(64, iga, dtype)
    scales = [workloads.deformational_scale(s) for s in range(20)]
    out, m = gpu_run(psi, gc, G, n_iters, opts, scales, dtype)
    ref = oracle_run(psi, gc, G, n_iters, opts, scales)
    check(out, ref, dtype, m, G)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_deformational_256_cubed_matches_oracle(dtype):
    """The full 3D workload (256^3, n_iters = 3 + tot + FCT + G), two steps, every cell."""
    n_iters, opts = 3, capi.TOT | capi.FCT | capi.NUG
    psi, gc, G = _deform(256, False, dtype)
    scales = [workloads.deformational_scale(s) for s in range(2)]
    out, m = gpu_run(psi, gc, G, n_iters, opts, scales, dtype)
    ref = oracle_run(psi, gc, G, n_iters, opts, scales)
    check(out, ref, dtype, m, G)
