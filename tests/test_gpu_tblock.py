"""Temporal blocking (MPDATA_TUNE_STEPS_PER_LAUNCH = 2..4: several MPDATA steps per launch)
against the FP64 oracle, element by element, and against one step per launch.

Shapes: several 32-cell output tiles with ragged last tiles in both dimensions, fields
narrower than the 3S-cell halo (the periodic wrap then reaches around the field more than
once), a single row, and the full 1024^2 rotation workload in the launch configuration the
benchmark times.  Step counts leave a remainder group at every depth; in-place calls with an
odd number of groups go through the ping-pong copy; per-step advector factors (gc_scale)
reach every sub-step of a launch.
Bars: FP64 max-norm relative error <= 1e-12; FP32 relative L2 error <= 1e-5 and relative mass
drift <= 1e-6 (inputs rounded to FP32 on both sides).
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
DEV = torch.device("cuda")

OPTS = {"basic": 0, "fct": capi.FCT, "iga_fct": capi.IGA | capi.FCT, "iga": capi.IGA}
SHAPES = [(70, 45), (33, 97), (64, 64), (5, 7), (1, 40), (130, 3)]


def r32(a):
    return None if a is None else a.astype(np.float32).astype(np.float64)


def gpu_run(psi, gc, opts, n_steps, dtype, depth, gc_scale=None, in_place=False):
    t = lambda a: torch.tensor(a, dtype=dtype, device=DEV)
    with Mpdata(psi.shape, dtype=dtype, n_iters=2, opts=opts) as m:
        m.tune(capi.TUNE_STEPS_PER_LAUNCH, depth)
        a = t(psi)
        b = a if in_place else torch.empty_like(a)
        m.advance(a, b, [t(v) for v in gc], None, None, 0.0, n_steps, gc_scale)
        torch.cuda.synchronize()
        return b.cpu().numpy().astype(np.float64), m.mass(b)


def inputs(shape, name, seed_extra=""):
    rng = np.random.default_rng(zlib.crc32(repr((shape, name, seed_extra)).encode()))
    gc = nondivergent(shape, rng, 0.4)
    psi = boxes(shape, rng) if rng.uniform() < 0.5 else smooth_positive(shape, rng)
    if OPTS[name] & capi.IGA:
        psi = psi - 2.5  # variable sign
    return psi, gc


def check(out, ref, dtype, mass=None):
    if dtype == torch.float64:
        assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()
    else:
        assert np.linalg.norm(out - ref) <= 1e-5 * np.linalg.norm(ref)
        if mass is not None:
            assert abs(mass - ref.sum()) <= 1e-6 * np.abs(ref).sum()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("depth", [2, 3, 4])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}")
@pytest.mark.parametrize("name", sorted(OPTS))
def test_depth_matches_oracle(name, shape, depth, dtype):
    psi, gc = inputs(shape, name)
    if dtype == torch.float32:
        psi, gc = r32(psi), [r32(v) for v in gc]
    n = 7  # a remainder group at depths 2, 3 and 4
    ref = oracle.step(psi, gc, n_iters=2, opts=OPTS[name], n_steps=n)
    out, mass = gpu_run(psi, gc, OPTS[name], n, dtype, depth)
    check(out, ref, dtype, mass)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("depth", [2, 4])
def test_depth_with_time_dependent_advector_and_in_place(depth, dtype):
    """Per-step factors on the advector reach each sub-step of a launch; in place with an odd
    number of groups (5 steps at depth 2 and 4: 3 and 2 groups) and an even one."""
    shape = (97, 70)
    psi, gc = inputs(shape, "fct", "scale")
    if dtype == torch.float32:
        psi, gc = r32(psi), [r32(v) for v in gc]
    scales = [1.0, 0.5, -0.75, 1.25, 0.875]
    ref = psi
    for s in scales:
        ref = oracle.step(ref, [v * s for v in gc], n_iters=2, opts=oracle.FCT)
    for in_place in (False, True):
        out, mass = gpu_run(psi, gc, capi.FCT, len(scales), dtype, depth, np.array(scales), in_place)
        check(out, ref, dtype, mass)


@pytest.mark.parametrize("name", sorted(OPTS))
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_depths_agree_with_one_step_per_launch(name, dtype):
    """The blocked kernel evaluates the warp march's expressions in the same order; depths
    1..4 agree to rounding (FP64 1e-14 max-norm, FP32 1e-6 relative L2)."""
    shape = (203, 261)
    psi, gc = inputs(shape, name, "agree")
    base, _ = gpu_run(psi, gc, OPTS[name], 8, dtype, 1)
    for depth in (2, 3, 4):
        out, _ = gpu_run(psi, gc, OPTS[name], 8, dtype, depth)
        if dtype == torch.float64:
            assert np.abs(out - base).max() <= 1e-14 * np.abs(base).max(), depth
        else:
            assert np.linalg.norm(out - base) <= 1e-6 * np.linalg.norm(base), depth


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("depth", [2, 4])
def test_rotation_1024_at_depth(depth, dtype):
    """The full-size rotation workload (1024^2, FCT, two passes), 8 steps at the given depth,
    against the oracle element by element."""
    psi, gc, _ = workloads.rotation_2d(1024)
    if dtype == torch.float32:
        psi, gc = r32(psi), [r32(v) for v in gc]
    oracle.set_threads(0)
    ref = oracle.step(psi, gc, n_iters=2, opts=oracle.FCT, n_steps=8)
    out, mass = gpu_run(psi, gc, capi.FCT, 8, dtype, depth)
    check(out, ref, dtype, mass)


def test_depth_is_ignored_where_the_kernel_does_not_apply():
    """Options outside the blocked kernel (G, third-order terms) run one step per launch at
    any depth setting, with unchanged results."""
    shape = (40, 50)
    rng = np.random.default_rng(3)
    gc = nondivergent(shape, rng, 0.3)
    psi = smooth_positive(shape, rng)
    G = 1.0 + 0.2 * rng.uniform(size=shape)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device=DEV)
    outs = []
    for depth in (1, 4):
        with Mpdata(shape, dtype=torch.float64, n_iters=2, opts=capi.FCT | capi.NUG) as m:
            m.tune(capi.TUNE_STEPS_PER_LAUNCH, depth)
            b = torch.empty_like(t(psi))
            m.advance(t(psi), b, [t(v) for v in gc], t(G), None, 0.0, 5)
            torch.cuda.synchronize()
            outs.append(b.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    ref = oracle.step(psi, gc, g=G, n_iters=2, opts=oracle.FCT, n_steps=5)
    assert np.abs(outs[1] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_depth_knob_rejects_values_out_of_range():
    with Mpdata((8, 8), dtype=torch.float32, n_iters=2, opts=capi.FCT) as m:
        for bad in (-1, 5):
            with pytest.raises(RuntimeError):
                m.tune(capi.TUNE_STEPS_PER_LAUNCH, bad)
        for good in (0, 1, 2, 3, 4):
            m.tune(capi.TUNE_STEPS_PER_LAUNCH, good)
