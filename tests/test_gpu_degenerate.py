"""Degenerate cases of the method on every GPU path (warp march, band march, staged kernels,
compensated state): no flow, a constant field, a zero field, and the one-cell shift at
Courant number 1 (Sect. 3.1.1: the donor-cell flux then moves each cell's content exactly
one cell; the pseudo-advector (|V| - V^2) A vanishes, so the corrective pass adds nothing).
"""
import numpy as np
import pytest
import torch

from helpers import nondivergent, smooth_positive
from paper_1407_1309_gb300 import capi
from paper_1407_1309_gb300.solver import Mpdata

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")
PATHS = {"warp": (1, 0), "band": (2, 0), "staged": (None, capi.STAGED)}


def run(psi, gc, path, opts, dtype=torch.float64, steps=3):
    fam, extra = PATHS[path]
    with Mpdata(psi.shape, dtype=dtype, n_iters=2, opts=opts | extra) as m:
        if fam is not None:
            m.tune(capi.TUNE_KERNEL, fam)
        a = torch.tensor(psi, dtype=dtype, device=DEV)
        b = torch.empty_like(a)
        m.advance(a, b, [torch.tensor(v, dtype=dtype, device=DEV) for v in gc], n_steps=steps)
        torch.cuda.synchronize()
        return b.cpu().numpy()


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("opts", [0, capi.FCT, capi.FCT | capi.IGA], ids=["basic", "fct", "iga_fct"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_no_flow_leaves_the_field_unchanged(path, opts, dtype):
    shape = (67, 131)
    psi = smooth_positive(shape, np.random.default_rng(0))
    if opts & capi.IGA:
        psi = psi - 2.0
    psi = psi.astype(np.float32).astype(np.float64) if dtype == torch.float32 else psi
    out = run(psi, [np.zeros(shape), np.zeros(shape)], path, opts, dtype)
    assert np.array_equal(out, psi)


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("opts", [0, capi.FCT], ids=["basic", "fct"])
def test_constant_and_zero_fields_under_nondivergent_flow(path, opts):
    shape = (96, 150)
    gc = nondivergent(shape, np.random.default_rng(1), 0.45)
    const = run(np.full(shape, 3.25), gc, path, opts, steps=5)
    assert np.abs(const - 3.25).max() <= 1e-14 * 3.25
    zero = run(np.zeros(shape), gc, path, opts, steps=5)
    assert np.array_equal(zero, np.zeros(shape))


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("axis", [0, 1])
def test_unit_courant_number_shifts_by_one_cell(path, axis):
    shape = (40, 136)
    psi = smooth_positive(shape, np.random.default_rng(2))
    gc = [np.zeros(shape), np.zeros(shape)]
    gc[axis][:] = 1.0
    out = run(psi, gc, path, capi.FCT, steps=3)
    ref = np.roll(psi, 3, axis=axis)
    if path == "staged":  # the oracle's summation order psi - F_out + F_in: exact
        assert np.array_equal(out, ref)
    else:  # fused kernels add the flux differences first: one rounding per step
        assert np.abs(out - ref).max() <= 4 * np.spacing(np.abs(ref).max())


def test_compensated_state_no_flow_and_unit_shift():
    shape = (64, 128)
    psi = smooth_positive(shape, np.random.default_rng(3))
    hi = psi.astype(np.float32)
    lo = (psi - hi.astype(np.float64)).astype(np.float32)
    for gc0, expect in ((0.0, psi), (1.0, np.roll(psi, 2, axis=0))):
        with Mpdata(shape, dtype=torch.float32, n_iters=2, opts=capi.FCT) as m:
            th, tl = torch.tensor(hi, device=DEV), torch.tensor(lo, device=DEV)
            oh, ol = torch.empty_like(th), torch.empty_like(tl)
            g = [torch.full(shape, gc0, device=DEV), torch.zeros(shape, device=DEV)]
            m.advance_compensated(th, tl, oh, ol, g, n_steps=2)
            torch.cuda.synchronize()
            got = oh.double().cpu().numpy() + ol.double().cpu().numpy()
        assert np.abs(got - expect).max() <= 1e-13 * np.abs(expect).max()
