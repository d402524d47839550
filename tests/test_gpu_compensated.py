"""mpdata_advance_compensated: the fused 2D step on an FP32 state carried as hi + lo.

The arithmetic of the step is FP32 (as mpdata_advance); only the state keeps the rounding
error of the donor-cell updates. Checks: parity with the FP64 oracle on short runs (tighter
than plain FP32), conservation of sum(hi + lo) to round-off of the small parts, a long
rotation run whose error against the oracle stays below plain FP32's, in-place stepping,
and argument validation.
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


def split(x):
    """FP64 field -> (hi, lo) FP32 tensors with hi + lo = x to ~1e-14 relative."""
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return torch.tensor(hi, device=DEV), torch.tensor(lo, device=DEV)


def joined(hi, lo):
    return hi.double().cpu().numpy() + lo.double().cpu().numpy()


def run_comp(psi, gc, steps, opts, G=None, R=None, dt=0.0, scale=None, rows=0, kernel=0):
    f = lambda a: None if a is None else torch.tensor(a, dtype=torch.float32, device=DEV)
    o = opts | (capi.NUG if G is not None else 0)
    with Mpdata(psi.shape, dtype=torch.float32, n_iters=2, opts=o) as m:
        m.tune(capi.TUNE_KERNEL, kernel)
        m.tune(capi.TUNE_TILE_ROWS, rows)
        hi, lo = split(psi)
        ho, lout = torch.empty_like(hi), torch.empty_like(lo)
        m.advance_compensated(hi, lo, ho, lout, [f(v) for v in gc], f(G), f(R), dt, steps, scale)
        torch.cuda.synchronize()
        return ho, lout


def run_plain32(psi, gc, steps, opts):
    f = lambda a: torch.tensor(a, dtype=torch.float32, device=DEV)
    with Mpdata(psi.shape, dtype=torch.float32, n_iters=2, opts=opts) as m:
        a, b = f(psi), torch.empty(psi.shape, dtype=torch.float32, device=DEV)
        m.advance(a, b, [f(v) for v in gc], n_steps=steps)
        torch.cuda.synchronize()
        return b.double().cpu().numpy()


r32 = lambda a: None if a is None else a.astype(np.float32).astype(np.float64)

OPTS = {"basic": 0, "fct": capi.FCT, "iga_fct": capi.IGA | capi.FCT}


@pytest.mark.parametrize("shape", [(200, 130), (57, 123), (9, 250)], ids=lambda s: f"{s[0]}x{s[1]}")
@pytest.mark.parametrize("name", sorted(OPTS))
@pytest.mark.parametrize("extra", ["plain", "nug", "euler_a", "euler_b"])
@pytest.mark.parametrize("rows,kernel", [(0, 0), (5, 0), (0, 3), (12, 3)], ids=lambda v: str(v))
def test_short_run_parity(shape, name, extra, rows, kernel):
    """kernel 3: lanes of 2 columns (taken for FCT without G; other options fall back to 4)."""
    opts = OPTS[name]
    rng = np.random.default_rng(zlib.crc32(repr((shape, name, extra)).encode()))
    gc = [r32(v) for v in nondivergent(shape, rng, 0.35)]
    psi = boxes(shape, rng) if rng.uniform() < 0.5 else smooth_positive(shape, rng)
    if opts & capi.IGA:
        psi = psi - 2.5
    G = r32(1.0 + 0.3 * rng.uniform(size=shape)) if extra == "nug" else None
    R = r32(rng.normal(size=shape)) if extra.startswith("euler") else None
    rhs = extra if extra.startswith("euler") else "euler_a"
    o = opts | (capi.RHS_EULER_A if extra == "euler_a" else capi.RHS_EULER_B if extra == "euler_b" else 0)
    dt = float(np.float32(0.1))
    hi, lo = run_comp(psi, gc, 5, o, G, R, dt, rows=rows, kernel=kernel)
    ref = oracle.step(psi, gc, g=G, r=R, dt=dt, n_iters=2, opts=opts, n_steps=5, rhs=rhs)
    got = joined(hi, lo)
    assert np.linalg.norm(got - ref) <= 2e-6 * np.linalg.norm(ref)
    # the pair is renormalised: lo is below one unit in the last place of hi
    h = hi.cpu().numpy()
    assert np.all(np.abs(lo.cpu().numpy()) <= np.spacing(np.abs(h)) + 1e-38)


def test_mass_conserved_to_roundoff_of_the_low_parts():
    """Rotation workload, 256^2, FCT, 400 steps: sum(hi + lo) against the start, next to the
    plain FP32 state's drift (G = 1: the mass is the plain sum)."""
    psi, gc, _ = workloads.rotation_2d(256)
    gc = [r32(v) for v in gc]
    hi, lo = run_comp(psi, gc, 400, capi.FCT)
    m0 = psi.sum()
    drift_comp = abs(joined(hi, lo).sum() - m0) / m0
    h2, l2 = run_comp(psi, gc, 400, capi.FCT, kernel=3)  # lanes of 2 columns
    assert abs(joined(h2, l2).sum() - m0) / m0 <= 1e-11
    drift_plain = abs(run_plain32(r32(psi), gc, 400, capi.FCT).sum() - r32(psi).sum()) / m0
    assert drift_comp <= 1e-11, (drift_comp, drift_plain)
    assert drift_comp < 1e-2 * max(drift_plain, 1e-12)


def test_long_run_error_below_plain_fp32():
    """Rotation 256^2, FCT, 1500 steps against the FP64 oracle on the same (FP32-representable)
    advector: the compensated state's error is below the plain FP32 state's (what remains is
    the FP32 arithmetic of the fluxes and the limiter, which the compensation leaves as it is;
    its main gain is mass conservation)."""
    psi, gc, _ = workloads.rotation_2d(256)
    gc = [r32(v) for v in gc]
    oracle.set_threads(0)
    ref = oracle.step(psi, gc, n_iters=2, opts=oracle.FCT, n_steps=1500)
    hi, lo = run_comp(psi, gc, 1500, capi.FCT)
    err_comp = np.linalg.norm(joined(hi, lo) - ref) / np.linalg.norm(ref)
    err_plain = np.linalg.norm(run_plain32(r32(psi), gc, 1500, capi.FCT) - ref) / np.linalg.norm(ref)
    assert err_comp < err_plain, (err_comp, err_plain)
    assert err_comp <= 1e-5


def test_one_revolution_256_against_oracle():
    """The rotation workload at 256^2 (FCT, two passes) over one full revolution (1609 steps),
    both FP32 paths against the FP64 oracle on the same FP32-representable input: the
    compensated state keeps the FP32 bars (relative L2 <= 1e-5, relative mass drift <= 1e-6);
    the plain FP32 state's errors are checked against the bars it reaches at this size."""
    psi, gc, rev = workloads.rotation_2d(256)
    assert rev == workloads.rotation_steps(256) == 1609
    psi, gc = r32(psi), [r32(v) for v in gc]
    oracle.set_threads(0)
    ref = oracle.step(psi, gc, n_iters=2, opts=oracle.FCT, n_steps=rev)
    m0 = psi.sum()
    hi, lo = run_comp(psi, gc, rev, capi.FCT)
    comp = joined(hi, lo)
    plain = run_plain32(psi, gc, rev, capi.FCT)
    l2 = lambda x: float(np.linalg.norm(x - ref) / np.linalg.norm(ref))
    drift = lambda x: float(abs(x.sum() - m0) / abs(m0))
    assert l2(comp) <= 1e-5 and drift(comp) <= 1e-6, (l2(comp), drift(comp))
    assert l2(plain) <= 1e-5 and drift(plain) <= 1e-6, (l2(plain), drift(plain))
    assert drift(comp) < drift(plain)


def test_in_place_odd_steps_and_time_dependent_scale():
    shape = (96, 136)
    rng = np.random.default_rng(5)
    gc = [r32(v) for v in nondivergent(shape, rng, 0.3)]
    psi = smooth_positive(shape, rng)
    scales = [1.0, -0.5, 0.75]
    ho, lo_ = run_comp(psi, gc, 3, capi.FCT, scale=scales)
    f = lambda a: torch.tensor(a, dtype=torch.float32, device=DEV)
    with Mpdata(shape, dtype=torch.float32, n_iters=2, opts=capi.FCT) as m:
        hi, lo = split(psi)
        m.advance_compensated(hi, lo, hi, lo, [f(v) for v in gc], n_steps=3, gc_scale=scales)
        torch.cuda.synchronize()
    assert torch.equal(hi, ho) and torch.equal(lo, lo_)
    ref = psi
    for s in scales:
        ref = oracle.step(ref, [v * s for v in gc], n_iters=2, opts=oracle.FCT)
    assert np.linalg.norm(joined(hi, lo) - ref) <= 2e-6 * np.linalg.norm(ref)


def test_rejected_configurations():
    z2 = lambda dt=torch.float32: torch.zeros(16, 16, dtype=dt, device=DEV)
    with Mpdata((16, 16), dtype=torch.float64, n_iters=2, opts=capi.FCT) as m:
        a = z2(torch.float64)
        assert capi.mpdata_advance_compensated(m.h, a, a, a, a, [a, a], raw=True) == capi.EUNSUPPORTED
    with Mpdata((16, 16), dtype=torch.float32, n_iters=3, opts=capi.FCT) as m:
        a = z2()
        assert capi.mpdata_advance_compensated(m.h, a, z2(), z2(), z2(), [a, a], raw=True) == capi.EUNSUPPORTED
    with Mpdata((16, 16), dtype=torch.float32, n_iters=2, opts=capi.FCT) as m:
        a, b, c = z2(), z2(), z2()
        # psi in place but lo out of place
        assert capi.mpdata_advance_compensated(m.h, a, b, a, c, [a, a], raw=True) == capi.EINVAL
        assert capi.mpdata_advance_compensated(m.h, a, None, b, c, [a, a], raw=True) == capi.EINVAL
    with Mpdata((8, 8, 8), dtype=torch.float32, n_iters=2, opts=capi.FCT) as m:
        a = torch.zeros(8, 8, 8, device=DEV)
        assert capi.mpdata_advance_compensated(m.h, a, a.clone(), a.clone(), a.clone(), [a, a, a],
                                               raw=True) == capi.EUNSUPPORTED
