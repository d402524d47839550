"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

Bars: FP64 max-norm relative error <= 1e-12; FP32 relative L2 error <= 1e-5 and
relative mass drift <= 1e-6, both sides fed the same (FP32-rounded) inputs.
Sizes are small, ragged and degenerate (extents 1 and 2, extents not multiples
of any tile, extents below the halo radius) so the oracle finishes in seconds.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import boxes, nondivergent, smooth_positive
from paper_1407_1309_gb300 import capi, workloads
from paper_1407_1309_gb300.solver import Mpdata

pytestmark = pytest.mark.gpu

OPTS = {
    "donor": (1, 0),
    "basic": (2, 0),
    "fct": (2, capi.FCT),
    "it3_fct": (3, capi.FCT),
    "tot3_fct": (3, capi.TOT | capi.FCT),
    "tot2": (2, capi.TOT),
    "iga_fct": (2, capi.IGA | capi.FCT),
    "iga_tot_fct": (2, capi.IGA | capi.TOT | capi.FCT),
    "kahan_fct": (2, capi.KAHAN | capi.FCT),
}
# the oracle's option bits have the same values as the library's
SHAPES = [(37,), (2,), (1,), (12, 9), (33, 70), (2, 3), (1, 5), (6, 5, 7), (9, 4, 11), (2, 1, 3)]
FP64_TOL = 1e-12
FP32_L2 = 1e-5
FP32_MASS = 1e-6


def make_inputs(shape, seed, nug, rhs, sign="pos"):
    rng = np.random.default_rng(seed)
    gc = nondivergent(shape, rng, 0.3)
    psi = boxes(shape, rng) if seed % 2 == 0 else smooth_positive(shape, rng)
    if sign == "var":
        psi = psi - 2.5
    G = 1.0 + 0.3 * rng.uniform(size=shape) if nug else None
    R = rng.normal(size=shape) if rhs else None
    return psi, gc, G, R


def run_gpu(psi, gc, G, R, dt, n_iters, opts, n_steps, dtype, rhs="euler_a"):
    dev = torch.device("cuda")
    t = lambda a: None if a is None else torch.tensor(a, dtype=dtype, device=dev)
    o = opts | (capi.NUG if G is not None else 0)
    if R is not None:
        o |= capi.RHS_EULER_A if rhs == "euler_a" else capi.RHS_EULER_B
    with Mpdata(psi.shape, dtype=dtype, n_iters=n_iters, opts=o) as m:
        p = t(psi)
        m.step(p, [t(v) for v in gc], t(G), t(R), dt, n_steps)
        torch.cuda.synchronize()
        mass = m.mass(p, t(G))
        return p.cpu().numpy().astype(np.float64), mass


def rounded(a, dtype):
    if a is None:
        return None
    return a.astype(np.float32).astype(np.float64) if dtype == torch.float32 else a


def check(out, ref, dtype, m_gpu=None, m0=None, scale=None):
    """FP64: max-norm relative error; FP32: relative L2 error and mass drift relative to
    sum |G psi| (the field's scale: a variable-sign field can have zero net mass)."""
    if dtype == torch.float64:
        err = np.abs(out - ref).max() / max(np.abs(ref).max(), 1e-300)
        assert err <= FP64_TOL, err
    else:
        l2 = np.linalg.norm(out - ref) / max(np.linalg.norm(ref), 1e-300)
        assert l2 <= FP32_L2, l2
        if m_gpu is not None:
            assert abs(m_gpu - m0) <= FP32_MASS * (scale if scale is not None else abs(m0))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("name", sorted(OPTS))
def test_parity_vs_oracle(name, shape, dtype):
    n_iters, opts = OPTS[name]
    sign = "var" if opts & capi.IGA else "pos"
    for seed, nug, rhs in ((0, False, None), (1, True, None), (2, False, "euler_a"), (3, True, "euler_b")):
        psi, gc, G, R = make_inputs(shape, seed, nug, rhs is not None, sign)
        psi, gc, G, R = rounded(psi, dtype), [rounded(v, dtype) for v in gc], rounded(G, dtype), rounded(R, dtype)
        dt = 0.125
        n_steps = 7
        out, m_gpu = run_gpu(psi, gc, G, R, dt, n_iters, opts, n_steps, dtype, rhs or "euler_a")
        ref = oracle.step(psi, gc, g=G, r=R, dt=dt, n_iters=n_iters, opts=opts, n_steps=n_steps,
                          rhs=rhs or "euler_a")
        m0 = oracle.mass(ref, G)
        check(out, ref, dtype, m_gpu, m0, oracle.mass(np.abs(ref), G))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("staged", [False, True], ids=["auto", "staged"])
def test_rotation_config_small(dtype, staged):
    """The solid-body-rotation workload (cone, FCT, two passes) at 64^2 for 100 steps."""
    from paper_1407_1309_gb300 import workloads as wl
    psi, gc, _ = wl.rotation_2d(64)
    psi, gc = rounded(psi, dtype), [rounded(v, dtype) for v in gc]
    out, m = run_gpu(psi, gc, None, None, 0.0, 2, capi.FCT | (capi.STAGED if staged else 0), 100, dtype)
    ref = oracle.step(psi, gc, n_iters=2, opts=oracle.FCT, n_steps=100)
    check(out, ref, dtype, m, oracle.mass(psi))


def test_inplace_out_of_place_and_step_splitting_agree():
    """advance(in, out) == step in place; n steps in one call == n calls of one step (bitwise)."""
    rng = np.random.default_rng(5)
    shape = (40, 33)
    gc = [torch.tensor(v, dtype=torch.float32, device="cuda") for v in nondivergent(shape, rng, 0.4)]
    psi0 = torch.tensor(boxes(shape, rng), dtype=torch.float32, device="cuda")
    for n_iters, opts in OPTS.values():
        with Mpdata(shape, dtype=torch.float32, n_iters=n_iters, opts=opts) as m:
            a = psi0.clone()
            m.step(a, gc, n_steps=3)
            b = torch.empty_like(psi0)
            m.advance(psi0, b, gc, n_steps=3)
            c = psi0.clone()
            for _ in range(3):
                m.step(c, gc)
            torch.cuda.synchronize()
            assert torch.equal(a, b) and torch.equal(a, c)


def test_time_dependent_advector_scale():
    """gc_scale[s] multiplies the advector of step s (flow evaluated at the half step)."""
    rng = np.random.default_rng(6)
    shape = (20, 17)
    gc = nondivergent(shape, rng, 0.4)
    psi = smooth_positive(shape, rng)
    scales = [0.9, -0.4, 0.2]
    dev = torch.device("cuda")
    with Mpdata(shape, dtype=torch.float64, n_iters=2, opts=capi.FCT) as m:
        a = torch.tensor(psi, device=dev)
        out = torch.empty_like(a)
        m.advance(a, out, [torch.tensor(v, device=dev) for v in gc], n_steps=3, gc_scale=scales)
        got = out.cpu().numpy()
    ref = psi.copy()
    for s in scales:
        ref = oracle.step(ref, [v * s for v in gc], n_iters=2, opts=oracle.FCT)
    assert np.abs(got - ref).max() <= FP64_TOL * np.abs(ref).max()


def test_reductions_match_fp64_sums():
    rng = np.random.default_rng(7)
    shape = (50, 41)
    a, b, G = rng.normal(size=shape), rng.normal(size=shape), rng.uniform(0.5, 1.5, size=shape)
    dev = torch.device("cuda")
    with Mpdata(shape, dtype=torch.float64) as m:
        ta, tb, tg = (torch.tensor(x, device=dev) for x in (a, b, G))
        assert abs(m.mass(ta) - a.sum()) <= 1e-13 * np.abs(a).sum()
        assert abs(m.mass(ta, tg) - (a * G).sum()) <= 1e-13 * np.abs(a * G).sum()
        l2, li = m.diff_norms(ta, tb)
        assert abs(l2 - ((a - b) ** 2).sum()) <= 1e-12 * ((a - b) ** 2).sum()
        assert li == np.abs(a - b).max()


def test_courant_check():
    shape = (16, 16)
    dev = torch.device("cuda")
    with Mpdata(shape, dtype=torch.float32) as m:
        ok = [torch.full(shape, 0.3, device=dev), torch.full(shape, -0.2, device=dev)]
        rc, mx = m.check_courant(ok)
        assert rc == capi.OK and abs(mx - 0.5) < 1e-6
        bad = [torch.full(shape, 0.7, device=dev), torch.full(shape, 0.6, device=dev)]
        rc, mx = m.check_courant(bad)
        assert rc == capi.ECOURANT and abs(mx - 1.3) < 1e-6


def test_stop_flag_and_errors():
    shape = (8, 8)
    dev = torch.device("cuda")
    gc = [torch.zeros(shape, device=dev), torch.zeros(shape, device=dev)]
    psi = torch.ones(shape, device=dev)
    with Mpdata(shape, dtype=torch.float32) as m:
        m.request_stop()
        assert capi.mpdata_step(m.h, psi, gc, raw=True) == capi.ESTOPPED
        m.clear_stop()
        assert capi.mpdata_step(m.h, psi, gc, raw=True) == capi.OK
        # missing G for a NUG handle / stray R: invalid
        assert capi.mpdata_step(m.h, psi, gc, g=psi, raw=True) == capi.EINVAL
        assert capi.mpdata_step(m.h, psi, gc, r=psi, raw=True) == capi.EINVAL
        assert capi.mpdata_step(m.h, psi, gc, n_steps=0, raw=True) == capi.EINVAL
        assert capi.mpdata_step(m.h, psi.data_ptr() + 2, gc, raw=True) == capi.EINVAL
        m.sync()


@pytest.mark.parametrize("n", [7, 500, 2235, 3000])
@pytest.mark.parametrize("name", ["basic", "fct", "tot3_fct", "iga_fct", "kahan_fct", "donor"])
def test_1d_one_launch_path_matches_staged_and_oracle(n, name):
    """1D fields small enough for shared memory run every step of a call in one launch of one
    block (2235 FP64 cells is the largest; 3000 falls back to the per-sub-step kernels): same
    arithmetic as the staged kernels, checked against them and against the oracle."""
    n_iters, opts = {"basic": (2, 0), "fct": (2, capi.FCT), "tot3_fct": (3, capi.TOT | capi.FCT),
                     "iga_fct": (2, capi.IGA | capi.FCT), "kahan_fct": (2, capi.KAHAN | capi.FCT),
                     "donor": (1, 0)}[name]
    rng = np.random.default_rng(n)
    psi = workloads.hello_1d(n)[0] if n >= 400 else 1.0 + rng.uniform(size=n)
    if opts & capi.IGA:
        psi = psi - 0.5
    gc = [np.full(n, 0.5) if n >= 400 else rng.uniform(-0.6, 0.6, size=n)]
    dev = torch.device("cuda")
    outs = []
    for staged in (False, True):
        with Mpdata((n,), dtype=torch.float64, n_iters=n_iters, opts=opts | (capi.STAGED if staged else 0)) as m:
            a = torch.tensor(psi, dtype=torch.float64, device=dev)
            b = torch.empty_like(a)
            m.advance(a, b, [torch.tensor(gc[0], dtype=torch.float64, device=dev)], n_steps=40)
            torch.cuda.synchronize()
            outs.append(b.cpu().numpy())
    ref = oracle.step(psi, gc, n_iters=n_iters, opts=opts, n_steps=40)
    scale = np.abs(ref).max()
    assert np.abs(outs[0] - outs[1]).max() <= 1e-13 * scale
    assert np.abs(outs[0] - ref).max() <= 1e-12 * scale
