"""The variable-sign option abs (Sect. 3.1.5: |psi| in every psi-fraction of the
pseudo-velocity) and the divergent-flow option dfl (Sect. 3.1.3) on the GPU against the
oracle: 1D, 2D and 3D, with the limiter and the third-order terms, FP64 and FP32, single and
batched handles; on a positive field abs is the basic scheme bit for bit.  (Their reverse
steps are checked against the oracle's adjoint in test_gpu_adjoint.py.)"""
import numpy as np
import pytest
import torch

import oracle
from helpers import nondivergent, smooth_positive
from paper_1407_1309_gb300 import capi
from paper_1407_1309_gb300.solver import Mpdata

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")
SHAPES = [(300,), (67, 131), (20, 18, 22)]
CASES = {"abs": (2, capi.ABS), "abs_fct": (2, capi.ABS | capi.FCT), "abs_it3_fct": (3, capi.ABS | capi.FCT),
         "abs_tot3_fct": (3, capi.ABS | capi.TOT | capi.FCT)}


def variable_sign(shape, seed):
    rng = np.random.default_rng(seed)
    psi = smooth_positive(shape, rng) - 1.6  # crosses zero on a large part of the domain
    return psi, nondivergent(shape, rng, 0.4)


def run(psi, gc, n_iters, opts, dtype, steps, G=None):
    with Mpdata(psi.shape, dtype=dtype, n_iters=n_iters, opts=opts | (capi.NUG if G is not None else 0)) as m:
        t = lambda a: None if a is None else torch.tensor(a, dtype=dtype, device=DEV)
        p, q = t(psi), torch.empty(psi.shape, dtype=dtype, device=DEV)
        m.advance(p, q, [t(v) for v in gc], n_steps=steps, g=t(G))
        torch.cuda.synchronize()
        return q.double().cpu().numpy()


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
@pytest.mark.parametrize("name", sorted(CASES))
def test_abs_fp64_matches_oracle(shape, name):
    n_iters, opts = CASES[name]
    psi, gc = variable_sign(shape, len(shape) + n_iters)
    ref = oracle.step(psi, gc, n_iters=n_iters, opts=int(opts), n_steps=4)
    out = run(psi, gc, n_iters, opts, torch.float64, 4)
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
@pytest.mark.parametrize("name", ["abs_fct", "abs_tot3_fct"])
def test_abs_fp32_close_to_oracle(shape, name):
    n_iters, opts = CASES[name]
    psi, gc = variable_sign(shape, 7 * len(shape))
    r = lambda a: a.astype(np.float32).astype(np.float64)
    psi, gc = r(psi), [r(v) for v in gc]
    ref = oracle.step(psi, gc, n_iters=n_iters, opts=int(opts), n_steps=4)
    out = run(psi, gc, n_iters, opts, torch.float32, 4)
    assert np.linalg.norm(out - ref) <= 1e-5 * np.linalg.norm(ref)


def test_abs_with_nonunit_g_matches_oracle():
    shape = (48, 61)
    psi, gc = variable_sign(shape, 3)
    G = 1.0 + 0.2 * np.random.default_rng(4).uniform(size=shape)
    opts = capi.ABS | capi.FCT
    ref = oracle.step(psi, gc, g=G, n_iters=2, opts=int(opts), n_steps=3)
    out = run(psi, gc, 2, opts, torch.float64, 3, G=G)
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
def test_abs_is_the_basic_scheme_on_a_positive_field(shape):
    rng = np.random.default_rng(2)
    psi = smooth_positive(shape, rng)
    gc = nondivergent(shape, rng, 0.4)
    for n_iters, opts in ((2, capi.FCT), (3, capi.TOT | capi.FCT)):
        with_abs = run(psi, gc, n_iters, opts | capi.ABS, torch.float64, 3)
        basic = run(psi, gc, n_iters, opts | capi.STAGED, torch.float64, 3)
        assert np.array_equal(with_abs, basic)


def test_abs_batched_handle_matches_oracle():
    shapes = [(40, 56), (64, 64), (33, 47)]
    fields = [variable_sign(s, 20 + k) for k, s in enumerate(shapes)]
    opts = capi.ABS | capi.FCT
    dt = torch.float64
    with Mpdata(shapes, dtype=dt, n_iters=2, opts=opts) as m:
        cat = lambda arrs: torch.tensor(np.concatenate([a.ravel() for a in arrs]), dtype=dt, device=DEV)
        p = cat([f[0] for f in fields])
        gc = [cat([f[1][d] for f in fields]) for d in range(2)]
        q = torch.empty_like(p)
        m.advance(p, q, gc, n_steps=3)
        torch.cuda.synchronize()
        out = q.cpu().numpy()
    off = 0
    for (psi, g), s in zip(fields, shapes):
        n = int(np.prod(s))
        ref = oracle.step(psi, g, n_iters=2, opts=int(opts), n_steps=3)
        assert np.abs(out[off:off + n].reshape(s) - ref).max() <= 1e-12 * np.abs(ref).max()
        off += n


def test_abs_excludes_iga():
    shape = (16, 16)
    rc, h = capi.mpdata_create(2, [shape], capi.F64, 2, capi.ABS | capi.IGA, raw=True)
    assert rc == capi.EINVAL and not h


# ----------------------------------------------------------------------------- divergent-flow option

DFL_CASES = {"dfl": (2, capi.DFL), "dfl_fct": (2, capi.DFL | capi.FCT), "dfl_it3_fct": (3, capi.DFL | capi.FCT),
             "dfl_tot3": (3, capi.DFL | capi.TOT), "dfl_abs_fct": (2, capi.DFL | capi.ABS | capi.FCT)}


def divergent(shape, seed):
    rng = np.random.default_rng(seed)
    psi = smooth_positive(shape, rng) - (0.0 if seed % 2 else 1.2)
    gc = [0.3 * rng.uniform(-1, 1, size=shape) / len(shape) for _ in shape]  # divergent everywhere
    return psi, gc


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
@pytest.mark.parametrize("name", sorted(DFL_CASES))
def test_dfl_fp64_matches_oracle(shape, name):
    n_iters, opts = DFL_CASES[name]
    psi, gc = divergent(shape, 2 * len(shape) + n_iters)
    if not opts & capi.ABS:
        psi = np.abs(psi) + 0.5
    ref = oracle.step(psi, gc, n_iters=n_iters, opts=int(opts), n_steps=4)
    out = run(psi, gc, n_iters, opts, torch.float64, 4)
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
def test_dfl_fp32_and_nonunit_g_close_to_oracle(shape):
    psi, gc = divergent(shape, 9)
    r = lambda a: a.astype(np.float32).astype(np.float64)
    G = r(1.0 + 0.2 * np.random.default_rng(5).uniform(size=shape))
    psi, gc = r(psi), [r(v) for v in gc]
    opts = capi.DFL | capi.FCT
    ref = oracle.step(psi, gc, g=G, n_iters=2, opts=int(opts), n_steps=4)
    out = run(psi, gc, 2, opts, torch.float32, 4, G=G)
    assert np.linalg.norm(out - ref) <= 1e-5 * np.linalg.norm(ref)
    ref64 = oracle.step(psi, gc, g=G, n_iters=3, opts=int(opts), n_steps=4)
    out64 = run(psi, gc, 3, opts, torch.float64, 4, G=G)
    assert np.abs(out64 - ref64).max() <= 1e-12 * np.abs(ref64).max()


def test_dfl_excludes_iga():
    shape = (16, 16)
    rc, h = capi.mpdata_create(2, [shape], capi.F64, 2, capi.DFL | capi.IGA, raw=True)
    assert rc == capi.EINVAL and not h
