"""Open edges (Sect. 2.4, bcond::open) on the GPU against the FP64 oracle: 1D, 2D and 3D fields
with every dimension open or a mix of open and periodic dimensions, with and without the
limiter, third-order terms, infinite gauge, non-unit G and sources; the paper's 1D "hello
world" (Sect. 3.3) as printed; batched and allocation-free entry points; argument checks."""
import numpy as np
import pytest
import torch

import oracle
from helpers import smooth_positive
from paper_1407_1309_gb300 import capi, workloads
from paper_1407_1309_gb300.solver import Mpdata

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")

CASES = {
    "donor": (1, 0),
    "basic": (2, 0),
    "fct": (2, capi.FCT),
    "tot3_fct": (3, capi.TOT | capi.FCT),
    "iga_fct": (2, capi.IGA | capi.FCT),
    "iga_tot_fct": (2, capi.IGA | capi.TOT | capi.FCT),
    "kahan_fct": (2, capi.KAHAN | capi.FCT),
    "abs_fct": (2, capi.ABS | capi.FCT),
    "dfl_fct": (2, capi.DFL | capi.FCT),
}
SHAPES = [(53,), (2,), (19, 23), (2, 7), (9, 8, 11)]
MASKS = {"all": None, "first": (0,), "last": (-1,)}


def mask(shape, which):
    nd = len(shape)
    dims = range(nd) if which is None else [w % nd for w in which]
    return sum(capi.OPEN0 << d for d in dims)


def inputs(shape, seed, sign):
    rng = np.random.default_rng(seed)
    psi = smooth_positive(shape, rng)
    if sign == "var":
        psi = psi - 2.1
    gc = [rng.uniform(-0.3, 0.3, size=shape) / len(shape) for _ in shape]  # divergent, |C| sum <= 0.3
    return psi, gc


def gpu(psi, gc, n_iters, opts, dtype, steps, G=None, R=None, dt=0.0):
    t = lambda a: None if a is None else torch.tensor(a, dtype=dtype, device=DEV)
    o = opts | (capi.NUG if G is not None else 0) | (capi.RHS_EULER_A if R is not None else 0)
    with Mpdata(psi.shape, dtype=dtype, n_iters=n_iters, opts=o) as m:
        p, q = t(psi), torch.empty(psi.shape, dtype=dtype, device=DEV)
        m.advance(p, q, [t(v) for v in gc], g=t(G), r=t(R), dt=dt, n_steps=steps)
        torch.cuda.synchronize()
        return q.double().cpu().numpy()


def check(out, ref, dtype):
    if dtype == torch.float64:
        assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()
    else:
        assert np.linalg.norm(out - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("which", sorted(MASKS))
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("name", sorted(CASES))
def test_open_edges_match_oracle(name, shape, which, dtype):
    n_iters, opts = CASES[name]
    opts |= mask(shape, MASKS[which])
    psi, gc = inputs(shape, len(shape) + n_iters, "var" if opts & capi.IGA else "pos")
    if dtype == torch.float32:
        r = lambda a: a.astype(np.float32).astype(np.float64)
        psi, gc = r(psi), [r(v) for v in gc]
    ref = oracle.step(psi, gc, n_iters=n_iters, opts=int(opts), n_steps=6)
    check(gpu(psi, gc, n_iters, opts, dtype, 6), ref, dtype)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_open_edges_with_g_and_source(dtype):
    shape = (21, 18)
    rng = np.random.default_rng(3)
    psi, gc = inputs(shape, 5, "pos")
    G = 1.0 + 0.3 * rng.uniform(size=shape)
    R = rng.normal(size=shape)
    if dtype == torch.float32:
        r = lambda a: a.astype(np.float32).astype(np.float64)
        psi, gc, G, R = r(psi), [r(v) for v in gc], r(G), r(R)
    opts = capi.FCT | capi.OPEN0 | capi.OPEN1
    ref = oracle.step(psi, gc, g=G, r=R, dt=0.1, n_iters=2, opts=int(opts), n_steps=4)
    check(gpu(psi, gc, 2, opts, dtype, 4, G=G, R=R, dt=0.1), ref, dtype)


def test_hello_world_as_printed():
    """Sect. 3.3: 101 points, C = 0.5, 100 steps, open edges, the default options (two passes,
    FCT, infinite gauge, compensated summation), FP64, against the oracle."""
    psi, gc = workloads.agnesi_1d()
    opts = capi.FCT | capi.IGA | capi.KAHAN | capi.OPEN0
    ref = oracle.step(psi, gc, n_iters=2, opts=int(opts), n_steps=100)
    out = gpu(psi, gc, 2, opts, torch.float64, 100)
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()


def test_open_edges_on_batched_and_allocation_free_entry_points():
    shapes = [(17, 13), (12, 20)]
    opts = capi.FCT | capi.OPEN0 | capi.OPEN1
    fields = [inputs(s, 11 + i, "pos") for i, s in enumerate(shapes)]
    refs = [oracle.step(p, g, n_iters=2, opts=int(opts), n_steps=3) for p, g in fields]
    t = lambda a: torch.tensor(a, dtype=torch.float64, device=DEV)
    with Mpdata(shapes, dtype=torch.float64, n_iters=2, opts=opts) as m:
        psi = torch.cat([t(p).flatten() for p, _ in fields])
        gc = [torch.cat([t(g[d]).flatten() for _, g in fields]) for d in range(2)]
        out = torch.empty_like(psi)
        m.advance(psi, out, gc, n_steps=3)
        torch.cuda.synchronize()
    got = out.cpu().numpy()
    off = 0
    for ref in refs:
        assert np.abs(got[off:off + ref.size].reshape(ref.shape) - ref).max() <= 1e-12 * np.abs(ref).max()
        off += ref.size
    p, g = fields[0]
    a = t(p)
    for _ in range(3):
        capi.mpdata_step_noalloc(2, shapes[0], capi.F64, 2, opts, a, a, [t(v) for v in g])
    torch.cuda.synchronize()
    assert np.abs(a.cpu().numpy() - refs[0]).max() <= 1e-12 * np.abs(refs[0]).max()


def test_open_edge_argument_checks():
    z = torch.zeros(8, 8, dtype=torch.float64, device=DEV)
    with pytest.raises(capi.MpdataError):
        Mpdata((8, 1), dtype=torch.float64, opts=capi.OPEN1)  # an open dimension needs 2 cells
    with pytest.raises(capi.MpdataError):
        Mpdata((8, 8), dtype=torch.float64, opts=capi.OPEN2)  # no third dimension
    with Mpdata((8, 8), dtype=torch.float64, n_iters=2, opts=capi.FCT | capi.OPEN0) as m:
        assert capi.mpdata_adjoint_step(m.h, z, [z, z], None, z.clone(), raw=True) == capi.EUNSUPPORTED
