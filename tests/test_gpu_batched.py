"""Batched handles (ensembles of independent 2D fields of uneven sizes, one persistent
launch per step) against the per-field staged kernels and the oracle, and CUDA-graph
capture of a step loop."""
import numpy as np
import pytest
import torch

import oracle
from helpers import boxes, nondivergent, smooth_positive
from paper_1407_1309_gb300 import capi, workloads
from paper_1407_1309_gb300.solver import Mpdata

pytestmark = pytest.mark.gpu

SHAPES = [(64, 64), (96, 96), (33, 57), (130, 7), (200, 130), (8, 9), (250, 64), (1, 5), (121, 240)]


def ensemble(shapes, seed, var=False):
    rng = np.random.default_rng(seed)
    out = []
    for s in shapes:
        gc = nondivergent(s, rng, 0.35)
        psi = boxes(s, rng) if rng.uniform() < 0.5 else smooth_positive(s, rng)
        out.append((psi - 2.5 if var else psi, gc))
    return out


def run_batch(fields, dtype, n_iters, opts, n_steps, G=None, tile_rows=0, kernel=0):
    dev = torch.device("cuda")
    shapes = [p.shape for p, _ in fields]
    cat = lambda arrs: torch.tensor(np.concatenate([a.ravel() for a in arrs]), dtype=dtype, device=dev)
    psi = cat([p for p, _ in fields])
    gc = [cat([g[d] for _, g in fields]) for d in range(2)]
    Gt = cat(G) if G is not None else None
    with Mpdata(shapes, dtype=dtype, n_iters=n_iters, opts=opts | (capi.NUG if G is not None else 0)) as m:
        if tile_rows:
            m.tune(capi.TUNE_TILE_ROWS, tile_rows)
        if kernel:
            m.tune(capi.TUNE_KERNEL, kernel)
        out = torch.empty_like(psi)
        m.advance(psi, out, gc, Gt, None, 0.0, n_steps)
        masses = m.mass(out, Gt)
        torch.cuda.synchronize()
    res, o = [], 0
    host = out.double().cpu().numpy()
    for s in shapes:
        n = int(np.prod(s))
        res.append(host[o:o + n].reshape(s))
        o += n
    return res, masses


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("name,opts", [("basic", 0), ("fct", capi.FCT), ("iga_fct", capi.IGA | capi.FCT)])
@pytest.mark.parametrize("nug", [False, True], ids=["g1", "nug"])
def test_batched_matches_staged_and_oracle(dtype, name, opts, nug):
    fields = ensemble(SHAPES, 1, var=bool(opts & capi.IGA))
    if dtype == torch.float32:
        fields = [(p.astype(np.float32).astype(np.float64), [g.astype(np.float32).astype(np.float64) for g in gc])
                  for p, gc in fields]
    rng = np.random.default_rng(2)
    G = [(1.0 + 0.25 * rng.uniform(size=p.shape)) for p, _ in fields] if nug else None
    if G is not None and dtype == torch.float32:
        G = [g.astype(np.float32).astype(np.float64) for g in G]
    got, masses = run_batch(fields, dtype, 2, opts, 5, G)
    staged, _ = run_batch(fields, dtype, 2, opts | capi.STAGED, 5, G)
    for f, ((p, gc), a, b) in enumerate(zip(fields, got, staged)):
        ref = oracle.step(p, gc, g=None if G is None else G[f], n_iters=2, opts=opts, n_steps=5)
        scale = np.abs(ref).max()
        if dtype == torch.float64:
            assert np.abs(a - ref).max() <= 1e-12 * scale
            assert np.abs(a - b).max() <= 1e-13 * scale
        else:
            assert np.linalg.norm(a - ref) <= 1e-5 * np.linalg.norm(ref)
        m_ref = oracle.mass(p, None if G is None else G[f])
        assert abs(masses[f] - m_ref) <= (1e-12 if dtype == torch.float64 else 1e-6) * oracle.mass(np.abs(p), None if G is None else G[f])


@pytest.mark.parametrize("tile_rows", [8, 32, 64])
def test_batched_ensemble_workload_tiles(tile_rows):
    """Sixteen fields of the ensemble workload (sides 64..512), FP32, 20 steps."""
    ens = workloads.ensemble_2d(16, seed=3)
    fields = [(p.astype(np.float32).astype(np.float64), [g.astype(np.float32).astype(np.float64) for g in gc])
              for p, gc in ens]
    got, _ = run_batch(fields, torch.float32, 2, capi.FCT, 20, tile_rows=tile_rows)
    for (p, gc), a in zip(fields, got):
        ref = oracle.step(p, gc, n_iters=2, opts=oracle.FCT, n_steps=20)
        assert np.linalg.norm(a - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("batched", [False, True], ids=["single", "batched"])
def test_cuda_graph_replay_equals_direct_run(batched):
    dev = torch.device("cuda")
    if batched:
        fields = ensemble([(64, 64), (96, 32), (40, 80)], 4)
        shapes = [p.shape for p, _ in fields]
        cat = lambda arrs: torch.tensor(np.concatenate([a.ravel() for a in arrs]), dtype=torch.float32, device=dev)
        psi0 = cat([p for p, _ in fields])
        gc = [cat([g[d] for _, g in fields]) for d in range(2)]
    else:
        psi_np, gc_np, _ = workloads.rotation_2d(128)
        shapes = [(128, 128)]
        psi0 = torch.tensor(psi_np, dtype=torch.float32, device=dev)
        gc = [torch.tensor(v, dtype=torch.float32, device=dev) for v in gc_np]
    with Mpdata(shapes, dtype=torch.float32, n_iters=2, opts=capi.FCT) as m:
        direct = torch.empty_like(psi0)
        m.advance(psi0, direct, gc, n_steps=10)
        src = psi0.clone()
        out = torch.empty_like(psi0)
        graph = m.capture(src, out, gc, 10)
        out.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, direct)
        # replay on new contents of the captured input buffer
        src.copy_(direct)
        graph.replay()
        again = torch.empty_like(psi0)
        m.advance(direct, again, gc, n_steps=10)
        torch.cuda.synchronize()
        assert torch.equal(out, again)


@pytest.mark.parametrize("tile_rows", [0, 8, 48])
@pytest.mark.parametrize("name,opts", [("fct", capi.FCT), ("iga_fct", capi.IGA | capi.FCT), ("basic", 0)])
def test_batched_lanes_of_two_columns(name, opts, tile_rows):
    """MPDATA_TUNE_KERNEL = 3 on a batched FP32 handle: the persistent kernel with lanes of 2
    columns (strips of 56 outputs), against the oracle field by field (FP32 bars) and against
    the 4-column lanes (to rounding)."""
    fields = ensemble(SHAPES, 3, var=bool(opts & capi.IGA))
    fields = [(p.astype(np.float32).astype(np.float64), [g.astype(np.float32).astype(np.float64) for g in gc])
              for p, gc in fields]
    got, masses = run_batch(fields, torch.float32, 2, opts, 5, tile_rows=tile_rows, kernel=3)
    wide, _ = run_batch(fields, torch.float32, 2, opts, 5, tile_rows=tile_rows)
    for f, ((p, gc), a, b) in enumerate(zip(fields, got, wide)):
        ref = oracle.step(p, gc, n_iters=2, opts=opts, n_steps=5)
        assert np.linalg.norm(a - ref) <= 1e-5 * np.linalg.norm(ref)
        assert np.linalg.norm(a - b) <= 1e-6 * max(np.linalg.norm(b), 1e-30)
        assert abs(masses[f] - oracle.mass(p, None)) <= 1e-6 * oracle.mass(np.abs(p), None)
