"""The adjoint kernels against the oracle's adjoint, and autograd gradients against
central finite differences of the GPU forward.

FP64 GPU adjoint vs FP64 oracle adjoint: max-norm relative error <= 1e-12 on
generic smooth positive inputs (no flat regions and no ties, where the limiter's
branches are differentiable).  Gradients of a rollout loss: relative error <= 1e-4
against central differences along seeded smooth directions.  The FCT limiter makes
the step only piecewise smooth (min/max switches), so over many steps a
perturbation of 1e-3, or even 1e-6 on a coarse grid, crosses switches somewhere in
the field and the difference quotient itself is off; with FCT the check therefore
uses eps = 1e-7 in FP64 (where the quotient has converged to the adjoint
gradient), and eps = 1e-4 for the smooth scheme without the limiter (at 1e-3 the
O(eps^2) truncation of the quotient reaches ~2e-4 on directions with a small
derivative).
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import nondivergent, smooth_positive
from paper_1407_1309_gb300 import capi, workloads
from paper_1407_1309_gb300.autograd import rollout
from paper_1407_1309_gb300.solver import Mpdata

pytestmark = pytest.mark.gpu

CASES = {
    "donor": (1, 0),
    "basic": (2, 0),
    "fct": (2, capi.FCT),
    "iga_fct": (2, capi.IGA | capi.FCT),
    "it3_fct": (3, capi.FCT),
    "kahan_fct": (2, capi.KAHAN | capi.FCT),
}
SHAPES = [(41,), (14, 11), (6, 7, 5)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("nug", [False, True], ids=["g1", "nug"])
def test_adjoint_matches_oracle(shape, name, nug):
    n_iters, opts = CASES[name]
    rng = np.random.default_rng(len(shape) * 10 + n_iters)
    psi = smooth_positive(shape, rng)
    if opts & capi.IGA:
        psi = psi - 2.0
    gc = nondivergent(shape, rng, 0.3)
    G = 1.0 + 0.2 * rng.uniform(size=shape) if nug else None
    y = rng.normal(size=shape)
    ref_pb, ref_gcb = oracle.adj_step(psi, gc, y, g=G, n_iters=n_iters, opts=opts)
    dev = torch.device("cuda")
    t = lambda a: None if a is None else torch.tensor(a, dtype=torch.float64, device=dev)
    o = opts | (capi.NUG if nug else 0)
    with Mpdata(shape, dtype=torch.float64, n_iters=n_iters, opts=o) as m:
        pb = t(y)
        gcb = [torch.full(shape, 0.5, dtype=torch.float64, device=dev) for _ in shape]  # accumulated onto
        m.adjoint_step(t(psi), [t(v) for v in gc], pb, g=t(G), gc_bar=gcb)
        torch.cuda.synchronize()
        got_pb = pb.cpu().numpy()
        got_gcb = [v.cpu().numpy() - 0.5 for v in gcb]
    scale = max(np.abs(ref_pb).max(), max(np.abs(v).max() for v in ref_gcb))
    assert np.abs(got_pb - ref_pb).max() <= 1e-12 * scale
    for a, b in zip(got_gcb, ref_gcb):
        assert np.abs(a - b).max() <= 1e-12 * scale


def test_adjoint_fp32_close_to_oracle():
    shape = (33, 29)
    rng = np.random.default_rng(3)
    psi, gc, y = smooth_positive(shape, rng), nondivergent(shape, rng, 0.35), rng.normal(size=shape)
    r = lambda a: a.astype(np.float32).astype(np.float64)
    psi, gc, y = r(psi), [r(v) for v in gc], r(y)
    ref_pb, ref_gcb = oracle.adj_step(psi, gc, y, n_iters=2, opts=oracle.FCT)
    dev = torch.device("cuda")
    with Mpdata(shape, dtype=torch.float32, n_iters=2, opts=capi.FCT) as m:
        pb = torch.tensor(y, dtype=torch.float32, device=dev)
        gcb = [torch.zeros(shape, device=dev) for _ in shape]
        m.adjoint_step(torch.tensor(psi, dtype=torch.float32, device=dev),
                       [torch.tensor(v, dtype=torch.float32, device=dev) for v in gc], pb, gc_bar=gcb)
        torch.cuda.synchronize()
    assert np.linalg.norm(pb.cpu().numpy() - ref_pb) <= 1e-5 * np.linalg.norm(ref_pb)
    for a, b in zip(gcb, ref_gcb):
        assert np.linalg.norm(a.cpu().numpy() - b) <= 1e-5 * np.linalg.norm(b)


# the options with the second form of the pseudo-advector's reverse: the third-order terms
# (Sect. 3.1.2), |psi| in the psi-fractions (Sect. 3.1.5) and the divergent-flow term (Sect.
# 3.1.3, on a divergent advector), with and without the limiter
EXT_CASES = {
    "dfl": (2, capi.DFL),
    "dfl3_fct": (3, capi.DFL | capi.FCT),
    "dfl_tot3_fct": (3, capi.DFL | capi.TOT | capi.FCT),
    "tot2_fct": (2, capi.TOT | capi.FCT),
    "tot3_fct": (3, capi.TOT | capi.FCT),
    "tot3": (3, capi.TOT),
    "iga_tot_fct": (2, capi.IGA | capi.TOT | capi.FCT),
    "abs_fct": (2, capi.ABS | capi.FCT),
    "abs_tot3": (3, capi.ABS | capi.TOT),
}
EXT_SHAPES = [(41,), (14, 11), (6, 7, 5), (9, 10, 11)]


def ext_inputs(shape, opts, seed):
    rng = np.random.default_rng(seed)
    psi = smooth_positive(shape, rng)
    if opts & capi.IGA:
        psi = psi - 2.0
    if opts & capi.ABS:
        psi = psi - 2.1  # variable sign: the fractions read |psi|
    if opts & capi.DFL:  # a divergent advector, |C| <= 0.3
        gc = [workloads.low_modes(rng, shape, 4) for _ in shape]
        gc = [0.3 * v / np.abs(v).max() for v in gc]
    else:
        gc = nondivergent(shape, rng, 0.3)
    return psi, gc, rng.normal(size=shape), rng


@pytest.mark.parametrize("shape", EXT_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("name", sorted(EXT_CASES))
@pytest.mark.parametrize("nug", [False, True], ids=["g1", "nug"])
def test_adjoint_third_order_and_abs_match_oracle(shape, name, nug):
    """FP64 GPU reverse step with the third-order terms or |psi| against the oracle's adjoint
    (the exact transpose of its dual-number derivatives), max-norm 1e-12; the 3D cases with
    n_iters = 3, tot, FCT and G are the 3D configuration's step."""
    n_iters, opts = EXT_CASES[name]
    psi, gc, y, rng = ext_inputs(shape, opts, len(shape) * 10 + n_iters + 100 * int(nug))
    G = 1.0 + 0.2 * rng.uniform(size=shape) if nug else None
    ref_pb, ref_gcb = oracle.adj_step(psi, gc, y, g=G, n_iters=n_iters, opts=opts)
    dev = torch.device("cuda")
    t = lambda a: None if a is None else torch.tensor(a, dtype=torch.float64, device=dev)
    with Mpdata(shape, dtype=torch.float64, n_iters=n_iters, opts=opts | (capi.NUG if nug else 0)) as m:
        pb = t(y)
        gcb = [torch.full(shape, 0.5, dtype=torch.float64, device=dev) for _ in shape]
        m.adjoint_step(t(psi), [t(v) for v in gc], pb, g=t(G), gc_bar=gcb)
        torch.cuda.synchronize()
        got_pb = pb.cpu().numpy()
        got_gcb = [v.cpu().numpy() - 0.5 for v in gcb]
    scale = max(np.abs(ref_pb).max(), max(np.abs(v).max() for v in ref_gcb))
    assert np.abs(got_pb - ref_pb).max() <= 1e-12 * scale
    for a, b in zip(got_gcb, ref_gcb):
        assert np.abs(a - b).max() <= 1e-12 * scale


@pytest.mark.parametrize("name", ["tot3_fct", "abs_fct", "dfl3_fct"])
def test_adjoint_third_order_and_abs_fp32_close_to_oracle(name):
    """FP32 reverse step of the 3D configuration (n_iters = 3, tot, FCT, G) and of the |psi|
    option against the FP64 oracle (inputs rounded to FP32 on both sides): relative L2 1e-5."""
    n_iters, opts = EXT_CASES[name]
    shape = (12, 13, 14)
    psi, gc, y, rng = ext_inputs(shape, opts, 7)
    G = 1.0 + 0.2 * rng.uniform(size=shape)
    r = lambda a: a.astype(np.float32).astype(np.float64)
    psi, gc, y, G = r(psi), [r(v) for v in gc], r(y), r(G)
    ref_pb, ref_gcb = oracle.adj_step(psi, gc, y, g=G, n_iters=n_iters, opts=opts)
    dev = torch.device("cuda")
    t = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)
    with Mpdata(shape, dtype=torch.float32, n_iters=n_iters, opts=opts | capi.NUG) as m:
        pb = t(y)
        gcb = [torch.zeros(shape, device=dev) for _ in shape]
        m.adjoint_step(t(psi), [t(v) for v in gc], pb, g=t(G), gc_bar=gcb)
        torch.cuda.synchronize()
    assert np.linalg.norm(pb.cpu().numpy() - ref_pb) <= 1e-5 * np.linalg.norm(ref_pb)
    for a, b in zip(gcb, ref_gcb):
        assert np.linalg.norm(a.cpu().numpy() - b) <= 1e-5 * np.linalg.norm(b)


def test_autograd_gradient_3d_third_order_matches_finite_differences():
    """A 3D rollout with the third-order terms (n_iters = 3, 16^3, 6 steps, checkpoints every
    3): autograd gradient against central differences (eps = 1e-6, FP64) along 4 seeded smooth
    directions over (psi0, GC), relative error 1e-4.  Without the limiter, whose min/max
    switches a central difference can straddle, the step is smooth on these inputs; the
    limited step's reverse is checked against the oracle's adjoint above."""
    shape = (16, 16, 16)
    rng = np.random.default_rng(11)
    dev = torch.device("cuda")
    f64 = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    psi0 = smooth_positive(shape, rng)
    gc = [f64(v) for v in nondivergent(shape, rng, 0.3)]
    eps = 1e-6
    with Mpdata(shape, dtype=torch.float64, n_iters=3, opts=capi.TOT) as m:
        with torch.no_grad():
            target = rollout(m, f64(psi0 + 0.05 * workloads.low_modes(rng, shape, 4)), gc, 6, 3)

        def loss(p0, g):
            return 0.5 * ((rollout(m, p0, g, 6, 3) - target) ** 2).sum()

        p0 = f64(psi0).requires_grad_(True)
        gg = [v.clone().requires_grad_(True) for v in gc]
        loss(p0, gg).backward()
        errs = []
        for _ in range(4):
            dirs = [workloads.low_modes(rng, shape, 4) for _ in range(4)]
            dirs = [d / np.sqrt(np.mean(d ** 2)) for d in dirs]
            dp, dg = f64(dirs[0]), [f64(d) * 0.05 for d in dirs[1:]]
            with torch.no_grad():
                lp = loss(p0 + eps * dp, [a + eps * b for a, b in zip(gc, dg)])
                lm = loss(p0 - eps * dp, [a - eps * b for a, b in zip(gc, dg)])
            fd = float((lp - lm) / (2 * eps))
            an = float((p0.grad * dp).sum() + sum((a.grad * b).sum() for a, b in zip(gg, dg)))
            errs.append(abs(fd - an) / max(abs(fd), 1e-30))
    assert max(errs) <= 1e-4, errs


@pytest.mark.parametrize("shape", [(14, 11), (6, 7, 5)], ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("name", ["tot3_fct", "abs_fct", "dfl3_fct"])
def test_record_replay_third_order_and_abs(shape, name):
    """The split reverse step (tape, then the sweep from it) with these options gives the
    one-call reverse step (FP64, up to the order of the atomic additions) and the recorded step's
    result is the oracle's step."""
    n_iters, opts = EXT_CASES[name]
    psi, gc, y, _ = ext_inputs(shape, opts, 5)
    dev = torch.device("cuda")
    t = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    with Mpdata(shape, dtype=torch.float64, n_iters=n_iters, opts=opts) as m:
        p, g = t(psi), [t(v) for v in gc]
        pb1, gb1 = t(y), [torch.zeros(shape, dtype=torch.float64, device=dev) for _ in shape]
        m.adjoint_step(p, g, pb1, gc_bar=gb1)
        tape = torch.full((m.tape_numel(),), float("nan"), dtype=torch.float64, device=dev)
        nxt = torch.empty_like(p)
        m.adjoint_record(p, g, tape, psi_next=nxt)
        pb2, gb2 = t(y), [torch.zeros(shape, dtype=torch.float64, device=dev) for _ in shape]
        m.adjoint_replay(p, g, tape, pb2, gc_bar=gb2)
        torch.cuda.synchronize()
        scale = max(float(pb1.abs().max()), max(float(v.abs().max()) for v in gb1))
        assert float((pb1 - pb2).abs().max()) <= 1e-12 * scale
        for a, b in zip(gb1, gb2):
            assert float((a - b).abs().max()) <= 1e-12 * scale
    ref = oracle.step(psi, gc, n_iters=n_iters, opts=opts)
    assert np.abs(nxt.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


SRC_CASES = {"fct": (2, capi.FCT), "tot3_fct": (3, capi.TOT | capi.FCT)}


@pytest.mark.parametrize("shape", [(41,), (14, 11), (6, 7, 5)], ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("rhs", ["euler_a", "euler_b"])
@pytest.mark.parametrize("name", sorted(SRC_CASES))
def test_adjoint_with_euler_sources_matches_oracle(shape, rhs, name):
    """The reverse step of a step with an Euler source (Sect. 4.1; R given, dt = 0.3) against the
    oracle's adjoint (FP64, max-norm 1e-12), and dL/dR, accumulated onto r_bar, against its closed
    form dt * dL/dpsi^{n+1} (euler_a) or dt * dL/dpsi^n (euler_b) and against central differences
    of the oracle's forward step along a random direction."""
    n_iters, opts = SRC_CASES[name]
    rng = np.random.default_rng(len(shape) * 100 + n_iters + (7 if rhs == "euler_b" else 0))
    psi = smooth_positive(shape, rng)
    gc = nondivergent(shape, rng, 0.3)
    y = rng.normal(size=shape)
    R, dt = 0.5 * rng.normal(size=shape), 0.3
    ref_pb, ref_gcb = oracle.adj_step(psi, gc, y, r=R, dt=dt, n_iters=n_iters, opts=opts, rhs=rhs)
    dev = torch.device("cuda")
    t = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    bit = capi.RHS_EULER_A if rhs == "euler_a" else capi.RHS_EULER_B
    with Mpdata(shape, dtype=torch.float64, n_iters=n_iters, opts=opts | bit) as m:
        pb = t(y)
        gcb = [torch.zeros(shape, dtype=torch.float64, device=dev) for _ in shape]
        rb = torch.full(shape, 0.25, dtype=torch.float64, device=dev)  # accumulated onto
        m.adjoint_step(t(psi), [t(v) for v in gc], pb, gc_bar=gcb, r=t(R), dt=dt, r_bar=rb)
        torch.cuda.synchronize()
        got_pb, got_rb = pb.cpu().numpy(), rb.cpu().numpy() - 0.25
        got_gcb = [v.cpu().numpy() for v in gcb]
    scale = max(np.abs(ref_pb).max(), max(np.abs(v).max() for v in ref_gcb))
    assert np.abs(got_pb - ref_pb).max() <= 1e-12 * scale
    for a, b in zip(got_gcb, ref_gcb):
        assert np.abs(a - b).max() <= 1e-12 * scale
    want = dt * (y if rhs == "euler_a" else ref_pb)
    assert np.abs(got_rb - want).max() <= 1e-12 * np.abs(want).max()
    dR, eps = rng.normal(size=shape), 1e-6
    L = lambda rr: float(np.sum(y * oracle.step(psi, gc, r=rr, dt=dt, n_iters=n_iters, opts=opts, rhs=rhs)))
    fd = (L(R + eps * dR) - L(R - eps * dR)) / (2 * eps)
    assert abs(fd - float(np.sum(got_rb * dR))) <= 1e-6 * max(abs(fd), 1.0)


def test_adjoint_with_sources_argument_checks():
    dev = torch.device("cuda")
    shape = (8, 8)
    z = [torch.zeros(shape, dtype=torch.float64, device=dev) for _ in range(4)]
    with Mpdata(shape, dtype=torch.float64, n_iters=2, opts=capi.FCT) as m:  # no source bit
        assert capi.mpdata_adjoint_step_rhs(m.h, z[0], z[:2], None, z[2], 0.1, z[3], raw=True) == capi.EUNSUPPORTED
    with Mpdata(shape, dtype=torch.float64, n_iters=2, opts=capi.FCT | capi.RHS_EULER_A) as m:
        assert capi.mpdata_adjoint_step_rhs(m.h, z[0], z[:2], None, None, 0.1, z[3], raw=True) == capi.EINVAL
        assert capi.mpdata_adjoint_step(m.h, z[0], z[:2], None, z[3], raw=True) == capi.EUNSUPPORTED


def test_adjoint_rejects_unsupported():
    dev = torch.device("cuda")
    shape = (8, 8)
    z = [torch.zeros(shape, device=dev), torch.zeros(shape, device=dev)]
    for opts in (capi.RHS_EULER_A, capi.FCT | capi.RHS_EULER_B):
        with Mpdata(shape, dtype=torch.float32, n_iters=2, opts=opts) as m:
            rc = capi.mpdata_adjoint_step(m.h, z[0], z, None, z[1], raw=True)
            assert rc == capi.EUNSUPPORTED


def fd_check(n, steps, every, n_dirs, seed=0, eps=1e-7, opts=capi.FCT):
    """Loss 0.5 ||psi_T - psi_target||^2; autograd gradient vs central differences."""
    psi0_np, gc_np, pert = workloads.adjoint_2d(n, seed=seed)
    dev = torch.device("cuda")
    f64 = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    m = Mpdata((n, n), dtype=torch.float64, n_iters=2, opts=opts)
    gc = [f64(v) for v in gc_np]
    with torch.no_grad():
        target = rollout(m, f64(psi0_np + 0.05 * pert), gc, steps, every)

    def loss(p0, g):
        out = rollout(m, p0, g, steps, every)
        return 0.5 * ((out - target) ** 2).sum()

    p0 = f64(psi0_np).requires_grad_(True)
    gg = [v.clone().requires_grad_(True) for v in gc]
    L = loss(p0, gg)
    L.backward()
    rng = np.random.default_rng(seed + 1)
    errs = []
    for _ in range(n_dirs):
        dirs = []
        for _k in range(3):
            d = workloads.low_modes(rng, (n, n), 4)
            dirs.append(d / np.sqrt(np.mean(d ** 2)))
        dp, dg = f64(dirs[0]), [f64(dirs[1]) * 0.05, f64(dirs[2]) * 0.05]
        with torch.no_grad():
            lp = loss(p0 + eps * dp, [a + eps * b for a, b in zip(gc, dg)])
            lm = loss(p0 - eps * dp, [a - eps * b for a, b in zip(gc, dg)])
        fd = float((lp - lm) / (2 * eps))
        an = float((p0.grad * dp).sum() + sum((a.grad * b).sum() for a, b in zip(gg, dg)))
        errs.append(abs(fd - an) / max(abs(fd), 1e-30))
    m.close()
    return errs


def test_autograd_gradient_matches_finite_differences_small():
    errs = fd_check(48, 24, 5, 6)
    assert max(errs) <= 1e-4, errs


def test_autograd_gradient_smooth_scheme():
    """Without the limiter the step is smooth and a much larger eps agrees."""
    errs = fd_check(48, 24, 5, 6, eps=1e-4, opts=0)
    assert max(errs) <= 1e-4, errs


def test_autograd_gradient_adjoint_workload_512():
    """The adjoint workload (512^2, FCT, two passes, 200 steps, checkpoints every 20) on
    64 seeded smooth directions over (psi0, GC)."""
    errs = fd_check(512, 200, 20, 64)
    assert max(errs) <= 1e-4, errs


def test_graph_backward_equals_eager_backward():
    """Graph-replayed backward == eager backward, twice on one handle with the advector
    changed in place in between (the captured segments must take the new advector)."""
    psi0_np, gc_np, pert = workloads.adjoint_2d(96, seed=2)
    dev = torch.device("cuda")
    f64 = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    target = f64(psi0_np + 0.05 * pert)
    grads = {False: [], True: []}
    for use_graphs in (False, True):
        with Mpdata((96, 96), dtype=torch.float64, n_iters=2, opts=capi.FCT) as m:
            gg = [f64(v).requires_grad_(True) for v in gc_np]
            for scale in (1.0, 0.7):
                with torch.no_grad():
                    for g, v in zip(gg, gc_np):
                        g.copy_(f64(v * scale))
                    for g in gg:
                        g.grad = None
                p0 = f64(psi0_np).requires_grad_(True)
                out = rollout(m, p0, gg, 23, 5, use_graphs=use_graphs)
                (0.5 * (out - target) ** 2).sum().backward()
                torch.cuda.synchronize()
                grads[use_graphs].append([p0.grad.clone()] + [g.grad.clone() for g in gg])
    for eager, graph in zip(grads[False], grads[True]):
        for a, b in zip(eager, graph):
            assert torch.allclose(a, b, rtol=1e-12, atol=1e-14)
    assert not torch.allclose(grads[False][0][1], grads[False][1][1])


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_record_replay_equals_adjoint_step(shape, name, dtype):
    """The split reverse step (tape recorded with the step's result, then the reverse sweep
    from the tape) gives the one-call reverse step (up to the order of the scatter kernels'
    atomic additions), and the recorded step's result is the forward step (FP64: within
    1e-12 of the oracle)."""
    n_iters, opts = CASES[name]
    rng = np.random.default_rng(len(shape) * 7 + n_iters)
    psi = smooth_positive(shape, rng)
    if opts & capi.IGA:
        psi = psi - 2.0
    gc = nondivergent(shape, rng, 0.3)
    y = rng.normal(size=shape)
    dev = torch.device("cuda")
    t = lambda a: torch.tensor(a, dtype=dtype, device=dev)
    with Mpdata(shape, dtype=dtype, n_iters=n_iters, opts=opts) as m:
        p, g = t(psi), [t(v) for v in gc]
        pb1, gb1 = t(y), [torch.full(shape, 0.25, dtype=dtype, device=dev) for _ in shape]
        m.adjoint_step(p, g, pb1, gc_bar=gb1)
        tape = torch.full((m.tape_numel(),), float("nan"), dtype=dtype, device=dev)
        nxt = torch.empty_like(p)
        m.adjoint_record(p, g, tape, psi_next=nxt)
        pb2, gb2 = t(y), [torch.full(shape, 0.25, dtype=dtype, device=dev) for _ in shape]
        m.adjoint_replay(p, g, tape, pb2, gc_bar=gb2)
        torch.cuda.synchronize()
        rel = 1e-6 if dtype == torch.float32 else 1e-12  # 2D records on the fused kernels
        scale = max(float(pb1.abs().max()), max(float(v.abs().max()) for v in gb1))
        assert float((pb1 - pb2).abs().max()) <= rel * scale
        for a, b in zip(gb1, gb2):
            assert float((a - b).abs().max()) <= rel * scale
    ref = oracle.step(psi if dtype == torch.float64 else p.double().cpu().numpy(),
                      gc if dtype == torch.float64 else [v.double().cpu().numpy() for v in g],
                      n_iters=n_iters, opts=opts)
    tol = 1e-12 if dtype == torch.float64 else 2e-6
    assert np.abs(nxt.double().cpu().numpy() - ref).max() <= tol * np.abs(ref).max()


def test_tape_bytes_and_rejections():
    dev = torch.device("cuda")
    for shape, n_iters, opts, arrays in (((16, 12), 2, capi.FCT, 1 + 2 + 2 + 2 + 2), ((16, 12), 2, 0, 3),
                                         ((9, 8, 7), 3, capi.FCT, 2 * 4 + 6 + 2 + 4), ((40,), 1, capi.FCT, 2)):
        with Mpdata(shape, dtype=torch.float64, n_iters=n_iters, opts=opts) as m:
            assert m.tape_numel() == arrays * int(np.prod(shape))
    shape = (8, 8)
    z = [torch.zeros(shape, device=dev) for _ in range(3)]
    with Mpdata(shape, dtype=torch.float32, n_iters=2, opts=capi.FCT) as m:
        tape = torch.zeros(m.tape_numel(), device=dev)
        assert capi.mpdata_adjoint_record(m.h, z[0], z[:2], None, tape, z[0], raw=True) == capi.EINVAL
        assert capi.mpdata_adjoint_record(m.h, z[0], z[:2], None, None, z[1], raw=True) == capi.EINVAL
        assert capi.mpdata_adjoint_replay(m.h, z[0], z[:2], None, None, z[1], raw=True) == capi.EINVAL
    with Mpdata(shape, dtype=torch.float32, n_iters=2, opts=capi.RHS_EULER_A) as m:
        assert capi.mpdata_adjoint_record(m.h, z[0], z[:2], None, z[2], z[1], raw=True) == capi.EUNSUPPORTED


def test_taped_rollout_gradient_matches_untaped():
    """Backward through recorded tapes == backward that recomputes each tape, with graphs
    and without (states recomputed on the staged kernels instead of the fused ones: equal to
    FP64 rounding over the segment)."""
    from paper_1407_1309_gb300 import autograd
    psi0_np, gc_np, pert = workloads.adjoint_2d(80, seed=4)
    dev = torch.device("cuda")
    f64 = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    target = f64(psi0_np + 0.05 * pert)
    grads = []
    saved = autograd.tape_budget
    try:
        for budget, use_graphs in ((0, False), (None, False), (None, True)):
            autograd.tape_budget = budget
            with Mpdata((80, 80), dtype=torch.float64, n_iters=2, opts=capi.FCT) as m:
                gg = [f64(v).requires_grad_(True) for v in gc_np]
                p0 = f64(psi0_np).requires_grad_(True)
                out = rollout(m, p0, gg, 17, 6, use_graphs=use_graphs)
                (0.5 * (out - target) ** 2).sum().backward()
                torch.cuda.synchronize()
                grads.append([p0.grad.clone()] + [g.grad.clone() for g in gg])
    finally:
        autograd.tape_budget = saved
    for other in grads[1:]:
        for a, b in zip(grads[0], other):
            assert torch.allclose(a, b, rtol=1e-10, atol=1e-12 * float(a.abs().max()))


@pytest.mark.parametrize("shape", [(37, 150), (64, 64), (9, 1000)], ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("opts", [0, capi.FCT], ids=["basic", "fct"])
@pytest.mark.parametrize("family", [1, 2], ids=["warp", "band"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_fused_tape_matches_staged_tape(shape, opts, family, dtype):
    """2D: the fused step that records the tape in one launch (warp or band march) writes the
    arrays the staged recording writes (psi^(1), pseudo-advectors, bounds, factors capped at 1;
    the limited advectors are re-derived by the reverse step and left unwritten), to rounding;
    its step result is that family's forward step."""
    rng = np.random.default_rng(sum(shape) + opts)
    psi = smooth_positive(shape, rng)
    gc = nondivergent(shape, rng, 0.4)
    dev = torch.device("cuda")
    t = lambda a: torch.tensor(a, dtype=dtype, device=dev)
    tapes, nxts = {}, {}
    for staged in (False, True):
        with Mpdata(shape, dtype=dtype, n_iters=2, opts=opts | (capi.STAGED if staged else 0)) as m:
            p, g = t(psi), [t(v) for v in gc]
            if not staged:
                m.tune(capi.TUNE_KERNEL, family)
            tape = torch.full((m.tape_numel(),), float("nan"), dtype=dtype, device=dev)
            nxt = torch.empty_like(p)
            m.adjoint_record(p, g, tape, psi_next=nxt)
            if not staged:
                fwd = torch.empty_like(p)
                m.advance(p, fwd, g)
            torch.cuda.synchronize()
            tapes[staged], nxts[staged] = tape.view(-1, *shape).cpu().numpy(), nxt.cpu().numpy()
    f32 = dtype == torch.float32
    assert np.array_equal(nxts[False], fwd.cpu().numpy())
    assert np.abs(nxts[False] - nxts[True]).max() <= (1e-5 if f32 else 1e-13) * np.abs(psi).max()
    fused, ref = tapes[False], tapes[True]
    written = [0, 1, 2, 5, 6, 7, 8] if opts else [0, 1, 2]
    assert fused.shape[0] == (9 if opts else 3)
    if opts:
        ref[7:9] = np.minimum(ref[7:9], 1.0)
        assert np.isnan(fused[3:5]).all()
    for j in written:
        assert np.isfinite(fused[j]).all(), j
        scale = max(np.abs(ref[j]).max(), 1e-30)
        tol = (1e-3 if j >= 7 else 1e-5) if f32 else (1e-9 if j >= 7 else 1e-13)  # factors: small flux sums
        assert np.abs(fused[j] - ref[j]).max() <= tol * max(scale, 1.0), j


@pytest.mark.parametrize("shape", [(70, 45), (33, 97), (5, 200), (130, 3)], ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("name", ["basic", "fct"])
def test_adjoint_matches_oracle_on_larger_2d_fields(shape, name):
    """2D fields of several thread blocks with ragged edges, and fields narrower than the
    stencil: FP64 against the oracle adjoint to 1e-12, FP32 (inputs rounded to FP32) to 1e-5
    relative L2."""
    n_iters, opts = CASES[name]
    rng = np.random.default_rng(sum(shape) + n_iters)
    psi = smooth_positive(shape, rng)
    gc = nondivergent(shape, rng, 0.35)
    y = rng.normal(size=shape)
    dev = torch.device("cuda")
    for dtype in (torch.float64, torch.float32):
        r = (lambda a: a) if dtype == torch.float64 else (lambda a: a.astype(np.float32).astype(np.float64))
        p_, g_, y_ = r(psi), [r(v) for v in gc], r(y)
        ref_pb, ref_gcb = oracle.adj_step(p_, g_, y_, n_iters=n_iters, opts=opts)
        t = lambda a: torch.tensor(a, dtype=dtype, device=dev)
        with Mpdata(shape, dtype=dtype, n_iters=n_iters, opts=opts) as m:
            pb = t(y_)
            gcb = [torch.full(shape, 0.5, dtype=dtype, device=dev) for _ in shape]
            m.adjoint_step(t(p_), [t(v) for v in g_], pb, gc_bar=gcb)
            torch.cuda.synchronize()
            got_pb = pb.double().cpu().numpy()
            got_gcb = [v.double().cpu().numpy() - 0.5 for v in gcb]
        if dtype == torch.float64:
            scale = max(np.abs(ref_pb).max(), max(np.abs(v).max() for v in ref_gcb))
            assert np.abs(got_pb - ref_pb).max() <= 1e-12 * scale
            for a, b in zip(got_gcb, ref_gcb):
                assert np.abs(a - b).max() <= 1e-12 * scale
        else:
            assert np.linalg.norm(got_pb - ref_pb) <= 1e-5 * np.linalg.norm(ref_pb)
            for a, b in zip(got_gcb, ref_gcb):
                assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)


@pytest.mark.parametrize("name", ["basic", "fct"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_reverse_from_fused_tape_matches_staged_tape_512(name, dtype):
    """The reverse step on the 512^2 adjoint workload from the tape the fused step kernel
    records against the one the staged kernels record (MPDATA_STAGED): FP64 to 1e-12 (max-norm,
    relative to the largest adjoint), FP32 to 1e-5 relative L2 (the two FP32 tapes differ by
    rounding, which the ratios of Eq. 6 amplify where psi1 + psi1' is small)."""
    n_iters, opts = CASES[name]
    psi0_np, gc_np, pert = workloads.adjoint_2d(512, seed=5)
    y = np.random.default_rng(9).normal(size=psi0_np.shape)
    dev = torch.device("cuda")
    t = lambda a: torch.tensor(a, dtype=dtype, device=dev)
    res = []
    for staged in (False, True):
        with Mpdata(psi0_np.shape, dtype=dtype, n_iters=n_iters, opts=opts | (capi.STAGED if staged else 0)) as m:
            pb = t(y)
            gcb = [torch.zeros(psi0_np.shape, dtype=dtype, device=dev) for _ in range(2)]
            m.adjoint_step(t(psi0_np), [t(v) for v in gc_np], pb, gc_bar=gcb)
            torch.cuda.synchronize()
            res.append([pb.double().cpu().numpy()] + [v.double().cpu().numpy() for v in gcb])
    scale = max(np.abs(a).max() for a in res[1])
    for a, b in zip(res[0], res[1]):
        if dtype == torch.float64:
            assert np.abs(a - b).max() <= 1e-12 * scale
        else:
            assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)


def test_forward_recorded_segments_are_used_only_by_their_own_backward():
    """With graphs and tapes the forward records its last two segments for the backward, in the
    backward's buffers; a second rollout on the same handle takes those buffers over, and the
    first rollout's backward then recomputes its segments: the gradients equal those of a
    rollout whose backward follows its forward directly."""
    psi0_np, gc_np, pert = workloads.adjoint_2d(64, seed=3)
    dev = torch.device("cuda")
    f64 = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    target = f64(psi0_np + 0.05 * pert)

    def grads(interleave):
        with Mpdata((64, 64), dtype=torch.float64, n_iters=2, opts=capi.FCT) as m:
            gg = [f64(v).requires_grad_(True) for v in gc_np]
            p0 = f64(psi0_np).requires_grad_(True)
            out = rollout(m, p0, gg, 30, 7)
            if interleave:
                q0 = f64(0.9 * psi0_np).requires_grad_(True)
                other = rollout(m, q0, [f64(1.1 * v).requires_grad_(True) for v in gc_np], 30, 7)
                assert other.shape == out.shape
            (0.5 * (out - target) ** 2).sum().backward()
            torch.cuda.synchronize()
            return [p0.grad.clone()] + [g.grad.clone() for g in gg]

    direct, interleaved = grads(False), grads(True)
    for a, b in zip(direct, interleaved):
        assert torch.allclose(a, b, rtol=1e-12, atol=1e-14 * float(a.abs().max()))
