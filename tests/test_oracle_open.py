"""Pins of the oracle's open edges (Sect. 2.4: bcond::open, a zero-divergence condition on the
domain edges), read as: the halo cells beyond an open edge hold the edge value; the n-1 faces
between the cells along an open dimension are interior, and each boundary face carries the
value of the adjacent interior face for every vector field (the advector and each pass's
pseudo-velocity, limited or not), so that its flux is that value times the edge cell's psi.

Each test names what fixes the expected result: agreement with the periodic scheme while no
stencil reaches a non-constant value across an edge, the exact shift at |C| = 1 with the edge
value flowing in, the flux-form budget (interior fluxes telescope, only the two boundary fluxes
remain), constant preservation, mirror symmetry, and the FCT bounds in the domain interior.
"""
import numpy as np
import pytest

import oracle
from paper_1407_1309_gb300 import workloads as wl

OPEN = (oracle.OPEN0, oracle.OPEN1, oracle.OPEN2)
OPTION_SETS = {
    "donor": (1, 0),
    "basic": (2, 0),
    "fct": (2, oracle.FCT),
    "it3_fct": (3, oracle.FCT),
    "tot3_fct": (3, oracle.TOT | oracle.FCT),
    "iga_fct": (2, oracle.IGA | oracle.FCT),
    "iga_tot_fct": (2, oracle.IGA | oracle.TOT | oracle.FCT),
    "kahan_fct": (2, oracle.KAHAN | oracle.FCT),
    "abs_fct": (2, oracle.ABS | oracle.FCT),
    "dfl_fct": (2, oracle.DFL | oracle.FCT),
}


def all_open(nd):
    return sum(OPEN[:nd])


def central_blob(shape, c=1.5, r=3):
    psi = np.full(shape, c)
    idx = tuple(slice(n // 2 - r, n // 2 + r + 1) for n in shape)
    rng = np.random.default_rng(len(shape))
    psi[idx] += rng.uniform(0.5, 2.0, size=psi[idx].shape)
    return psi


@pytest.mark.parametrize("shape", [(64,), (48, 44), (34, 32, 30)], ids=lambda s: f"{len(s)}d")
@pytest.mark.parametrize("name", sorted(OPTION_SETS))
def test_open_equals_periodic_away_from_the_edges(shape, name):
    """With a uniform advector and psi constant within the stencil's reach of every edge, a
    stencil that crosses an edge reads the same values under both conditions (the edge value,
    the uniform advector), so open and periodic edges give the same result bit for bit."""
    n_iters, opts = OPTION_SETS[name]
    if len(shape) == 3 and name not in ("tot3_fct", "iga_tot_fct", "fct"):
        pytest.skip("3D: the options that widen the stencil most")
    psi = central_blob(shape)
    gc = [np.full(shape, v) for v in (0.3, -0.2, 0.25)[:len(shape)]]
    per = oracle.step(psi, gc, n_iters=n_iters, opts=opts, n_steps=2)
    opn = oracle.step(psi, gc, n_iters=n_iters, opts=opts | all_open(len(shape)), n_steps=2)
    np.testing.assert_array_equal(opn, per)
    # the unread last advector entry along an open dimension changes nothing
    gc2 = [v.copy() for v in gc]
    for d, v in enumerate(gc2):
        v[(slice(None),) * d + (-1,)] = 7.0
    np.testing.assert_array_equal(oracle.step(psi, gc2, n_iters=n_iters, opts=opts | all_open(len(shape)),
                                              n_steps=2), opn)


@pytest.mark.parametrize("courant", [1.0, -1.0])
@pytest.mark.parametrize("name", sorted(OPTION_SETS))
def test_open_exact_shift_with_inflow_of_the_edge_value(courant, name):
    """At |C| = 1 every corrective advector vanishes (|C| - C^2 = 0) and the donor pass moves psi
    one cell per step: the signal leaves through the downstream edge and the upstream edge cell,
    whose inflow carries its own value (halo = edge value), keeps that value."""
    n_iters, opts = OPTION_SETS[name]
    if opts & oracle.DFL:
        pytest.skip("the divergent-flow term needs an advector difference; uniform here (it is zero)")
    rng = np.random.default_rng(4)
    n, k = 23, 5
    psi = rng.uniform(0.1, 3.0, size=n)
    out = oracle.step(psi, [np.full(n, courant)], n_iters=n_iters, opts=opts | oracle.OPEN0, n_steps=k)
    if courant > 0:
        expect = np.concatenate([np.full(k, psi[0]), psi[:n - k]])
        np.testing.assert_array_equal(out, expect)
    else:
        expect = np.concatenate([psi[k:], np.full(k, psi[-1])])
        np.testing.assert_allclose(out, expect, rtol=4 * 2.0 ** -52, atol=0)


@pytest.mark.parametrize("opened", [(0,), (1,), (0, 1)], ids=lambda o: "open" + "".join(map(str, o)))
def test_open_donor_budget(opened):
    """Eq. 4 is in flux form: summed over the domain the interior fluxes cancel and the change of
    sum(psi) is what enters through the boundary faces of the open dimensions, F_{-1/2} - F_{n-1/2}
    with F_{-1/2} = V_{1/2} psi_0 and F_{n-1/2} = V_{n-3/2} psi_{n-1} (periodic dimensions add
    nothing)."""
    rng = np.random.default_rng(9)
    shape = (17, 13)
    psi = rng.uniform(0.5, 2.0, size=shape)
    gc = [rng.uniform(-0.2, 0.2, size=shape) for _ in range(2)]
    opts = sum(OPEN[d] for d in opened)
    out = oracle.step(psi, gc, n_iters=1, opts=opts)
    budget = 0.0
    for d in opened:
        first = (slice(None),) * d + (0,)
        last = (slice(None),) * d + (-1,)
        face_first = (slice(None),) * d + (0,)
        face_last = (slice(None),) * d + (-2,)
        budget += (gc[d][face_first] * psi[first]).sum() - (gc[d][face_last] * psi[last]).sum()
    assert abs((out.sum() - psi.sum()) - budget) <= 1e-13 * psi.sum()


@pytest.mark.parametrize("shape", [(37,), (12, 9), (6, 5, 7)], ids=lambda s: f"{len(s)}d")
@pytest.mark.parametrize("name", sorted(OPTION_SETS))
def test_open_constant_preserved_in_uniform_flow(shape, name):
    """psi = const under a uniform advector: every psi difference vanishes, and at an open edge
    the inflow (edge value times the copied advector) equals the outflow of the edge cell."""
    n_iters, opts = OPTION_SETS[name]
    gc = [np.full(shape, v) for v in (0.3, -0.2, 0.25)[:len(shape)]]
    G = 1.0 + 0.3 * np.random.default_rng(2).uniform(size=shape)
    psi = np.full(shape, 3.25)
    for g in (None, G):
        out = oracle.step(psi, gc, g=g, n_iters=n_iters, opts=opts | all_open(len(shape)), n_steps=5)
        assert np.abs(out - 3.25).max() <= 1e-14 * 3.25 * 8


@pytest.mark.parametrize("name", sorted(OPTION_SETS))
def test_open_mirror_symmetry(name):
    """Open edges have no preferred side: mirroring dimension 0 (cell i -> n-1-i, interior face
    i+1/2 -> (n-2-i)+1/2, V_0 negated) mirrors the result."""
    n_iters, opts = OPTION_SETS[name]
    rng = np.random.default_rng(6)
    shape = (11, 10)
    gc = [rng.uniform(-0.3, 0.3, size=shape) for _ in range(2)]
    psi = rng.uniform(0.5, 2.0, size=shape)
    o = opts | oracle.OPEN0 | oracle.OPEN1
    out = oracle.step(psi, gc, n_iters=n_iters, opts=o, n_steps=4)
    m = lambda a: a[::-1]
    mface = lambda v: -np.roll(v[::-1], -1, axis=0)
    outm = oracle.step(m(psi), [mface(gc[0]), m(gc[1])], n_iters=n_iters, opts=o, n_steps=4)
    np.testing.assert_allclose(outm, m(out), rtol=1e-13, atol=1e-13)


def test_open_hello_world_runs_as_printed():
    """Sect. 3.3: 101 points, C = 0.5, 100 steps, open edges, the library's default options
    (two passes, FCT, infinite gauge, compensated summation).  The Agnesi profile moves 50 cells
    to the right edge; with the limiter the field stays within its initial bounds in the
    interior, and nothing but the edge values enters."""
    psi, gc = wl.agnesi_1d()
    opts = oracle.FCT | oracle.IGA | oracle.KAHAN | oracle.OPEN0
    out = oracle.step(psi, gc, n_iters=2, opts=opts, n_steps=100)
    assert np.isfinite(out).all()
    lo, hi = psi.min(), psi.max()
    assert out.min() >= lo - 1e-12 and out.max() <= hi + 1e-12
    # the upstream edge keeps its value: only psi_0 flows in
    assert abs(out[0] - psi[0]) <= 1e-14
    # the peak has travelled 50 cells (C = 0.5, 100 steps) to the downstream edge region
    assert np.argmax(out) >= 95
