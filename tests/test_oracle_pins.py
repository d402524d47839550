"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  None of them re-types the oracle's
formulas: they check hand-worked values, exact invariants (conservation,
sign and constant preservation, exact shifts, symmetries), the paper's
convergence-order claims (Sect. 3.5) and derivative consistency (finite
differences, adjoint dot products).  A plausible slip anywhere in the oracle
(a dropped term, a wrong sign or index, a transposed operand) breaks at least
one of them.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1407_1309_gb300 import workloads as wl
from helpers import nondivergent

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

OPTION_SETS = {
    "donor": (1, 0),
    "basic": (2, 0),
    "fct": (2, oracle.FCT),
    "it3_fct": (3, oracle.FCT),
    "tot3": (3, oracle.TOT),
    "tot3_fct": (3, oracle.TOT | oracle.FCT),
    "iga": (2, oracle.IGA),
    "iga_fct": (2, oracle.IGA | oracle.FCT),
    "iga_tot_fct": (2, oracle.IGA | oracle.TOT | oracle.FCT),
    "kahan_fct": (2, oracle.KAHAN | oracle.FCT),
    "abs_fct": (2, oracle.ABS | oracle.FCT),
    "abs_tot3": (3, oracle.ABS | oracle.TOT),
    "dfl": (2, oracle.DFL),
    "dfl_it3_fct": (3, oracle.DFL | oracle.FCT),
}


SHAPES = [(37,), (12, 9), (6, 5, 7)]


# ----------------------------------------------------------------------------- P1

def test_four_cell_hand_example():
    """Sect. 3.1.1, Eqs. 4-6: the hand-worked 4-cell step (tests/golden/four_cell_basic.json)."""
    with open(os.path.join(GOLDEN, "four_cell_basic.json")) as f:
        gold = json.load(f)
    psi = np.array(gold["psi"], dtype=float)
    expect = np.array([float(Fraction(a, b)) for a, b in gold["result"]])
    out = oracle.step(psi, [np.full(4, gold["courant"])], n_iters=gold["n_iters"])
    np.testing.assert_allclose(out, expect, rtol=3e-16, atol=0)  # a few ulps: 1/6, 1/24 are inexact in binary
    # pass 1 alone is the donor-cell step of the same data
    p1 = oracle.step(psi, [np.full(4, gold["courant"])], n_iters=1)
    np.testing.assert_array_equal(p1, [float(Fraction(a, b)) for a, b in gold["pass1"]])
    # with Kahan summation the same exact values
    outk = oracle.step(psi, [np.full(4, gold["courant"])], n_iters=2, opts=oracle.KAHAN)
    np.testing.assert_allclose(outk, expect, rtol=3e-16, atol=0)


# ----------------------------------------------------------------------------- P2

@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
@pytest.mark.parametrize("name", sorted(OPTION_SETS))
def test_conservation(shape, name):
    """Eq. 4 is in flux form: on a periodic grid sum_i G_i psi_i is invariant."""
    n_iters, opts = OPTION_SETS[name]
    rng = np.random.default_rng(1)
    G = 1.0 + 0.3 * rng.uniform(size=shape)
    gc = nondivergent(shape, rng, 0.3)
    gc = [v * 1.0 for v in gc]
    psi = rng.uniform(0.5, 2.0, size=shape)
    m0 = oracle.mass(psi, G)
    out = oracle.step(psi, gc, g=G, n_iters=n_iters, opts=opts, n_steps=40)
    assert abs(oracle.mass(out, G) - m0) <= 1e-13 * abs(m0)
    out1 = oracle.step(psi, gc, n_iters=n_iters, opts=opts, n_steps=40)
    assert abs(out1.sum() - psi.sum()) <= 1e-13 * psi.sum()


# ----------------------------------------------------------------------------- P3

@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
@pytest.mark.parametrize("name", sorted(OPTION_SETS))
def test_constant_preserved(shape, name):
    """A constant field stays constant in a discretely nondivergent flow (Eq. 3 with
    div(G u) = 0, Eq. 2): every psi difference in Eq. 6 and its extensions vanishes."""
    n_iters, opts = OPTION_SETS[name]
    rng = np.random.default_rng(2)
    gc = nondivergent(shape, rng, 0.3)
    G = 1.0 + 0.3 * rng.uniform(size=shape)
    psi = np.full(shape, 3.25)
    for g in (None, G):
        out = oracle.step(psi, gc, g=g, n_iters=n_iters, opts=opts, n_steps=5)
        assert np.abs(out - 3.25).max() <= 1e-14 * 3.25 * 8


@pytest.mark.parametrize("name", ["donor", "basic", "fct", "it3_fct"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
def test_sign_preserving(shape, name):
    """MPDATA is sign-preserving (Sect. 1, footnote; Sect. 3.1.4): psi >= 0 stays >= 0."""
    n_iters, opts = OPTION_SETS[name]
    rng = np.random.default_rng(3)
    gc = nondivergent(shape, rng, 0.3)
    psi = np.where(rng.uniform(size=shape) < 0.5, 0.0, rng.uniform(0, 5, size=shape))
    out = oracle.step(psi, gc, n_iters=n_iters, opts=opts, n_steps=20)
    assert out.min() >= 0.0


# ----------------------------------------------------------------------------- P4

@pytest.mark.parametrize("courant", [1.0, -1.0])
@pytest.mark.parametrize("name", sorted(OPTION_SETS))
def test_exact_shift(courant, name):
    """At |C| = 1 the donor-cell pass (Eqs. 4-5) moves psi by one cell exactly, and
    |C| - C^2 = 0 makes every corrective advector vanish (Eq. 6), so full MPDATA
    moves it exactly too.  With the summation order psi - F_{i+1/2} + F_{i-1/2} the
    shift is bit-exact for C = +1 (psi_i - psi_i + psi_{i-1}); for C = -1 the sum
    (psi_i + psi_{i+1}) - psi_i may round once per step (also with Kahan summation,
    whose last compensation is not added back)."""
    n_iters, opts = OPTION_SETS[name]
    exact = courant > 0
    check = (np.testing.assert_array_equal if exact else
             lambda a, b: np.testing.assert_allclose(a, b, rtol=4 * 2.0 ** -52, atol=0))
    rng = np.random.default_rng(4)
    psi = rng.uniform(0.1, 3.0, size=23)
    out = oracle.step(psi, [np.full(23, courant)], n_iters=n_iters, opts=opts, n_steps=3)
    check(out, np.roll(psi, 3 if courant > 0 else -3))
    # 2D: C = (1, 0) shifts along dimension 0 only
    psi2 = rng.uniform(0.1, 3.0, size=(9, 8))
    out2 = oracle.step(psi2, [np.full((9, 8), courant), np.zeros((9, 8))], n_iters=n_iters, opts=opts)
    check(out2, np.roll(psi2, 1 if courant > 0 else -1, axis=0))


# ----------------------------------------------------------------------------- P5

@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
@pytest.mark.parametrize("name", sorted(OPTION_SETS))
def test_homogeneity_and_odd_symmetry(shape, name):
    """Every psi-dependence of the scheme is a ratio of psi values (Eq. 6) or linear
    (Eqs. 4-5), so step(2 psi) = 2 step(psi) and step(-psi) = -step(psi) bit for bit."""
    n_iters, opts = OPTION_SETS[name]
    rng = np.random.default_rng(5)
    gc = nondivergent(shape, rng, 0.3)
    psi = rng.uniform(0.5, 2.0, size=shape)
    out = oracle.step(psi, gc, n_iters=n_iters, opts=opts, n_steps=3)
    np.testing.assert_array_equal(oracle.step(2 * psi, gc, n_iters=n_iters, opts=opts, n_steps=3), 2 * out)
    np.testing.assert_array_equal(oracle.step(-psi, gc, n_iters=n_iters, opts=opts, n_steps=3), -out)


@pytest.mark.parametrize("name", sorted(OPTION_SETS))
def test_mirror_and_axis_permutation(name):
    """The scheme has no preferred direction: mirroring x (with V_x negated and moved
    to the mirrored faces) mirrors the result; swapping the axes swaps it."""
    n_iters, opts = OPTION_SETS[name]
    rng = np.random.default_rng(6)
    shape = (11, 10)
    gc = nondivergent(shape, rng, 0.35)
    psi = rng.uniform(0.5, 2.0, size=shape)
    out = oracle.step(psi, gc, n_iters=n_iters, opts=opts, n_steps=4)
    # mirror along axis 0: cell i -> N-1-i, face i+1/2 -> face N-2-i
    m = lambda a: a[::-1]
    mface = lambda v: -np.roll(v[::-1], -1, axis=0)
    outm = oracle.step(m(psi), [mface(gc[0]), m(gc[1])], n_iters=n_iters, opts=opts, n_steps=4)
    np.testing.assert_allclose(outm, m(out), rtol=1e-13, atol=1e-13)
    # axis swap
    outt = oracle.step(psi.T, [gc[1].T, gc[0].T], n_iters=n_iters, opts=opts, n_steps=4)
    np.testing.assert_allclose(outt, out.T, rtol=1e-13, atol=1e-13)


def test_infinite_gauge_is_linear_and_background_free():
    """Sect. 3.1.5 / 3.4.1: infinite gauge is the linear limit of MPDATA; its result
    does not depend on a constant background (nondivergent flow)."""
    rng = np.random.default_rng(7)
    shape = (14, 13)
    gc = nondivergent(shape, rng, 0.35)
    a, b = rng.normal(size=shape), rng.normal(size=shape)
    st = lambda p: oracle.step(p, gc, n_iters=2, opts=oracle.IGA | oracle.TOT, n_steps=3)
    np.testing.assert_allclose(st(2 * a - 3 * b), 2 * st(a) - 3 * st(b), atol=1e-13)
    np.testing.assert_allclose(st(a + 7.0), st(a) + 7.0, atol=1e-12)
    # the basic scheme is not background-free (Sect. 3.4.1: ripples depend on the background)
    bs = lambda p: oracle.step(p, gc, n_iters=2, n_steps=3)
    assert np.abs(bs(np.abs(a) + 7.0) - (bs(np.abs(a)) + 7.0)).max() > 1e-6


# ----------------------------------------------------------------------------- P6

@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
@pytest.mark.parametrize("name", ["fct", "it3_fct", "tot3_fct", "iga_fct", "iga_tot_fct"])
def test_fct_bounds(shape, name):
    """Sect. 3.1.4: the limited solution stays within the local bounds of psi^n and the
    donor-cell solution (Zalesak-type limiter of Smolarkiewicz & Grabowski 1990)."""
    n_iters, opts = OPTION_SETS[name]
    rng = np.random.default_rng(8)
    gc = nondivergent(shape, rng, 0.35)
    psi = np.where(rng.uniform(size=shape) < 0.3, 4.0, 1.0)   # boxcars: sharp gradients
    if opts & oracle.IGA:
        psi = psi - 2.5                                          # variable sign under iga
    out, mx, mn = oracle.step(psi, gc, n_iters=n_iters, opts=opts, return_bounds=True)
    tol = 1e-13 * np.abs(psi).max()
    assert (out <= mx + tol).all() and (out >= mn - tol).all()
    # the bounds are taken over the cell and its face neighbours of both psi^n and the
    # donor-cell (first-pass) solution
    first = oracle.step(psi, gc, n_iters=1)
    for f in (psi, first):
        for d in range(len(shape)):
            for s_ in (-1, 0, 1):
                assert (mx >= np.roll(f, s_, d)).all() and (mn <= np.roll(f, s_, d)).all()
    # without the limiter the same data over/undershoots
    plain = oracle.step(psi, gc, n_iters=n_iters, opts=opts & ~oracle.FCT)
    assert ((plain > mx + tol) | (plain < mn - tol)).any()


# ----------------------------------------------------------------------------- P7

def _conv_1d(C, k, n_iters, opts):
    """Sect. 3.5: X = 44 dx_m, T = 1, u = 1, cell-mean Gaussian (Eq. 7, sigma = 1.5,
    x0 = X/2); error of Eq. 8 after one unit of time."""
    dx = 2.0 ** -k
    nx = int(round(44.0 / dx))
    nt = int(round(1.0 / (C * dx)))
    psi = wl.gaussian_1d_cell_means(nx, dx, 22.0, 1.5)
    ex = wl.gaussian_1d_cell_means(nx, dx, 23.0, 1.5)
    out = oracle.step(psi, [np.full(nx, C)], n_iters=n_iters, opts=opts, n_steps=nt)
    return math.sqrt(np.mean((ex - out) ** 2))


def _order(errs):
    return math.log2(errs[-2] / errs[-1])


@pytest.mark.parametrize("name,C,lo,hi", [
    ("donor", 0.25, 0.9, 1.1), ("donor", 0.5, 0.9, 1.1),           # Fig. 3_it1: first order
    ("basic", 0.25, 1.9, 2.1), ("basic", 0.5, 1.9, 2.1),           # Fig. 3_it2: second order
    ("it3", 0.5, 2.85, 3.15), ("it3", 0.25, 1.9, 2.3),              # Fig. 3_it3: third-order groove at 45 deg (C = 0.5)
    ("tot3", 0.25, 2.85, 3.15), ("tot3", 0.5, 2.85, 3.15),          # Fig. 3_tot: third order, >= 3 passes
    ("fct", 0.25, 1.7, 2.1), ("fct", 0.5, 1.7, 2.1),                # Fig. 3_fct: from 2 to ~1.8
    ("iga", 0.5, 2.85, 3.15), ("iga", 0.25, 1.9, 2.3),              # Fig. 3_iga: as accurate as three passes
    ("iga_tot", 0.25, 2.85, 3.15), ("iga_tot", 0.5, 2.85, 3.15),    # Fig. 3_iga_tot
])
def test_convergence_order_1d(name, C, lo, hi):
    """Sect. 3.5: convergence orders read along lines of constant Courant number."""
    n_iters, opts = {"donor": (1, 0), "basic": (2, 0), "it3": (3, 0), "tot3": (3, oracle.TOT),
                     "fct": (2, oracle.FCT), "iga": (2, oracle.IGA),
                     "iga_tot": (2, oracle.IGA | oracle.TOT)}[name]
    errs = [_conv_1d(C, k, n_iters, opts) for k in (2, 3, 4)]
    assert lo <= _order(errs) <= hi


def _conv_nd(C, k, n_iters, opts, X, sig):
    nd = len(C)
    dx = 2.0 ** -k
    nx = int(round(X / dx))
    nt = int(round(1.0 / (abs(C[0]) * dx)))
    g1 = lambda x0: sum(wl.gaussian_1d_cell_means(nx, dx, x0 + m * X, sig) for m in (-2, -1, 0, 1, 2))
    psi = g1(X / 2)
    ex = g1(X / 2 + C[0] / abs(C[0]))
    for q in range(1, nd):
        psi = np.multiply.outer(psi, g1(X / 2))
        ex = np.multiply.outer(ex, g1(X / 2 + C[q] / abs(C[0])))
    out = oracle.step(psi, [np.full(psi.shape, c) for c in C], n_iters=n_iters, opts=opts, n_steps=nt)
    return math.sqrt(np.mean((ex - out) ** 2))


@pytest.mark.parametrize("name,C,lo", [
    ("basic", (0.25, 0.25), 1.9), ("basic", (0.4, -0.2), 1.9),     # cross term: 2nd order on diagonal flow
    ("tot3", (0.25, 0.25), 2.8), ("tot3", (0.4, -0.2), 2.8),        # pairwise third-order terms
    ("iga_tot", (0.25, 0.25), 2.9), ("iga_tot", (0.4, -0.2), 2.9),
])
def test_convergence_order_2d_diagonal(name, C, lo):
    """Multi-D terms (Sect. 3.1.1 footnote and 3.1.2): second order for the basic scheme
    and third order with the third-order option on a flow oblique to the grid."""
    n_iters, opts = {"basic": (2, 0), "tot3": (3, oracle.TOT), "iga_tot": (2, oracle.IGA | oracle.TOT)}[name]
    errs = [_conv_nd(C, k, n_iters, opts, 16.0, 1.5) for k in (1, 2, 3)]
    assert _order(errs) >= lo


@pytest.mark.parametrize("name,C,lo", [
    ("basic", (0.25, 0.15, -0.1), 1.9),
    ("tot3", (0.25, 0.25, 0.25), 2.8),          # triple term matters when C_x C_y C_z is large
    ("iga_tot", (0.25, 0.25, -0.25), 2.85),
])
def test_convergence_order_3d_oblique(name, C, lo):
    """3D: the triple term of the third-order option (Sect. 3.1.2) is needed for third order."""
    n_iters, opts = {"basic": (2, 0), "tot3": (3, oracle.TOT), "iga_tot": (2, oracle.IGA | oracle.TOT)}[name]
    errs = [_conv_nd(C, k, n_iters, opts, 8.0, 1.0) for k in (1, 2, 3)]
    assert _order(errs) >= lo


# ----------------------------------------------------------------------------- sources, G

def test_source_terms_euler_a_and_b():
    """Sect. 4.1: euler_a adds dt R after advection, euler_b before (exact at C = 1)."""
    rng = np.random.default_rng(9)
    psi, R = rng.uniform(1, 2, size=17), rng.uniform(-1, 1, size=17)
    gc = [np.ones(17)]
    a = oracle.step(psi, gc, r=R, dt=0.5, n_iters=2, opts=oracle.FCT, rhs="euler_a")
    b = oracle.step(psi, gc, r=R, dt=0.5, n_iters=2, opts=oracle.FCT, rhs="euler_b")
    np.testing.assert_array_equal(a, np.roll(psi, 1) + 0.5 * R)
    np.testing.assert_array_equal(b, np.roll(psi + 0.5 * R, 1))
    # no flow: psi + dt R either way
    z = [np.zeros(17)]
    np.testing.assert_array_equal(oracle.step(psi, z, r=R, dt=0.25, rhs="euler_a"), psi + 0.25 * R)


def test_uniform_g_is_scale_free():
    """Eq. 3: with a uniform G = g0 and advector g0 C the step equals the G = 1 step with C."""
    rng = np.random.default_rng(10)
    shape = (10, 9)
    gc = nondivergent(shape, rng, 0.35)
    psi = rng.uniform(0.5, 2.0, size=shape)
    for n_iters, opts in OPTION_SETS.values():
        a = oracle.step(psi, gc, n_iters=n_iters, opts=opts, n_steps=3)
        b = oracle.step(psi, [2.5 * v for v in gc], g=np.full(shape, 2.5), n_iters=n_iters, opts=opts, n_steps=3)
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-13)


def test_config1_one_transit_error():
    """1D configuration (N = 500, C = 0.5, 1000 steps = one transit): the result
    approximates the initial profile; the error is reported, not bounded tightly."""
    psi, gc = wl.hello_1d()
    out = oracle.step(psi, gc, n_iters=2, n_steps=1000)
    assert abs(out.sum() - psi.sum()) < 1e-10
    err = np.sqrt(np.mean((out - psi) ** 2))
    assert err < 0.1


# ----------------------------------------------------------------------------- P9

@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
@pytest.mark.parametrize("name", ["basic", "fct", "tot3_fct", "iga_tot_fct", "kahan_fct"])
def test_tangent_linear_matches_central_differences(shape, name):
    """The tangent-linear step agrees with central finite differences of the forward step
    on smooth, strictly positive, generic data (seeded random low modes: no flat regions
    and no symmetric ties, so the limiter's min/max selections are differentiable there)."""
    n_iters, opts = OPTION_SETS[name]
    rng = np.random.default_rng(11)
    f = wl.low_modes(rng, shape, 6)
    psi = 2.0 + 0.5 * f / np.abs(f).max()
    gc = nondivergent(shape, rng, 0.3)
    dpsi = rng.normal(size=shape)
    dgc = [rng.normal(size=shape) * 0.1 for _ in shape]
    tl = oracle.tl_step(psi, gc, dpsi, dgc, n_iters=n_iters, opts=opts)
    eps = 1e-6
    fp = oracle.step(psi + eps * dpsi, [v + eps * dv for v, dv in zip(gc, dgc)], n_iters=n_iters, opts=opts)
    fm = oracle.step(psi - eps * dpsi, [v - eps * dv for v, dv in zip(gc, dgc)], n_iters=n_iters, opts=opts)
    fd = (fp - fm) / (2 * eps)
    assert np.linalg.norm(fd - tl) <= 1e-8 * np.linalg.norm(tl)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
@pytest.mark.parametrize("name", ["basic", "fct", "tot3_fct", "iga_tot_fct"])
def test_adjoint_dot_product(shape, name):
    """<TL dx, y> = <dx, AD y> for the step's Jacobian with respect to (psi, GC)."""
    n_iters, opts = OPTION_SETS[name]
    rng = np.random.default_rng(12)
    psi = rng.uniform(1.0, 3.0, size=shape)
    gc = nondivergent(shape, rng, 0.3)
    dpsi = rng.normal(size=shape)
    dgc = [rng.normal(size=shape) for _ in shape]
    y = rng.normal(size=shape)
    tl = oracle.tl_step(psi, gc, dpsi, dgc, n_iters=n_iters, opts=opts)
    pb, gcb = oracle.adj_step(psi, gc, y, n_iters=n_iters, opts=opts)
    lhs = float(np.sum(tl * y))
    rhs = float(np.sum(dpsi * pb) + sum(np.sum(a * b) for a, b in zip(dgc, gcb)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


# ----------------------------------------------------------------------------- variable-sign option (abs)

ABS_SETS = {"basic": (2, 0), "fct": (2, oracle.FCT), "it3_fct": (3, oracle.FCT), "tot3_fct": (3, oracle.TOT | oracle.FCT)}


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
@pytest.mark.parametrize("name", sorted(ABS_SETS))
def test_abs_equals_the_basic_scheme_on_one_signed_fields(shape, name):
    """Sect. 3.1.5: the abs option replaces psi by |psi| in the psi-fractions only, so on a
    positive field it is the basic scheme, bit for bit, and on a negative field the basic
    scheme's odd reflection."""
    n_iters, opts = ABS_SETS[name]
    rng = np.random.default_rng(len(shape) + n_iters)
    gc = nondivergent(shape, rng, 0.4)
    psi = 1.0 + rng.uniform(size=shape)
    st = lambda p, o: oracle.step(p, gc, n_iters=n_iters, opts=o, n_steps=3)
    assert np.array_equal(st(psi, opts | oracle.ABS), st(psi, opts))
    assert np.array_equal(st(-psi, opts | oracle.ABS), -st(psi, opts))


def test_abs_keeps_the_psi_fraction_bounded():
    """Sect. 3.1.5: with a variable-sign field the psi-fraction of Eq. 6 is unbounded where two
    neighbouring values nearly cancel (here psi^(1) = 1 and -1 + 1e-6 after the donor pass at
    C = 1/2, so the basic scheme's pseudo-velocity is about -5e5); with |psi| it stays within
    [-1, 1] and the step stays within the initial range.  Both conserve the sum."""
    eps = 1e-6
    psi = np.array([0.5, 1.0, 1.0, -3.0 + 2 * eps, -2.0, -1.0, 0.0, 0.2])
    gc = [np.full(psi.shape, 0.5)]
    basic = oracle.step(psi, gc, n_iters=2)
    absv = oracle.step(psi, gc, n_iters=2, opts=oracle.ABS)
    assert np.abs(basic).max() > 1e5
    assert np.abs(absv).max() <= np.abs(psi).max()
    for out in (basic, absv):
        assert abs(out.sum() - psi.sum()) <= 1e-9 * np.abs(psi).sum()


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
@pytest.mark.parametrize("name", ["fct", "tot3_fct"])
def test_abs_on_variable_sign_fields(shape, name):
    """abs on a variable-sign field: conservation (the fluxes telescope, Eq. 4), odd symmetry
    and scaling by powers of two (|psi| fractions are invariant under both; exact in floating
    point), the FCT bounds (Sect. 3.1.4), and a constant field of either sign is kept."""
    n_iters, opts = ABS_SETS[name]
    opts |= oracle.ABS
    rng = np.random.default_rng(11 * len(shape))
    gc = nondivergent(shape, rng, 0.4)
    psi = rng.normal(size=shape)
    st = lambda p: oracle.step(p, gc, n_iters=n_iters, opts=opts, n_steps=5)
    out = st(psi)
    assert abs(out.sum() - psi.sum()) <= 1e-13 * np.abs(psi).sum() * 5
    assert np.array_equal(st(-psi), -out)
    assert np.array_equal(st(4.0 * psi), 4.0 * out)
    one = oracle.step(psi, gc, n_iters=n_iters, opts=opts)
    assert one.max() <= psi.max() + 1e-12 and one.min() >= psi.min() - 1e-12
    for c in (2.5, -2.5):
        const = st(np.full(shape, c))
        assert np.abs(const - c).max() <= 1e-13 * abs(c)


def test_abs_depends_on_the_background_and_excludes_iga():
    """Sect. 3.4.1 (the abs results' ripples depend on the constant background, unlike the
    infinite gauge, the linear limit): abs(psi + c) != abs(psi) + c; and abs and the infinite
    gauge are alternatives (the combination is rejected)."""
    rng = np.random.default_rng(5)
    shape = (14, 13)
    gc = nondivergent(shape, rng, 0.35)
    a = rng.normal(size=shape)
    st = lambda p: oracle.step(p, gc, n_iters=2, opts=oracle.ABS, n_steps=3)
    assert np.abs(st(a + 3.0) - (st(a) + 3.0)).max() > 1e-6
    with pytest.raises(ValueError):
        oracle.step(a, gc, n_iters=2, opts=oracle.ABS | oracle.IGA)


# ----------------------------------------------------------------------------- divergent-flow option (dfl)

def _gl_means(f, n, pts=5):
    """Cell means on [0, 1) with n cells by Gauss-Legendre quadrature."""
    gx, gw = np.polynomial.legendre.leggauss(pts)
    dx = 1.0 / n
    q = ((np.arange(n) + 0.5) * dx)[:, None] + 0.5 * dx * gx[None, :]
    return q, gw, (f(q) * gw[None, :]).sum(1) / 2.0


def _foot(vel, x, t):
    """Foot at time 0 of the characteristic dx/dt = vel(x) through x at time t (steady flow)."""
    integrate = pytest.importorskip("scipy.integrate")
    sol = integrate.solve_ivp(lambda s, X: -vel(X), (0.0, t), x.ravel(), rtol=1e-12, atol=1e-13, method="DOP853")
    return sol.y[:, -1].reshape(x.shape)


def _divergent_1d_error(n, opts, T=0.3, a=0.5):
    """psi_t + (u psi)_x = 0 with the steady divergent u = 1 + a sin(2 pi x): u psi is constant
    along characteristics, so the exact cell means follow from the characteristics' feet."""
    u = lambda x: 1.0 + a * np.sin(2 * np.pi * x)
    p0 = lambda x: 2.0 + np.sin(2 * np.pi * x)
    dx = 1.0 / n
    steps = int(np.ceil(T / (0.5 * dx / (1.0 + a))))
    dt = T / steps
    q, gw, psi = _gl_means(p0, n)
    X0 = _foot(u, q, T)
    ref = ((u(X0) * p0(X0) / u(q)) * gw[None, :]).sum(1) / 2.0
    gc = [u((np.arange(n) + 1) * dx) * dt / dx]
    out = oracle.step(psi, gc, n_iters=2, opts=opts, n_steps=steps)
    return np.sqrt(np.mean((out - ref) ** 2))


def test_dfl_restores_second_order_in_divergent_1d_flow():
    """Sect. 3.1.3: in a divergent flow the basic pseudo-velocity leaves the donor-cell scheme's
    -dt/2 (V/G) psi div(V) error uncancelled (first order); the divergent-flow term removes it
    (second order).  A dropped term, a wrong sign or factor leaves first order."""
    ns = (64, 128, 256, 512)
    for opts, lo, hi in ((0, 0.9, 1.2), (oracle.DFL, 1.9, 2.1)):
        errs = [_divergent_1d_error(n, opts) for n in ns]
        order = math.log2(errs[-2] / errs[-1])
        assert lo <= order <= hi, (opts, errs)


def test_dfl_restores_second_order_in_divergent_2d_flow():
    """The multi-D form: the divergence at a face is the mean of its two cells' divergences over
    every dimension.  Separable steady flow u(x), v(y) (both divergent): u v psi is carried
    unchanged along characteristics, so the exact cell means follow from the feet."""
    a, b, T = 0.5, 0.4, 0.3
    u = lambda x: 1.0 + a * np.sin(2 * np.pi * x)
    v = lambda y: 0.7 * (1.0 + b * np.cos(2 * np.pi * y))
    p0 = lambda x, y: 2.0 + np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    gx, gw = np.polynomial.legendre.leggauss(4)

    def err(n, opts):
        dx = 1.0 / n
        steps = int(np.ceil(T / (0.25 * dx / 1.5)))
        dt = T / steps
        q = ((np.arange(n) + 0.5) * dx)[:, None] + 0.5 * dx * gx[None, :]
        Y, X = q[:, None, :, None], q[None, :, None, :]  # arrays [y, x]
        W = gw[:, None] * gw[None, :] / 4.0
        psi = (p0(X, Y) * W).sum((2, 3))
        X0, Y0 = _foot(u, q, T), _foot(v, q, T)
        ex = p0(X0[None, :, None, :], Y0[:, None, :, None]) * u(X0)[None, :, None, :] * v(Y0)[:, None, :, None] \
            / (u(X) * v(Y))
        ref = (ex * W).sum((2, 3))
        f = (np.arange(n) + 1) * dx
        g0 = np.broadcast_to((v(f) * dt / dx)[:, None], (n, n)).copy()
        g1 = np.broadcast_to((u(f) * dt / dx)[None, :], (n, n)).copy()
        out = oracle.step(psi, [g0, g1], n_iters=2, opts=opts, n_steps=steps)
        return np.sqrt(np.mean((out - ref) ** 2))

    errs = [err(n, oracle.DFL) for n in (32, 64, 128)]
    assert math.log2(errs[-2] / errs[-1]) >= 1.85, errs
    base = [err(n, 0) for n in (64, 128)]
    assert math.log2(base[0] / base[1]) <= 1.4, base


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
def test_dfl_term_vanishes_for_nondivergent_flow_and_conserves(shape):
    """For a (discretely) nondivergent advector the divergent-flow term is zero in the first
    corrective pass (two passes: the basic result to rounding); on a divergent advector the
    step stays in flux form and conserves the sum; it excludes the infinite gauge."""
    rng = np.random.default_rng(31 + len(shape))
    gc = nondivergent(shape, rng, 0.4)
    psi = 1.0 + rng.uniform(size=shape)
    a = oracle.step(psi, gc, n_iters=2, opts=oracle.DFL, n_steps=3)
    b = oracle.step(psi, gc, n_iters=2, opts=0, n_steps=3)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)
    div = [0.3 * rng.uniform(size=shape) for _ in shape]
    out = oracle.step(psi, div, n_iters=3, opts=oracle.DFL | oracle.FCT, n_steps=4)
    assert abs(out.sum() - psi.sum()) <= 1e-13 * psi.sum() * 4
    with pytest.raises(ValueError):
        oracle.step(psi, gc, n_iters=2, opts=oracle.DFL | oracle.IGA)


# ----------------------------------------------------------------------------- Kahan

def _exact_donor(psi, gc):
    """One donor-cell step (Eqs. 4-5, G = 1) in exact rational arithmetic."""
    shape, nd = psi.shape, psi.ndim
    p = np.empty(shape, dtype=object)
    for idx in np.ndindex(shape):
        p[idx] = Fraction(float(psi[idx]))
    new = p.copy()
    for d in range(nd):
        right = np.roll(p, -1, axis=d)
        F = np.empty(shape, dtype=object)
        for idx in np.ndindex(shape):
            v = Fraction(float(gc[d][idx]))
            F[idx] = v * (p[idx] if v > 0 else right[idx])
        new = new - F + np.roll(F, 1, axis=d)
    return new


@pytest.mark.parametrize("shape,ratio", [((64,), 0.85), ((12, 11), 0.6), ((6, 5, 7), 0.5)],
                         ids=["1d", "2d", "3d"])
def test_kahan_summation_is_closer_to_exact_than_plain(shape, ratio):
    """Sect. 3.1.1, the Kahan option: the donor pass adds its 2 x nd flux terms to psi with
    compensated summation.  On psi = 1e8 + O(1) with power-of-two Courant numbers every flux
    product is exact in FP64, so the only roundings are those of the sum; against the exact
    rational result the compensated sum must be clearly closer than the plain one (RMS error
    below `ratio` times the plain sum's, and within 1.5 units in the last place everywhere).
    Dropping the compensation makes the two sums identical and fails this."""
    rng = np.random.default_rng(11)
    psi = 1e8 + rng.uniform(-1.0, 1.0, size=shape)
    gc = [rng.choice([-0.25, -0.125, 0.125, 0.25], size=shape) for _ in shape]
    exact = _exact_donor(psi, gc)
    ulp = np.spacing(1e8)
    errs = {}
    for name, opts in (("plain", 0), ("kahan", oracle.KAHAN)):
        out = oracle.step(psi, gc, n_iters=1, opts=opts)
        errs[name] = np.array([float(Fraction(float(out[i])) - exact[i]) for i in np.ndindex(shape)]) / ulp
    rms = {k: float(np.sqrt((e ** 2).mean())) for k, e in errs.items()}
    assert rms["kahan"] < ratio * rms["plain"], rms
    assert np.abs(errs["kahan"]).max() <= 1.5


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
@pytest.mark.parametrize("name", ["fct", "tot3_fct"])
def test_abs_tangent_linear_and_adjoint(shape, name):
    """abs on a variable-sign field (no cell near zero, where |psi| has its kink): the
    tangent-linear step agrees with central differences of the forward step, and the adjoint is
    its transpose (<TL dx, y> = <dx, AD y>)."""
    n_iters, opts = ABS_SETS[name]
    opts |= oracle.ABS
    rng = np.random.default_rng(13)
    f = wl.low_modes(rng, shape, 6)
    psi = 0.5 * f / np.abs(f).max()
    psi = np.where(np.abs(psi) < 0.05, psi + 0.1, psi)  # keep every cell away from the kink
    gc = nondivergent(shape, rng, 0.3)
    dpsi = rng.normal(size=shape)
    dgc = [rng.normal(size=shape) * 0.1 for _ in shape]
    tl = oracle.tl_step(psi, gc, dpsi, dgc, n_iters=n_iters, opts=opts)
    eps = 1e-6
    fp = oracle.step(psi + eps * dpsi, [v + eps * dv for v, dv in zip(gc, dgc)], n_iters=n_iters, opts=opts)
    fm = oracle.step(psi - eps * dpsi, [v - eps * dv for v, dv in zip(gc, dgc)], n_iters=n_iters, opts=opts)
    assert np.linalg.norm((fp - fm) / (2 * eps) - tl) <= 1e-8 * np.linalg.norm(tl)
    y = rng.normal(size=shape)
    pb, gcb = oracle.adj_step(psi, gc, y, n_iters=n_iters, opts=opts)
    lhs = float(np.sum(tl * y))
    rhs = float(np.sum(dpsi * pb) + sum(np.sum(a * b) for a, b in zip(dgc, gcb)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
@pytest.mark.parametrize("name", ["dfl", "dfl_it3_fct"])
def test_dfl_tangent_linear_and_adjoint(shape, name):
    """The divergent-flow term on a divergent advector (smooth seeded fields, |C| <= 0.3): the
    tangent-linear step agrees with central differences of the forward step, and the adjoint is
    its transpose (<TL dx, y> = <dx, AD y>)."""
    n_iters, opts = OPTION_SETS[name]
    rng = np.random.default_rng(17)
    f = wl.low_modes(rng, shape, 6)
    psi = 2.0 + 0.5 * f / np.abs(f).max()
    gc = []
    for _ in shape:
        v = wl.low_modes(rng, shape, 4)
        gc.append(0.3 * v / np.abs(v).max())
    dpsi = rng.normal(size=shape)
    dgc = [rng.normal(size=shape) * 0.1 for _ in shape]
    tl = oracle.tl_step(psi, gc, dpsi, dgc, n_iters=n_iters, opts=opts)
    eps = 1e-6
    fp = oracle.step(psi + eps * dpsi, [v + eps * dv for v, dv in zip(gc, dgc)], n_iters=n_iters, opts=opts)
    fm = oracle.step(psi - eps * dpsi, [v - eps * dv for v, dv in zip(gc, dgc)], n_iters=n_iters, opts=opts)
    assert np.linalg.norm((fp - fm) / (2 * eps) - tl) <= 1e-8 * np.linalg.norm(tl)
    y = rng.normal(size=shape)
    pb, gcb = oracle.adj_step(psi, gc, y, n_iters=n_iters, opts=opts)
    lhs = float(np.sum(tl * y))
    rhs = float(np.sum(dpsi * pb) + sum(np.sum(a * b) for a, b in zip(dgc, gcb)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{len(s)}d")
@pytest.mark.parametrize("rhs", ["euler_a", "euler_b"])
def test_adjoint_dot_product_with_sources(shape, rhs):
    """Euler sources (Sect. 4.1) with a given R: the tangent-linear step agrees with central
    differences of the forward step, and the adjoint is its transpose."""
    n_iters, opts = OPTION_SETS["fct"]
    rng = np.random.default_rng(19)
    f = wl.low_modes(rng, shape, 6)
    psi = 2.0 + 0.5 * f / np.abs(f).max()
    gc = nondivergent(shape, rng, 0.3)
    R, dt = 0.5 * rng.normal(size=shape), 0.3
    dpsi = rng.normal(size=shape)
    dgc = [rng.normal(size=shape) * 0.1 for _ in shape]
    kw = dict(r=R, dt=dt, n_iters=n_iters, opts=opts, rhs=rhs)
    tl = oracle.tl_step(psi, gc, dpsi, dgc, **kw)
    eps = 1e-6
    fp = oracle.step(psi + eps * dpsi, [v + eps * dv for v, dv in zip(gc, dgc)], **kw)
    fm = oracle.step(psi - eps * dpsi, [v - eps * dv for v, dv in zip(gc, dgc)], **kw)
    assert np.linalg.norm((fp - fm) / (2 * eps) - tl) <= 1e-8 * np.linalg.norm(tl)
    y = rng.normal(size=shape)
    pb, gcb = oracle.adj_step(psi, gc, y, **kw)
    lhs = float(np.sum(tl * y))
    rhs_ = float(np.sum(dpsi * pb) + sum(np.sum(a * b) for a, b in zip(dgc, gcb)))
    assert abs(lhs - rhs_) <= 1e-12 * max(abs(lhs), 1.0)
