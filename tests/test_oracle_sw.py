"""Pins of the oracle's prognosed-velocity shallow-water system (Sect. 5: the advector at n + 1/2
extrapolated linearly from the velocities q/h at n and n-1 and interpolated to the cell walls; the
momentum sources -h grad h by the trapezoidal scheme of Sect. 4.1, explicit in its second half
because h has no source).

What fixes the results: the drop spreading under gravity has self-similar solutions,
h = (1 - x^2/lambda^2)/lambda, u = x lambda_t/lambda in 1D with lambda'' = 2/lambda^2 (integrated
here by RK4), and h = 1/lambda^2 - (x^2 + y^2)/lambda^4 with lambda = (2 t^2 + 1)^(1/2) in 2D (the
paper's closed form, Sect. 5.4); the numerical solution must approach them as the grid and the
step are refined.  Besides: the depth is conserved exactly (flux form), the drop stays mirror
symmetric, and a lake at rest stays at rest."""
import math

import numpy as np
import pytest

import oracle

OPTS = {"abs_fct_dfl": oracle.ABS | oracle.FCT | oracle.DFL, "iga_fct": oracle.IGA | oracle.FCT}


def lambda_1d(t, n=3000):
    """lambda(t) of the 1D self-similar drop: lambda'' = 2 / lambda^2, lambda(0) = 1, lambda'(0) = 0."""
    y, v, h = 1.0, 0.0, t / n
    f = lambda y_, v_: (v_, 2.0 / y_ ** 2)
    for _ in range(n):
        k1 = f(y, v)
        k2 = f(y + 0.5 * h * k1[0], v + 0.5 * h * k1[1])
        k3 = f(y + 0.5 * h * k2[0], v + 0.5 * h * k2[1])
        k4 = f(y + h * k3[0], v + h * k3[1])
        y, v = y + h / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0]), v + h / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
    return y, v


def drop_1d(n, dx):
    x = -0.5 * n * dx + (np.arange(n) + 0.5) * dx
    return x, np.where(np.abs(x) <= 1.0, 1.0 - x ** 2, 0.0)


def run_1d(name, n, dx, dt, T=3.0):
    x, h0 = drop_1d(n, dx)
    h, qs, _ = oracle.step_shallow_water(h0, [np.zeros(n)], dt, dx, n_iters=2, opts=OPTS[name] | oracle.OPEN0,
                                         n_steps=int(round(T / dt)))
    return x, h0, h, qs[0]


@pytest.mark.parametrize("name,bound", [("abs_fct_dfl", 2e-2), ("iga_fct", 5e-3)])
def test_1d_drop_approaches_the_self_similar_solution(name, bound):
    """Sect. 5.3: the 1D drop (dx = 0.05, dt = 0.01, t = 3) against the self-similar solution; the
    error shrinks as dx and dt are halved (orders 1.3-1.7 measured)."""
    lam, lam_t = lambda_1d(3.0)
    errs = []
    for n, dx, dt in ((320, 0.05, 0.01), (640, 0.025, 0.005)):
        x, _, h, q = run_1d(name, n, dx, dt)
        ha = np.maximum((1.0 - x ** 2 / lam ** 2) / lam, 0.0)
        errs.append(np.linalg.norm(h - ha) / np.linalg.norm(ha))
        if n == 320:
            assert errs[0] <= bound, errs
            u = np.where(h > 1e-8, q / np.where(h > 1e-8, h, 1.0), 0.0)
            inside = np.abs(x) < 0.9 * lam
            assert np.abs(u - x * lam_t / lam)[inside].max() <= 1e-2 * lam_t
    assert errs[1] < errs[0] / 2.0, errs


def test_2d_drop_approaches_the_closed_form():
    """Sect. 5.4: the axisymmetric drop against h = 1/lambda^2 - r^2/lambda^4, lambda = (2t^2+1)^(1/2),
    at t = 1.5 on dx = 0.1 and 0.05 (dt = dx / 5), with |psi| in the psi-fractions, FCT and the
    divergent-flow term: close, and closer on the finer grid."""
    T = 1.5
    lam = math.sqrt(2 * T * T + 1)
    errs = []
    for n, dx in ((80, 0.1), (160, 0.05)):
        c = -0.5 * n * dx + (np.arange(n) + 0.5) * dx
        X, Y = np.meshgrid(c, c, indexing="ij")
        h0 = np.maximum(1.0 - X ** 2 - Y ** 2, 0.0)
        z = np.zeros_like(h0)
        h, qs, _ = oracle.step_shallow_water(h0, [z, z], dx / 5, dx, n_iters=2,
                                             opts=OPTS["abs_fct_dfl"] | oracle.OPEN0 | oracle.OPEN1,
                                             n_steps=int(round(T / (dx / 5))))
        ha = np.maximum(1 / lam ** 2 - (X ** 2 + Y ** 2) / lam ** 4, 0.0)
        errs.append(np.linalg.norm(h - ha) / np.linalg.norm(ha))
        assert abs(h.sum() - h0.sum()) <= 1e-12 * h0.sum()  # depth conserved
        np.testing.assert_allclose(h, h.T, rtol=0, atol=1e-13)  # axis swap symmetry
    assert errs[0] <= 5e-2 and errs[1] < errs[0] / 1.7, errs


@pytest.mark.parametrize("name", sorted(OPTS))
def test_depth_conserved_and_mirror_symmetric(name):
    """Flux form (Eq. 4): sum(h) is constant while the drop stays clear of the open edges; the
    system is invariant under x -> -x with q -> -q."""
    x, h0, h, q = run_1d(name, 320, 0.05, 0.01, T=1.0)
    assert abs(h.sum() - h0.sum()) <= 1e-13 * h0.sum()
    np.testing.assert_allclose(h, h[::-1], rtol=0, atol=1e-14)
    np.testing.assert_allclose(q, -q[::-1], rtol=0, atol=1e-14)


@pytest.mark.parametrize("name", sorted(OPTS))
def test_lake_at_rest(name):
    """A flat surface at rest has no pressure gradient and no velocity: nothing changes."""
    h0 = np.full((24, 20), 0.7)
    z = np.zeros_like(h0)
    h, qs, _ = oracle.step_shallow_water(h0, [z, z], 0.01, 0.05, n_iters=2, opts=OPTS[name], n_steps=20)
    np.testing.assert_array_equal(h, h0)
    assert all(np.all(q == 0.0) for q in qs)
