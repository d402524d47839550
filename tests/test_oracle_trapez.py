"""Pins of the oracle's trapezoidal source scheme (Sect. 4.1, Eq. trapez) with sources affine in
the state, on the translating oscillator of Sect. 4.2 (R_psi = omega phi, R_phi = -omega psi).

At Courant number 1 every corrective pseudo-velocity vanishes and the advection is an exact shift
by one cell, so the discrete solution is known in closed form: per step the state is shifted and
rotated by the Cayley transform of dt A, a rotation by theta = 2 atan(omega dt / 2).  That fixes the
result to rounding, the conservation of psi^2 + phi^2, and the scheme's second order in time
(against the first order of the Euler scheme)."""
import math

import numpy as np
import pytest

import oracle
from paper_1407_1309_gb300 import workloads as wl

OPTION_SETS = {"donor": (1, 0), "basic": (2, 0), "fct": (2, oracle.FCT),
               "iga_fct_kahan": (2, oracle.IGA | oracle.FCT | oracle.KAHAN), "tot3_fct": (3, oracle.TOT | oracle.FCT)}


def osc(omega):
    return np.array([[0.0, omega], [-omega, 0.0]])


@pytest.mark.parametrize("name", sorted(OPTION_SETS))
def test_oscillator_at_courant_one_is_a_shifted_rotation(name):
    n_iters, opts = OPTION_SETS[name]
    rng = np.random.default_rng(1)
    n, k, omega, dt = 29, 6, 0.3, 0.7
    psi0, phi0 = rng.uniform(-1, 1, size=n), rng.uniform(-1, 1, size=n)
    psi, phi = oracle.step_trapez([psi0, phi0], [np.ones(n)], osc(omega), dt=dt, n_iters=n_iters, opts=opts,
                                  n_steps=k)
    th = k * 2.0 * math.atan(0.5 * omega * dt)
    sp, sf = np.roll(psi0, k), np.roll(phi0, k)
    np.testing.assert_allclose(psi, math.cos(th) * sp + math.sin(th) * sf, rtol=0, atol=1e-13)
    np.testing.assert_allclose(phi, -math.sin(th) * sp + math.cos(th) * sf, rtol=0, atol=1e-13)
    e0, e1 = (psi0 ** 2 + phi0 ** 2).sum(), (psi ** 2 + phi ** 2).sum()
    assert abs(e1 - e0) <= 1e-13 * e0


def _ode_error(k, scheme, T=4.0, omega=1.3, n=16):
    """Error after k steps over time T at Courant number 1 against the exact oscillation
    (the shift is exact, so only the time integration of the sources errs)."""
    rng = np.random.default_rng(2)
    psi0, phi0 = rng.uniform(-1, 1, size=n), np.zeros(n)
    dt = T / k
    A = osc(omega)
    if scheme == "trapez":
        psi, phi = oracle.step_trapez([psi0, phi0], [np.ones(n)], A, dt=dt, n_iters=2, n_steps=k)
    else:  # Euler, sources added before the advection (euler_b)
        psi, phi = psi0, phi0
        for _ in range(k):
            R = [omega * phi, -omega * psi]
            psi, phi = (oracle.step(x, [np.ones(n)], r=r, dt=dt, n_iters=2, rhs="euler_b") for x, r in zip((psi, phi), R))
    sp = np.roll(psi0, k)
    return np.abs(psi - math.cos(omega * T) * sp).max() + np.abs(phi + math.sin(omega * T) * sp).max()


def test_trapez_is_second_order_in_time_and_euler_first():
    """Sect. 4.1: trapez is second-order accurate (Crank-Nicolson), the Euler schemes first."""
    tr = [_ode_error(k, "trapez") for k in (16, 32, 64)]
    eu = [_ode_error(k, "euler") for k in (16, 32, 64)]
    for a, b in zip(tr, tr[1:]):
        assert 3.6 < a / b < 4.4, tr
    for a, b in zip(eu, eu[1:]):
        assert 1.7 < a / b < 2.3, eu


def test_translating_oscillator_as_in_sect_4_2():
    """Sect. 4.2: the cosine bell on (50, 150) with phi = 0, 1400 s at C = 0.5 (dt = 1 s, 1 m cells)
    with the library's default options (two passes, FCT, infinite gauge, compensated summation);
    omega = 2 pi / 1400 s here (the paper does not print it), so the run is one full period.
    psi and phi stay in phase (phi returns to ~0, psi's peak sits where the flow carried it) and
    the amplitude is kept (psi^2 + phi^2 does not grow; the Euler scheme's grows)."""
    psi0, phi0, gc, omega = wl.oscillator_1d()
    opts = oracle.FCT | oracle.IGA | oracle.KAHAN
    psi, phi = oracle.step_trapez([psi0, phi0], gc, osc(omega), dt=1.0, n_iters=2, opts=opts, n_steps=1400)
    assert np.abs(phi).max() <= 2e-3
    assert abs(int(np.argmax(psi)) - (100 + 700)) <= 2
    e0 = (psi0 ** 2).sum()
    e1 = (psi ** 2 + phi ** 2).sum()
    assert 0.9 * e0 < e1 <= e0 * (1 + 1e-12)
    # the Euler scheme (sources before the advection) gains amplitude every step
    p, f = psi0, phi0
    for _ in range(1400):
        R = [omega * f, -omega * p]
        p, f = (oracle.step(x, gc, r=r, dt=1.0, n_iters=2, opts=opts, rhs="euler_b") for x, r in zip((p, f), R))
    assert (p ** 2 + f ** 2).sum() > 1.005 * e1
