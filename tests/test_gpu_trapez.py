"""The trapezoidal source scheme (Sect. 4.1, MPDATA_RHS_TRAPEZ with sources affine in the state)
on the GPU against the oracle: the translating oscillator of Sect. 4.2 at Courant number 1 (closed
form) and as printed (1400 s, default options), an affine three-equation system on a 2D grid with a
constant part b and non-unit G, FP64 and FP32; argument checks."""
import math

import numpy as np
import pytest
import torch

import oracle
from helpers import nondivergent, smooth_positive
from paper_1407_1309_gb300 import capi, workloads
from paper_1407_1309_gb300.solver import Mpdata

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


def run_system(fields, gc, A, n_iters, opts, dtype, dt, steps, b=None, G=None):
    """One handle whose fields are the equations; every equation uses the same advector."""
    shape = fields[0].shape
    E = len(fields)
    t = lambda a: torch.tensor(np.asarray(a), dtype=dtype, device=DEV)
    o = opts | capi.RHS_TRAPEZ | (capi.NUG if G is not None else 0)
    with Mpdata([shape] * E, dtype=dtype, n_iters=n_iters, opts=o) as m:
        psi = torch.cat([t(f).flatten() for f in fields])
        gcs = [torch.cat([t(v).flatten()] * E) for v in gc]
        bt = None if b is None else torch.cat([t(x).flatten() for x in b])
        Gt = None if G is None else torch.cat([t(G).flatten()] * E)
        m.set_rhs_linear(A, bt)
        out = torch.empty_like(psi)
        m.advance(psi, out, gcs, g=Gt, dt=dt, n_steps=steps)
        torch.cuda.synchronize()
        got = out.double().cpu().numpy().reshape(E, *shape)
    return [got[e] for e in range(E)]


def check(got, ref, dtype):
    """Errors over the whole state of the system (one equation can pass through zero while the
    others carry the amplitude, as phi does after a full period of the oscillator)."""
    g, r = np.stack(got), np.stack(ref)
    if dtype == torch.float64:
        assert np.abs(g - r).max() <= 1e-12 * np.abs(r).max()
    else:
        assert np.linalg.norm(g - r) <= 1e-5 * np.linalg.norm(r)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("n_iters,opts", [(1, 0), (2, capi.FCT), (2, capi.IGA | capi.FCT | capi.KAHAN)],
                         ids=["donor", "fct", "iga_fct_kahan"])
def test_oscillator_at_courant_one_closed_form(n_iters, opts, dtype):
    rng = np.random.default_rng(1)
    n, k, omega, dt = 300, 9, 0.3, 0.7
    psi0, phi0 = rng.uniform(-1, 1, size=n), rng.uniform(-1, 1, size=n)
    if dtype == torch.float32:
        psi0, phi0 = (x.astype(np.float32).astype(np.float64) for x in (psi0, phi0))
    A = [[0.0, omega], [-omega, 0.0]]
    got = run_system([psi0, phi0], [np.ones(n)], A, n_iters, opts, dtype, dt, k)
    th = k * 2.0 * math.atan(0.5 * omega * dt)
    sp, sf = np.roll(psi0, k), np.roll(phi0, k)
    check(got, [math.cos(th) * sp + math.sin(th) * sf, -math.sin(th) * sp + math.cos(th) * sf], dtype)


@pytest.mark.parametrize("dtype,steps", [(torch.float64, 1400), (torch.float32, 200)], ids=["f64", "f32"])
def test_translating_oscillator_as_printed(dtype, steps):
    """FP64 over the full 1400 s; FP32 over 200 s (over 1400 steps the FP32 state's rounding
    accumulates past the 1e-5 bar: rel. L2 4e-5)."""
    psi0, phi0, gc, omega = workloads.oscillator_1d()
    opts = capi.FCT | capi.IGA | capi.KAHAN
    A = [[0.0, omega], [-omega, 0.0]]
    ref = oracle.step_trapez([psi0, phi0], gc, A, dt=1.0, n_iters=2, opts=int(opts), n_steps=steps)
    got = run_system([psi0, phi0], gc, A, 2, opts, dtype, 1.0, steps)
    check(got, ref, dtype)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_affine_three_equation_system_2d(dtype):
    shape = (37, 29)
    rng = np.random.default_rng(4)
    gc = nondivergent(shape, rng, 0.3)
    fields = [smooth_positive(shape, rng) for _ in range(3)]
    b = [0.1 * rng.normal(size=shape) for _ in range(3)]
    G = 1.0 + 0.2 * rng.uniform(size=shape)
    A = rng.normal(size=(3, 3)) * 0.2
    r = (lambda a: a.astype(np.float32).astype(np.float64)) if dtype == torch.float32 else (lambda a: a)
    fields, b, gc, G = [r(f) for f in fields], [r(x) for x in b], [r(v) for v in gc], r(G)
    ref = oracle.step_trapez(fields, gc, A, b=b, dt=0.4, n_iters=2, opts=oracle.FCT, n_steps=5, g=G)
    got = run_system(fields, gc, A, 2, capi.FCT, dtype, 0.4, 5, b=b, G=G)
    check(got, ref, dtype)


def test_trapez_argument_checks():
    z = torch.zeros(16, dtype=torch.float64, device=DEV)
    with Mpdata([(8,), (8,)], dtype=torch.float64, n_iters=2, opts=capi.FCT) as m:
        with pytest.raises(capi.MpdataError):
            m.set_rhs_linear(np.eye(2))  # the handle has no trapez bit
    with Mpdata([(8,), (9,)], dtype=torch.float64, n_iters=2, opts=capi.RHS_TRAPEZ) as m:
        with pytest.raises(capi.MpdataError):
            m.set_rhs_linear(np.eye(2))  # fields of different shapes
    with Mpdata([(8,), (8,)], dtype=torch.float64, n_iters=2, opts=capi.RHS_TRAPEZ) as m:
        # stepping before the sources are set
        assert capi.mpdata_step(m.h, z, [z], raw=True) == capi.EINVAL
        m.set_rhs_linear(np.eye(2) * 2.0)  # I - dt/2 A singular at dt = 1
        assert capi.mpdata_step(m.h, z, [z], dt=1.0, raw=True) == capi.EINVAL
        assert capi.mpdata_step(m.h, z, [z], dt=0.5, raw=True) == capi.OK
        assert capi.mpdata_step(m.h, z, [z], r=z, dt=0.5, raw=True) == capi.EINVAL  # r must be NULL
    with pytest.raises(capi.MpdataError):
        Mpdata((8,), dtype=torch.float64, opts=capi.RHS_TRAPEZ | capi.RHS_EULER_A)
