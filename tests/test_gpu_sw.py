"""The shallow-water system with prognosed velocity (Sect. 5, mpdata_sw_advance) on the GPU
against the oracle: the 1D drop of Sect. 5.3 (dx = 0.05, dt = 0.01, to t = 3) and the 2D drop of
Sect. 5.4, FP64 and FP32, with |psi| + FCT + the divergent-flow term and with the infinite gauge +
FCT; calls split and resumed; argument checks."""
import numpy as np
import pytest
import torch

import oracle
from paper_1407_1309_gb300 import capi
from paper_1407_1309_gb300.solver import Mpdata

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")
OPTS = {"abs_fct_dfl": capi.ABS | capi.FCT | capi.DFL, "iga_fct": capi.IGA | capi.FCT}


def drop(nd, n, dx):
    c = -0.5 * n * dx + (np.arange(n) + 0.5) * dx
    if nd == 1:
        return np.where(np.abs(c) <= 1.0, 1.0 - c ** 2, 0.0)
    X, Y = np.meshgrid(c, c, indexing="ij")
    return np.maximum(1.0 - X ** 2 - Y ** 2, 0.0)


def gpu(h0, opts, dtype, dt, dx, steps, splits=1):
    nd = h0.ndim
    open_bits = sum(capi.OPEN0 << d for d in range(nd))
    with Mpdata([h0.shape] * (nd + 1), dtype=dtype, n_iters=2, opts=opts | capi.SW | open_bits) as m:
        state = torch.cat([torch.tensor(h0, dtype=dtype, device=DEV).flatten()] +
                          [torch.zeros(h0.size, dtype=dtype, device=DEV) for _ in range(nd)])
        for k in range(splits):
            m.sw_advance(state, dt, dx, n_steps=steps // splits)
        torch.cuda.synchronize()
        out = state.double().cpu().numpy().reshape(nd + 1, *h0.shape)
    return out


def ref(h0, opts, dt, dx, steps):
    nd = h0.ndim
    open_bits = sum(oracle.OPEN0 << d for d in range(nd))
    h, qs, _ = oracle.step_shallow_water(h0, [np.zeros_like(h0)] * nd, dt, dx, n_iters=2, opts=int(opts) | open_bits,
                                         n_steps=steps)
    return np.stack([h] + qs)


def check(got, want, dtype):
    if dtype == torch.float64:
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    else:
        assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)


@pytest.mark.parametrize("dtype,steps", [(torch.float64, 300), (torch.float32, 100)], ids=["f64", "f32"])
@pytest.mark.parametrize("name", sorted(OPTS))
def test_1d_drop_matches_oracle(name, dtype, steps):
    h0 = drop(1, 320, 0.05)
    if dtype == torch.float32:
        h0 = h0.astype(np.float32).astype(np.float64)
    check(gpu(h0, OPTS[name], dtype, 0.01, 0.05, steps), ref(h0, OPTS[name], 0.01, 0.05, steps), dtype)


@pytest.mark.parametrize("dtype,steps", [(torch.float64, 75), (torch.float32, 40)], ids=["f64", "f32"])
def test_2d_drop_matches_oracle(dtype, steps):
    h0 = drop(2, 80, 0.1)
    if dtype == torch.float32:
        h0 = h0.astype(np.float32).astype(np.float64)
    opts = OPTS["abs_fct_dfl"]
    check(gpu(h0, opts, dtype, 0.02, 0.1, steps), ref(h0, opts, 0.02, 0.1, steps), dtype)


def test_split_calls_resume_the_run():
    """The handle keeps the last velocities: 4 calls of 15 steps equal one call of 60 bit for bit;
    after mpdata_sw_reset the run starts afresh."""
    h0 = drop(1, 160, 0.05)
    a = gpu(h0, OPTS["iga_fct"], torch.float64, 0.01, 0.05, 60, splits=1)
    b = gpu(h0, OPTS["iga_fct"], torch.float64, 0.01, 0.05, 60, splits=4)
    assert np.array_equal(a, b)
    with Mpdata([h0.shape] * 2, dtype=torch.float64, n_iters=2, opts=OPTS["iga_fct"] | capi.SW | capi.OPEN0) as m:
        s0 = torch.cat([torch.tensor(h0, device=DEV), torch.zeros(h0.size, dtype=torch.float64, device=DEV)])
        s1 = s0.clone()
        m.sw_advance(s1, 0.01, 0.05, n_steps=60)
        m.sw_reset()
        s2 = s0.clone()
        m.sw_advance(s2, 0.01, 0.05, n_steps=60)
        torch.cuda.synchronize()
        assert torch.equal(s1, s2)


def test_sw_argument_checks():
    z = torch.zeros(16, dtype=torch.float64, device=DEV)
    with Mpdata([(8,), (8,)], dtype=torch.float64, n_iters=2, opts=capi.FCT) as m:  # no SW bit
        assert capi.mpdata_sw_advance(m.h, z, 0.01, 0.05, raw=True) == capi.EINVAL
    with Mpdata([(8,), (8,)], dtype=torch.float64, n_iters=2, opts=capi.FCT | capi.SW) as m:
        assert capi.mpdata_sw_advance(m.h, z, 0.0, 0.05, raw=True) == capi.EINVAL
        assert capi.mpdata_sw_advance(m.h, z, 0.01, -1.0, raw=True) == capi.EINVAL
        assert capi.mpdata_sw_advance(m.h, z, 0.01, 0.05, raw=True) == capi.OK
