"""Fields whose tails fall below the smallest normal number of the precision (a narrow blob on
a zero background): every kernel family keeps them finite and matches the FP64 oracle.

The psi-fractions of Eq. 6 divide by sums of neighbouring psi values; where those sums are
subnormal the kernels' fast divisions have no reciprocal, and the guard counts them as zero
(the fluxes they would carry are below the smallest normal number)."""
import numpy as np
import pytest
import torch

import oracle
from helpers import nondivergent
from paper_1407_1309_gb300 import capi
from paper_1407_1309_gb300.solver import Mpdata

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")
FAMILIES = {"warp": (1, 0), "band": (2, 0), "warp2": (3, 0), "staged": (0, -1)}


def blob(n, sigma):
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    r2 = (x - n / 2) ** 2 + (y - n / 2) ** 2
    return np.exp(-r2 / (2 * sigma * sigma))


@pytest.mark.parametrize("family", sorted(FAMILIES))
@pytest.mark.parametrize("opts", [0, capi.FCT], ids=["basic", "fct"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_subnormal_tails_stay_finite_and_match_oracle(dtype, opts, family):
    n = 96
    psi = blob(n, 1.5)
    if dtype == torch.float32:
        psi = psi.astype(np.float32).astype(np.float64)
        tiny = np.finfo(np.float32).tiny
    else:
        tiny = np.finfo(np.float64).tiny
    assert ((psi > 0) & (psi < tiny)).any()  # subnormal values in the input already
    gc = nondivergent((n, n), np.random.default_rng(5), 0.4)
    if dtype == torch.float32:
        gc = [v.astype(np.float32).astype(np.float64) for v in gc]
    kernel, rows = FAMILIES[family]
    o = opts | (capi.STAGED if family == "staged" else 0)
    with Mpdata((n, n), dtype=dtype, n_iters=2, opts=o) as m:
        if family != "staged":
            m.tune(capi.TUNE_KERNEL, kernel)
        a = torch.tensor(psi, dtype=dtype, device=DEV)
        b = torch.empty_like(a)
        m.advance(a, b, [torch.tensor(v, dtype=dtype, device=DEV) for v in gc], n_steps=30)
        torch.cuda.synchronize()
        out = b.double().cpu().numpy()
    assert np.isfinite(out).all()
    ref = oracle.step(psi, gc, n_iters=2, opts=opts, n_steps=30)
    if dtype == torch.float64:
        assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()
    else:
        assert np.linalg.norm(out - ref) <= 1e-5 * np.linalg.norm(ref)
