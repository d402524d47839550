"""The Kahan option (Sect. 3.1.1: compensated summation of the donor-cell update) on the GPU in
FP32, against the FP64 oracle.  psi = 1000 + O(1) makes the rounding of the sum the dominant FP32
error.  Where the kernels add the flux terms to psi one after another (the staged kernels, the
oracle's order) the compensated sum must be clearly closer to the oracle than the plain one; the
fused 2D kernels form the flux divergence first and add it to psi once, which is already about
as accurate, and there the compensated sum must not be worse."""
import numpy as np
import pytest
import torch

import oracle
from helpers import nondivergent
from paper_1407_1309_gb300 import capi
from paper_1407_1309_gb300.solver import Mpdata

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")
r32 = lambda a: a.astype(np.float32).astype(np.float64)


def err(psi, gc, n_iters, opts, ref):
    with Mpdata(psi.shape, dtype=torch.float32, n_iters=n_iters, opts=opts) as m:
        p = torch.tensor(psi, dtype=torch.float32, device=DEV)
        q = torch.empty_like(p)
        m.advance(p, q, [torch.tensor(v, dtype=torch.float32, device=DEV) for v in gc], n_steps=10)
        torch.cuda.synchronize()
        out = q.double().cpu().numpy()
    return np.linalg.norm(out - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("shape", [(4096,), (256, 200), (40, 36, 34)], ids=lambda s: f"{len(s)}d")
@pytest.mark.parametrize("case", ["donor_pow2", "fct"])
def test_kahan_fp32_closer_to_oracle_than_plain(shape, case):
    rng = np.random.default_rng(5)
    psi = r32(1e3 + rng.uniform(-1, 1, size=shape))
    if case == "donor_pow2":  # power-of-two Courant numbers: exact flux products
        gc = [rng.choice([-0.25, -0.125, 0.125, 0.25], size=shape) for _ in shape]
        n_iters, base = 1, 0
    else:
        gc = [r32(v) for v in nondivergent(shape, rng, 0.4)]
        n_iters, base = 2, capi.FCT
    ref = oracle.step(psi, gc, n_iters=n_iters, opts=base, n_steps=10)
    staged = {k: err(psi, gc, n_iters, base | k | capi.STAGED, ref) for k in (0, capi.KAHAN)}
    auto = {k: err(psi, gc, n_iters, base | k, ref) for k in (0, capi.KAHAN)}
    assert staged[capi.KAHAN] < 0.8 * staged[0], staged
    assert auto[capi.KAHAN] <= auto[0], auto
    assert max(staged[capi.KAHAN], auto[capi.KAHAN]) <= 1e-5
