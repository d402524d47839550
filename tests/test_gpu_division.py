"""The kernels' FP64 division (Newton-Raphson reciprocal iteration from the approximate FP64
reciprocal, remainder-corrected quotient) against correctly rounded IEEE division: within one
unit in the last place for normal operands over a wide range; a zero, infinite or NaN divisor
gives NaN, and the kernels' uses map that to the same result as IEEE (checked through the
limiter factor min(1, x / 0))."""
import numpy as np
import pytest
import torch

from paper_1407_1309_gb300 import capi

pytestmark = pytest.mark.gpu


def run(n, d):
    dev = torch.device("cuda")
    tn = torch.tensor(n, dtype=torch.float64, device=dev)
    td = torch.tensor(d, dtype=torch.float64, device=dev)
    tq = torch.empty_like(tn)
    capi.mpdata_selftest_division(tn, td, tq)
    torch.cuda.synchronize()
    return tq.cpu().numpy()


def ulps(a, b):
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_within_one_ulp_on_wide_ranges():
    rng = np.random.default_rng(0)
    m = 1 << 20
    n = rng.uniform(-1, 1, m) * 10.0 ** rng.uniform(-30, 30, m)
    d = rng.uniform(-1, 1, m) * 10.0 ** rng.uniform(-35, 35, m)
    d[d == 0] = 1.0
    q = run(n, d)
    ref = n / d
    assert ulps(q, ref).max() <= 1.0
    assert np.mean(q == ref) > 0.95  # mostly correctly rounded


def test_mpdata_like_ratios():
    """psi-fractions and limiter ratios: differences over sums of O(1) values."""
    rng = np.random.default_rng(1)
    a, b = rng.uniform(0, 5, 1 << 18), rng.uniform(0, 5, 1 << 18)
    q = run(b - a, a + b)
    assert ulps(q, (b - a) / (a + b)).max() <= 1.0


def test_special_divisors_give_nan_and_extremes_stay_exact():
    n = np.array([1.0, 0.0, -2.0, 3.0, 1.0, 5.0, 7.0, 1e-300, 1e300])
    d = np.array([0.0, 0.0, 0.0, np.inf, np.nan, 1e-300, 1e300, 1e-40, 1e40])
    q = run(n, d)
    assert np.all(np.isnan(q[:5]))
    ref = n[5:] / d[5:]
    assert ulps(q[5:], ref).max() <= 1.0
    # the FCT factor min(1, x / s) with a zero flux sum is 1 for x > 0 (inf) and x = 0 (NaN) alike
    assert np.all(np.fmin(1.0, q[:2]) == 1.0)


def test_rejects_bad_arguments():
    assert capi.load().mpdata_selftest_division(None, None, None, -1, None) == capi.EINVAL
    assert capi.load().mpdata_selftest_division(None, None, None, 0, None) == capi.OK
