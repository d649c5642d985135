"""The float64 kernels' division num / |det J| (fem_cell.cuh's quot_abs: a float32 seed of the
reciprocal of the mantissa refined by two float64 Newton-Raphson steps, the exponent put back,
one product) against CUDA's IEEE division num / fabs(den) on the device: within 2 units in
the last place of the correctly rounded quotient over random mantissas and exponents across
[2^-1000, 2^1001) and random signs, and bit for bit equal to the IEEE division on the edges
it hands to it (|den| outside that range, zero, subnormal, infinite, NaN)."""

import numpy as np
import pytest
import torch

import paper_1607_04245_gb300 as fem

pytestmark = pytest.mark.gpu


def _ulps(a, b):
    """|a - b| in units in the last place of b (float64)."""
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_newton_quotient_within_two_ulps():
    rng = np.random.default_rng(1234)
    n = 1 << 20
    den = rng.uniform(1.0, 2.0, n) * np.exp2(rng.integers(-1000, 1001, n).astype(np.float64))
    den *= np.where(rng.random(n) < 0.5, -1.0, 1.0)
    num = rng.uniform(-2.0, 2.0, n) * np.exp2(rng.integers(-20, 21, n).astype(np.float64))
    # mantissas at the ends of [1, 2): the seed's worst cases
    den[:64] = np.ldexp(1.0 + np.arange(64) * 2.0 ** -52, 3)
    den[64:128] = np.ldexp(2.0 - (np.arange(64) + 1) * 2.0 ** -52, -7)
    d_num = torch.from_numpy(num).cuda()
    d_den = torch.from_numpy(den).cuda()
    q_lib, q_ieee = fem.fem_selftest_quotient(d_num, d_den)
    q_lib, q_ieee = q_lib.cpu().numpy(), q_ieee.cpu().numpy()
    assert np.array_equal(q_ieee, num / np.abs(den))  # CUDA's division is the correctly rounded one
    u = _ulps(q_lib, q_ieee)
    print(f"Newton quotient: max {u.max():.2f} ulp, exact in {np.mean(u == 0) * 100:.1f} % of cases")
    assert u.max() <= 2.0


def test_edges_take_the_ieee_division():
    tiny, huge = np.ldexp(1.0, -1001), np.ldexp(1.0, 1001)
    den = np.array([0.0, -0.0, 5e-324, -2.2e-308, 1e-310, tiny, -tiny, np.ldexp(1.5, -1010), huge, -huge,
                    np.ldexp(1.25, 1015), np.inf, -np.inf, np.nan, 1.7976931348623157e308])
    num = np.full_like(den, 3.0)
    num[3] = -1.0
    q_lib, q_ieee = fem.fem_selftest_quotient(torch.from_numpy(num).cuda(), torch.from_numpy(den).cuda())
    q_lib, q_ieee = q_lib.cpu().numpy(), q_ieee.cpu().numpy()
    assert np.array_equal(q_lib.view(np.uint64), q_ieee.view(np.uint64))  # bitwise, NaN included


def test_range_ends_inside_the_newton_path():
    """|den| at the first and last exponents the Newton path takes (2^-1000 and just
    below 2^1001): still within 2 ulps."""
    den = np.array([np.ldexp(1.0, -1000), np.ldexp(1.999999, -1000), np.ldexp(1.0, 1000),
                    np.ldexp(1.9999999999, 1000), -np.ldexp(1.3, 999)])
    num = np.array([1.0, -3.5, 7.25, 1e-3, 2.0])
    q_lib, q_ieee = fem.fem_selftest_quotient(torch.from_numpy(num).cuda(), torch.from_numpy(den).cuda())
    assert _ulps(q_lib.cpu().numpy(), q_ieee.cpu().numpy()).max() <= 2.0
