"""The FP64 step kernel's integer-pipe helpers against plain FP64 arithmetic on the host:
exact power-of-two scaling (bit-identical to x * k, signed zeros, infinities and NaNs
included), the reciprocal of rho (within two ulps of 1/x for 2^-126 <= |x| < 2^126,
non-finite where the diagnostics must see a non-finite node) and the FP32 truncation
that seeds it."""
import numpy as np
import pytest

from paper_2602_21242_gb300 import capi

pytestmark = pytest.mark.gpu


def normal_values(seed, n=20000, lo=-1000, hi=1000):
    rng = np.random.default_rng(seed)
    mant = rng.uniform(1.0, 2.0, n)
    exps = rng.integers(lo, hi, n)
    sign = rng.choice([-1.0, 1.0], n)
    return sign * np.ldexp(mant, exps)


@pytest.mark.parametrize("op,k", [(0, 0.5), (1, -0.5), (2, 0.25)])
def test_scaling_is_exact(op, k):
    special = np.array([0.0, -0.0, 1.0, -1.0, 0.1, -3.7e-5, 1.5e300, -2.2e-300, 1.5 * 2.0 ** -1020,
                        np.finfo(np.float64).max, np.inf, -np.inf])
    x = np.concatenate([special, normal_values(1 + op)])
    got = capi.lbm_selftest_fp64(op, x)
    want = x * k
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    nan = capi.lbm_selftest_fp64(op, np.array([np.nan, -np.nan]))
    assert np.all(np.isnan(nan))


def test_reciprocal_within_two_ulps():
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.uniform(0.5, 2.0, 20000),            # densities of the benchmarks
                        normal_values(8, lo=-120, hi=120),          # FP32's normal range
                        np.array([1.0, -1.0, 2.0 ** -126, 1.9999999 * 2.0 ** 125])])
    got = capi.lbm_selftest_fp64(3, x)
    want = 1.0 / x
    assert np.all(np.abs(got - want) <= 2.0 * np.spacing(np.abs(want)))


def test_reciprocal_of_bad_densities_is_not_finite():
    """rho = 0, non-finite rho and rho outside [2^-126, 2^126) (a blown-up state) give a
    non-finite 1/rho, so the node is counted by the diagnostics."""
    x = np.array([0.0, -0.0, np.nan, np.inf, -np.inf, 1e-40, -1e-300, 2.0 ** 127, -1e38, 1e40, 1e300])
    got = capi.lbm_selftest_fp64(3, x)
    assert not np.any(np.isfinite(got))


def test_fp32_truncation():
    x = np.concatenate([normal_values(9, lo=-120, hi=120), np.array([1.0, -1.0, 1.0 + 2.0 ** -30])])
    got = capi.lbm_selftest_fp64(4, x)
    assert np.all(got.astype(np.float32).astype(np.float64) == got)   # an FP32 value
    assert np.all(np.sign(got) == np.sign(x)) and np.all(np.abs(got) <= np.abs(x))
    ulp32 = np.spacing(np.abs(x).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(x) - np.abs(got) < ulp32)
    edge = capi.lbm_selftest_fp64(4, np.array([1e-40, -1e-40, 0.0, 1e40, -1e40, np.inf, np.nan]))
    np.testing.assert_array_equal(edge[:3], [0.0, -0.0, 0.0])
    assert np.signbit(edge[1])
    np.testing.assert_array_equal(edge[3:6], [np.inf, -np.inf, np.inf])
    assert np.isinf(edge[6])


def test_bad_arguments():
    with pytest.raises(capi.LBMError):
        capi.lbm_selftest_fp64(5, np.array([1.0]))
    assert capi.lbm_selftest_fp64(0, np.array([])).size == 0
