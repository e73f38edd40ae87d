"""The FP32 tolerance of the GPU tests (tests/helpers.py) is tight enough to
fail an FP32 error twenty times larger than the one measured, in every
workload family, and loose enough to pass the measured errors themselves.
No GPU: the comparison helper is exercised on recorded values."""
import pytest

from helpers import FP32_KAPPA, FP32_MEASURED, U32, assert_fp32, fp32_bounds, fp32_within


@pytest.mark.parametrize("family,steps,e,p", FP32_MEASURED)
def test_measured_errors_pass(family, steps, e, p):
    assert_fp32(family, steps, e, p)


@pytest.mark.parametrize("family,steps,e,p", FP32_MEASURED)
def test_errors_twenty_times_larger_fail(family, steps, e, p):
    assert not fp32_within(family, steps, 20 * e, p)
    assert not fp32_within(family, steps, e, 20 * p)
    with pytest.raises(AssertionError):
        assert_fp32(family, steps, 20 * e, p)


@pytest.mark.parametrize("family", sorted(FP32_KAPPA))
def test_bounds_grow_linearly_and_stay_within_ten_times_the_measurement(family):
    b1, b2 = fp32_bounds(family, 1000), fp32_bounds(family, 2000)
    assert b2[0] == pytest.approx(2 * b1[0]) and b2[1] == pytest.approx(2 * b1[1])
    rows = [r for r in FP32_MEASURED if r[0] == family]
    assert rows, family
    kE, kP = FP32_KAPPA[family]
    for _, n, e, p in rows:
        assert 1.0 < kE * U32 * n / e <= 10.0, (family, n, e)
        assert 1.0 < kP * U32 * n / p <= 10.0, (family, n, p)
