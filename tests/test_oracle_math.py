"""Pins of the oracle's FP64 elementary functions against libm error bounds.

The oracle's ln/exp/ln k! are written out step by step (atanh series, Taylor
polynomial, Stirling series) so that two independent implementations can agree
bit for bit; these tests pin them to the mathematics through libm within
stated error bounds, never by retyping the formulas.
"""
import math

import numpy as np
import pytest


def ulp_diff(a: float, b: float) -> float:
    if a == b:
        return 0.0
    return abs(a - b) / math.ulp(max(abs(a), abs(b)))


def test_exact_points(orc):
    assert orc.log(1.0) == 0.0
    assert orc.exp(0.0) == 1.0
    assert orc.log(2.0) == math.log(2.0)
    assert orc.log(0.5) == -math.log(2.0)
    assert orc.lnfact(0) == 0.0 and orc.lnfact(1) == 0.0
    assert orc.lnfact_diff(123456789.0, 0.0) == 0.0


def test_log_within_3ulp_of_libm(orc):
    rng = np.random.default_rng(11)
    xs = np.concatenate([
        rng.uniform(0.0, 1.0, 40000),                      # the uniforms fed to geometric skips
        np.exp(rng.uniform(-700, 700, 40000)),             # the whole exponent range
        1.0 + rng.uniform(-1e-6, 1e-6, 5000),              # close to 1
        np.arange(2, 5000, dtype=np.float64),              # integers (ln k!)
        [2.0 ** -53, 2.0 ** -1074, 1e-310, 1.7e308],       # extremes incl. subnormals
    ])
    worst = 0.0
    for x in xs:
        if x <= 0 or x == 1.0:
            continue
        worst = max(worst, ulp_diff(orc.log(float(x)), math.log(float(x))))
    # roundings of f+1, of the quotient, of the series and of the final sum
    assert worst <= 3.0, worst


def test_log1m_small_p_keeps_digits(orc):
    rng = np.random.default_rng(12)
    for p in np.concatenate([10.0 ** rng.uniform(-300, -0.7, 20000), rng.uniform(0.2, 0.999, 5000)]):
        a, b = orc.log1m(float(p)), math.log1p(-float(p))
        # p >= 1/4 goes through ln(1-p): the rounding of 1-p adds one ulp
        assert ulp_diff(a, b) <= (2.0 if p < 0.25 else 3.0), p


def test_exp_within_2ulp_of_libm(orc):
    rng = np.random.default_rng(13)
    worst = 0.0
    for x in np.concatenate([rng.uniform(-700, 700, 40000), rng.uniform(-30, 1, 20000),
                             rng.uniform(-1e-8, 1e-8, 2000)]):
        worst = max(worst, ulp_diff(orc.exp(float(x)), math.exp(float(x))))
    assert worst <= 2.0, worst
    assert orc.exp(-701.0) == 0.0 and math.isinf(orc.exp(701.0))


def test_lnfact_matches_lgamma(orc):
    ks = list(range(0, 300)) + [10 ** e for e in range(3, 16)] + [2 ** 44, 2 ** 52 + 2]
    rng = np.random.default_rng(14)
    ks += [int(x) for x in rng.integers(0, 1 << 50, 3000)]
    for k in ks:
        a, b = orc.lnfact(float(k)), math.lgamma(float(k) + 1.0)
        assert abs(a - b) <= 1e-13 * max(1.0, abs(b)), k


def test_lnfact_small_table_is_log_sum(orc):
    # ln k! = sum_{j<=k} ln j; math.fsum of libm logs is an independent route
    for k in range(0, 40):
        want = math.fsum(math.log(j) for j in range(2, k + 1))
        assert abs(orc.lnfact(k) - want) <= 4 * math.ulp(max(want, 1.0)), k


@pytest.mark.parametrize("a", [0, 5, 63, 64, 100, 1000, 12345, 2 ** 20, 2 ** 33 + 7, 2 ** 44, 2 ** 52])
def test_lnfact_diff_is_sum_of_logs(orc, a):
    """D(a, d) = ln (a+d)! - ln a! = sum_{i=1..d} ln(a+i) for d > 0 (negative d: minus
    the sum over the removed factors).  Pinned with libm logs summed exactly."""
    rng = np.random.default_rng(a % 997)
    ds = sorted({1, 2, 3, 7, 16, 100, 999} | {int(x) for x in rng.integers(1, 2000, 20)})
    for d in ds:
        for sign in (1, -1):
            dd = sign * d
            if a + dd < 0:
                continue
            if sign > 0:
                want = math.fsum(math.log(a + i) for i in range(1, d + 1))
            else:
                want = -math.fsum(math.log(a - d + i) for i in range(1, d + 1))
            got = orc.lnfact_diff(float(a), float(dd))
            # absolute error bound: a few ulp of the magnitude d*ln(a+d)
            tol = 64 * math.ulp(abs(want)) + 1e-12 * abs(dd)
            assert abs(got - want) <= tol, (a, dd, got, want)
