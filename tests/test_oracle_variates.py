"""Pins of the oracle's variates (Sec. 2.2: hypergeometric sample counts of a
split universe; Sec. 4.3: binomial chunk counts) against closed-form pmfs.

Every branch of the samplers is reached: inversion for small means, the
ratio-of-uniforms rejection sampler, the binomial approximation used when the
universe exceeds 2^32 times the sample count (including the fair-bit count of
an exactly even split) and the symmetry reductions.  The pmfs are computed in
Python from math.lgamma / exact fractions, independently of the oracle's own
ln k! routine.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

P_MIN = 1e-5  # chi-square p-value below which a test fails


def hyper_logpmf(N, K, t, k):
    lg = math.lgamma
    return (lg(K + 1) - lg(k + 1) - lg(K - k + 1) + lg(N - K + 1) - lg(t - k + 1)
            - lg(N - K - t + k + 1) - lg(N + 1) + lg(t + 1) + lg(N - t + 1))


def binom_logpmf(n, p, k):
    lg = math.lgamma
    return lg(n + 1) - lg(k + 1) - lg(n - k + 1) + k * math.log(p) + (n - k) * math.log1p(-p)


def chi2_pvalue(samples, logpmf, lo, hi):
    """Chi-square goodness of fit over [lo, hi], tails pooled until expected >= 5."""
    samples = np.asarray(samples, dtype=np.int64)
    S = len(samples)
    ks = np.arange(lo, hi + 1)
    probs = np.array([math.exp(logpmf(int(k))) for k in ks])
    probs = probs / probs.sum()
    obs = np.array([np.count_nonzero(samples == k) for k in ks], dtype=np.float64)
    assert obs.sum() == S, "sample outside the support"
    exp_ = probs * S
    # pool bins left to right into groups with expected >= 5
    o_g, e_g, o_acc, e_acc = [], [], 0.0, 0.0
    for o, e in zip(obs, exp_):
        o_acc += o
        e_acc += e
        if e_acc >= 5:
            o_g.append(o_acc)
            e_g.append(e_acc)
            o_acc = e_acc = 0.0
    if e_acc > 0:
        o_g[-1] += o_acc
        e_g[-1] += e_acc
    o_g, e_g = np.array(o_g), np.array(e_g)
    chi2 = float(((o_g - e_g) ** 2 / e_g).sum())
    return float(stats.chi2.sf(chi2, len(o_g) - 1))


def draw_hyper(orc, N, K, t, S, seed=0xC0FFEE):
    return [orc.hypergeometric(N, K, t, seed, node, 9) for node in range(S)]


def draw_binom(orc, n, p, S, seed=0xBEEF):
    return [orc.binomial(n, p, seed, node, 9) for node in range(S)]


# (N, K, t, branch) -- branch names the code path the parameters select
HYPER_CASES = [
    (40, 7, 13, "inversion, tiny N"),
    (1000, 30, 100, "inversion"),
    (1000, 970, 100, "inversion via K symmetry"),
    (1000, 30, 900, "inversion via t symmetry"),
    (1000, 300, 400, "ratio of uniforms"),
    (1000, 700, 800, "ratio of uniforms, both symmetries"),
    (100000, 50000, 50000, "ratio of uniforms, even split"),
    (2 ** 40, int(0.3 * 2 ** 40), 4096, "ratio of uniforms, large N exact regime"),
    (2 ** 24, 2 ** 23, 2 ** 12, "exact regime, even split (config-1 tile shape)"),
]


@pytest.mark.parametrize("N,K,t,branch", HYPER_CASES)
def test_hypergeometric_chi_square(orc, N, K, t, branch):
    S = 30000
    xs = draw_hyper(orc, N, K, t, S)
    lo, hi = max(0, t + K - N), min(t, K)
    pv = chi2_pvalue(xs, lambda k: hyper_logpmf(N, K, t, k), lo, hi)
    assert pv > P_MIN, (branch, pv)
    mean = t * K / N
    var = t * (K / N) * (1 - K / N) * (N - t) / (N - 1)
    assert abs(np.mean(xs) - mean) < 5 * math.sqrt(var / S) + 1e-9, branch


# binomial-regime cases: N >= 2^32 t, law = Binomial(t, K/N)
BINREG_CASES = [
    (2 ** 50, 2 ** 49, 2048, "fair-bit count (even split, t <= 2^15)"),
    (2 ** 50, 2 ** 49, 77, "fair-bit count, partial word"),
    (2 ** 50, 2 ** 49, 127, "fair-bit count, 63-bit last word"),
    (2 ** 60, 2 ** 59, 40000, "even split above 2^15: binomial ratio of uniforms"),
    (2 ** 60, 2 ** 60 // 100, 100000, "binomial ratio of uniforms"),
    (2 ** 72, 2 ** 52, 10 ** 6, "binomial inversion (mean ~ 0.95)"),
    (2 ** 72, 2 ** 72 - 2 ** 52, 10 ** 6, "binomial, K symmetry"),
]


@pytest.mark.parametrize("N,K,t,branch", BINREG_CASES)
def test_hypergeometric_binomial_regime(orc, N, K, t, branch):
    S = 20000
    xs = draw_hyper(orc, N, K, t, S)
    p = K / N
    mean, sd = t * p, math.sqrt(t * p * (1 - p))
    lo, hi = max(0, int(mean - 12 * sd) - 2), min(t, int(mean + 12 * sd) + 2)
    assert min(xs) >= lo and max(xs) <= hi, branch
    pv = chi2_pvalue(xs, lambda k: binom_logpmf(t, p, k), lo, hi)
    assert pv > P_MIN, (branch, pv)


BINOM_CASES = [
    (50, 0.1, "inversion"),
    (10 ** 6, 3e-6, "inversion, large n"),
    (1000, 0.3, "ratio of uniforms"),
    (1000, 0.8, "ratio of uniforms via symmetry"),
    (2 ** 40, 1e-6, "ratio of uniforms, huge n"),
    (2 ** 44, 1e-13, "inversion, tiny p"),
    (25, 0.5, "ratio of uniforms, just above the switch"),
]


@pytest.mark.parametrize("n,p,branch", BINOM_CASES)
def test_binomial_chi_square(orc, n, p, branch):
    S = 30000
    xs = draw_binom(orc, n, p, S)
    mean, sd = n * p, math.sqrt(n * p * (1 - p))
    lo, hi = max(0, int(mean - 12 * sd) - 2), min(n, int(mean + 12 * sd) + 2)
    assert min(xs) >= lo and max(xs) <= hi, branch
    pv = chi2_pvalue(xs, lambda k: binom_logpmf(n, p, k), lo, hi)
    assert pv > P_MIN, (branch, pv)
    assert abs(np.mean(xs) - mean) < 5 * sd / math.sqrt(S) + 1e-12


def test_hypergeometric_special_cases(orc):
    for node in range(50):
        assert orc.hypergeometric(100, 0, 40, 1, node, 9) == 0
        assert orc.hypergeometric(100, 100, 40, 1, node, 9) == 40
        assert orc.hypergeometric(100, 37, 100, 1, node, 9) == 37
        assert orc.hypergeometric(100, 37, 0, 1, node, 9) == 0
        assert orc.hypergeometric(2 ** 80, 2 ** 79, 0, 1, node, 9) == 0
        x = orc.hypergeometric(10, 8, 9, 1, node, 9)  # support [7, 8]
        assert 7 <= x <= 8
    assert orc.binomial(0, 0.3, 1, 0, 9) == 0
    assert orc.binomial(17, 0.0, 1, 0, 9) == 0
    assert orc.binomial(17, 1.0, 1, 0, 9) == 17


def test_hypergeometric_tiny_exact_law(orc):
    """N = 6, K = 3, t = 3: pmf 1/20, 9/20, 9/20, 1/20 exactly."""
    S = 40000
    xs = np.array(draw_hyper(orc, 6, 3, 3, S, seed=77))
    want = [Fraction(1, 20), Fraction(9, 20), Fraction(9, 20), Fraction(1, 20)]
    obs = [np.count_nonzero(xs == k) for k in range(4)]
    chi2 = sum((o - float(w) * S) ** 2 / (float(w) * S) for o, w in zip(obs, want))
    assert stats.chi2.sf(chi2, 3) > P_MIN


# ---- the rejection sampler's envelope (the hat must cover the pmf) ----

D1 = 2 * math.sqrt(2 / math.e)
D2 = 3 - 2 * math.sqrt(3 / math.e)


def _envelope_ok(logpmf, lo, hi, mean, var, mode):
    """Ratio of uniforms: (X, V) uniform on (0,1] x [-s/2, s/2), W = a + V/X,
    accept k = floor(W) iff X^2 <= f(k)/f(mode).  Exact iff for every w:
    f(floor w) <= f(mode) and |w - a| sqrt(f(floor w)/f(mode)) <= s/2."""
    a = mean + 0.5
    s = D1 * math.sqrt(var + 0.5) + D2
    lm = logpmf(mode)
    for k in range(lo, hi + 1):
        r = logpmf(k) - lm
        if r > 1e-12:
            return False, ("mode is not a maximum", k)
        h = math.exp(0.5 * r)
        if max(abs(k - a), abs(k + 1 - a)) * h > s / 2 * (1 + 1e-12):
            return False, ("outside the hat", k)
    return True, None


@pytest.mark.parametrize("N", [40, 100, 1000, 10 ** 5, 10 ** 7])
def test_hypergeometric_hat_covers_pmf(N):
    rng = np.random.default_rng(N)
    for _ in range(60):
        K = int(rng.integers(1, N // 2 + 1))
        t = int(rng.integers(1, N // 2 + 1))
        mean = t * K / N
        if mean < 10 or (t << 32) <= N:
            continue
        p = K / N
        var = (N - t) * t * p * (1 - p) / (N - 1)
        mode = ((t + 1) * (K + 1)) // (N + 2)
        span = int(40 * math.sqrt(var)) + 40
        lo, hi = max(0, int(mean) - span), min(t, K, int(mean) + span)
        ok, why = _envelope_ok(lambda k: hyper_logpmf(N, K, t, k), lo, hi, mean, var, mode)
        assert ok, (N, K, t, why)


@pytest.mark.parametrize("n", [20, 50, 200, 5000, 10 ** 6])
def test_binomial_hat_covers_pmf(n):
    rng = np.random.default_rng(n)
    for _ in range(60):
        p = float(rng.uniform(0.0, 0.5))
        if n * p < 10:
            continue
        mean, var = n * p, n * p * (1 - p)
        mode = math.floor((n + 1) * p)
        span = int(40 * math.sqrt(var)) + 40
        lo, hi = max(0, int(mean) - span), min(n, int(mean) + span)
        ok, why = _envelope_ok(lambda k: binom_logpmf(n, p, k), lo, hi, mean, var, mode)
        assert ok, (n, p, why)
