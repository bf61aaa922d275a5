"""Pins of the RGG oracle (Sec. 5) against what the definition and the
mathematics fix: the edge set of a brute-force all-pairs test, the
multinomial law of the cell counts, uniform points, and the closed-form
probability that two uniform points of the unit square / cube lie within
distance r."""
import math

import numpy as np
import pytest

import oracle as orc_mod

stats = pytest.importorskip("scipy.stats")


@pytest.fixture(scope="module")
def orc():
    orc_mod.lib()
    return orc_mod


def brute_force_entries(x, r):
    """Every ordered pair (u, v), u != v, with |x_u - x_v|^2 <= floor(r 2^32)^2
    in exact integer arithmetic, sorted by (u, v)."""
    R = int(math.floor(r * 2 ** 32))
    n, dim = x.shape
    xi = x.astype(np.int64)
    us, vs = [], []
    for a in range(n):
        d = np.abs(xi - xi[a])                     # < 2^32 per coordinate
        ok = np.all(d <= R, axis=1)
        ok[a] = False
        dd = d[ok].astype(np.uint64)
        s = (dd * dd).sum(axis=1)                  # each term <= 2^62: no overflow
        vv = np.nonzero(ok)[0][s <= np.uint64(R) * np.uint64(R)]
        us.append(np.full(len(vv), a, dtype=np.uint64))
        vs.append(vv.astype(np.uint64))
    if not us:
        return np.zeros(0, np.uint64), np.zeros(0, np.uint64)
    return np.concatenate(us), np.concatenate(vs)


BRUTE_CASES = [
    # dim, n, r, seed
    (2, 2000, 0.03, 1),
    (3, 1500, 0.08, 2),
    (2, 300, 0.5, 3),      # the largest radius: 2 x 2 cells
    (3, 200, 0.5, 4),
    (2, 4000, 0.001, 5),   # cells bounded by n, far wider than r
    (3, 3000, 0.02, 6),
    (2, 50, 0.0, 7),       # r = 0: only coincident points would connect
    (2, 1, 0.3, 8),
    (3, 0, 0.1, 9),
    (2, 700, 0.25, 10),    # side exactly 2^30 lattice units = R
]


@pytest.mark.parametrize("dim,n,r,seed", BRUTE_CASES)
def test_rgg_edges_equal_brute_force(orc, dim, n, r, seed):
    x = orc.rgg_points(dim, n, r, seed)
    u, v = orc.rgg(dim, n, r, seed)
    bu, bv = brute_force_entries(x, r)
    assert len(u) == len(bu)
    assert np.array_equal(u, bu) and np.array_equal(v, bv)


def test_rgg_grid_level(orc):
    # side 2^(32-g) >= R, at most n cells, g <= 15 / 10
    assert orc.rgg_grid_level(2, 10 ** 6, 0.25) == 2
    assert orc.rgg_grid_level(2, 10 ** 6, 0.2) == 2   # side 2^30 >= 0.2 * 2^32, 2^29 is not
    assert orc.rgg_grid_level(2, 1000, 1e-6) == 4      # 2^(2*4) <= 1000 < 2^(2*5)
    assert orc.rgg_grid_level(3, 1 << 31, 1e-9) == 10
    assert orc.rgg_grid_level(2, (1 << 32) - 1, 0.0) == 15
    assert orc.rgg_grid_level(3, 7, 0.01) == 0


def test_rgg_argument_errors(orc):
    L = orc.lib()
    cnt = np.zeros(4, dtype=np.uint64)
    p = cnt.ctypes.data_as(orc_mod.ctypes.POINTER(orc_mod.ctypes.c_uint64))
    assert L.or_rgg_cell_counts(4, 10, 0.1, 1, p) == 1
    assert L.or_rgg_cell_counts(2, 10, 0.6, 1, p) == 1
    assert L.or_rgg_cell_counts(2, 10, -0.1, 1, p) == 1
    assert L.or_rgg_cell_counts(2, 10, float("nan"), 1, p) == 1
    assert L.or_rgg_cell_counts(2, 1 << 32, 0.1, 1, p) == 2


@pytest.mark.parametrize("dim,n,r", [(2, 5000, 0.02), (3, 4000, 0.05)])
def test_rgg_points_lie_in_their_cells_and_ids_follow_cells(orc, dim, n, r):
    g = orc.rgg_grid_level(dim, n, r)
    cnt = orc.rgg_cell_counts(dim, n, r, 11)
    assert int(cnt.sum()) == n
    x = orc.rgg_points(dim, n, r, 11)
    c = (x.astype(np.uint64) >> np.uint64(32 - g)).astype(np.int64)
    q = np.zeros(n, dtype=np.int64)
    for k in reversed(range(dim)):
        q = q * (1 << g) + c[:, k]
    # ids are grouped by row-major cell, cells in increasing order
    assert np.all(np.diff(q) >= 0)
    assert np.array_equal(np.bincount(q, minlength=len(cnt)), cnt.astype(np.int64))


def test_rgg_cell_counts_exact_multinomial_law(orc):
    """4 points over the 4 cells of a 2 x 2 grid: the 35 compositions have
    multinomial probabilities 4! / prod(k_i!) / 4^4."""
    from collections import Counter
    n, dim, r, seeds = 4, 2, 0.5, 6000
    assert orc.rgg_grid_level(dim, n, r) == 1
    freq = Counter()
    for s in range(seeds):
        freq[tuple(int(a) for a in orc.rgg_cell_counts(dim, n, r, s))] += 1
    comps = [(a, b, c, n - a - b - c) for a in range(n + 1) for b in range(n + 1 - a)
             for c in range(n + 1 - a - b)]
    assert len(comps) == 35
    expected = np.array([math.factorial(n) / np.prod([math.factorial(k) for k in cp]) / 4 ** n
                         for cp in comps]) * seeds
    observed = np.array([freq[cp] for cp in comps])
    assert observed.sum() == seeds
    chi2 = ((observed - expected) ** 2 / expected).sum()
    assert stats.chi2.sf(chi2, len(comps) - 1) > 1e-4


@pytest.mark.parametrize("dim,n,r", [(2, 20000, 0.05), (3, 20000, 0.2)])
def test_rgg_cell_counts_chi_square(orc, dim, n, r):
    """Every cell count is a Binomial(n, 1/cells) marginal of one multinomial."""
    for seed in (1, 2, 3):
        cnt = orc.rgg_cell_counts(dim, n, r, seed).astype(np.float64)
        e = n / len(cnt)
        chi2 = ((cnt - e) ** 2 / e).sum()
        assert stats.chi2.sf(chi2, len(cnt) - 1) > 1e-4


def test_rgg_root_split_above_the_fair_bit_limit_is_binomial(orc):
    """n = 5000 > 1024: the root split uses the Sec. 2.2 binomial variate; the
    lower half along the last dimension holds Binomial(5000, 1/2) points."""
    n, dim, r = 5000, 2, 0.5
    assert orc.rgg_grid_level(dim, n, r) == 1
    xs = np.array([int(orc.rgg_cell_counts(dim, n, r, s)[:2].sum()) for s in range(1500)])
    edges = np.array([0, 2440, 2460, 2480, 2490, 2500, 2510, 2520, 2540, 2560, 5001])
    obs = np.histogram(xs, bins=edges)[0]
    cdf = stats.binom.cdf(edges - 1, n, 0.5)
    exp = np.diff(cdf) * len(xs)
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-4


@pytest.mark.parametrize("dim", [2, 3])
def test_rgg_points_uniform_in_the_cube(orc, dim):
    """Bins of width 1/10 (not aligned with the power-of-two cells) hold equal shares."""
    n = 1 << 16
    x = orc.rgg_points(dim, n, 0.1, 21).astype(np.float64) / 2 ** 32
    for k in range(dim):
        obs = np.histogram(x[:, k], bins=10, range=(0, 1))[0]
        chi2 = ((obs - n / 10) ** 2 / (n / 10)).sum()
        assert stats.chi2.sf(chi2, 9) > 1e-4
    obs = np.histogram2d(x[:, 0], x[:, 1], bins=7, range=((0, 1), (0, 1)))[0].ravel()
    chi2 = ((obs - n / 49) ** 2 / (n / 49)).sum()
    assert stats.chi2.sf(chi2, 48) > 1e-4


def pair_probability(dim, r):
    """P(|X - Y| <= r) for independent uniform X, Y in [0,1]^dim, r <= 1.
    The displacement has density prod(1 - |a_k|) on [-1,1]^dim; integrating it
    over the ball of radius r term by term gives
      dim 2: pi r^2 - 8 r^3 / 3 + r^4 / 2,
      dim 3: 4 pi r^3 / 3 - 3 pi r^4 / 2 + 8 r^5 / 5 - r^6 / 6."""
    if dim == 2:
        return math.pi * r ** 2 - 8 * r ** 3 / 3 + r ** 4 / 2
    return 4 * math.pi * r ** 3 / 3 - 3 * math.pi * r ** 4 / 2 + 8 * r ** 5 / 5 - r ** 6 / 6


def test_pair_probability_by_monte_carlo():
    """The closed form itself, against direct sampling (independent of the oracle)."""
    rng = np.random.default_rng(5)
    for dim, r in ((2, 0.3), (3, 0.4)):
        a, b = rng.random((400000, dim)), rng.random((400000, dim))
        p = np.mean(((a - b) ** 2).sum(axis=1) <= r * r)
        assert abs(p - pair_probability(dim, r)) < 5 * math.sqrt(p * (1 - p) / 400000)


@pytest.mark.parametrize("dim,n,r", [(2, 2000, 0.05), (3, 2000, 0.1), (2, 500, 0.45)])
def test_rgg_mean_edge_count_matches_closed_form(orc, dim, n, r):
    rr = math.floor(r * 2 ** 32) / 2 ** 32
    want = n * (n - 1) / 2 * pair_probability(dim, rr)
    m = np.array([len(orc.rgg(dim, n, r, s)[0]) // 2 for s in range(40)], dtype=np.float64)
    se = m.std(ddof=1) / math.sqrt(len(m))
    assert abs(m.mean() - want) < 4.5 * se + 1e-9 * want


@pytest.mark.parametrize("dim,n,r", [(2, 3000, 0.04), (3, 2000, 0.1)])
def test_rgg_invariants_rows_and_digest(orc, dim, n, r):
    u, v = orc.rgg(dim, n, r, 31)
    assert len(u) % 2 == 0
    assert np.all(u != v)
    key = u * np.uint64(n) + v
    assert np.all(np.diff(key.astype(np.int64)) > 0)          # sorted, no duplicates
    assert np.array_equal(np.sort(v * np.uint64(n) + u), key)   # both directions
    a, b = n // 3, 2 * n // 3
    parts = [orc.rgg_rows(dim, n, r, 31, lo, hi) for lo, hi in ((0, a), (a, b), (b, n))]
    assert np.array_equal(np.concatenate([p[0] for p in parts]), u)
    assert np.array_equal(np.concatenate([p[1] for p in parts]), v)
    entries, digest, hist = orc.rgg_digest(dim, n, r, 31)
    assert entries == len(u)
    assert digest == orc.edge_checksum(u, v)
    deg = np.bincount(u.astype(np.int64), minlength=n)
    assert np.array_equal(hist, np.bincount(np.minimum(deg, 64), minlength=65).astype(np.uint64))
