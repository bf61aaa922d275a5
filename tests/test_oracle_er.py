"""Pins of the oracle's Erdos-Renyi generators against what the paper fixes.

* G(n,m) is uniform over all graphs with m edges (Sec. 2.1): brute-force
  enumeration of all graphs on n <= 5 vertices, for several chunk counts P
  (Sec. 4.1 / 4.2: the decomposition must not change the law) and with a
  tiny leaf size so the tile tree and the re-split of full leaves are used.
* G(n,p) draws every pair independently with probability p (Sec. 2.1):
  exact graph probabilities on n <= 4, E[m] z-tests, degree chi-square and
  inclusion frequencies of pairs on tile and chunk borders.
* Simple graphs (Sec. 2): no self-loops, no duplicates; undirected output
  holds both directions; the chunk tree distributes exactly m samples.
"""
import itertools
import math
from collections import Counter

import numpy as np
import pytest
from scipy import stats

P_MIN = 1e-5


def chi2_uniform(counts, n_cells):
    S = sum(counts.values())
    exp_ = S / n_cells
    chi2 = sum((c - exp_) ** 2 / exp_ for c in counts.values()) + (n_cells - len(counts)) * exp_
    return float(stats.chi2.sf(chi2, n_cells - 1))


def check_simple(u, v, n, directed, m=None):
    assert np.all(u < n) and np.all(v < n)
    assert not np.any(u == v), "self-loop"
    key = u.astype(object) * n + v.astype(object) if n > 2 ** 31 else u * np.uint64(n) + v
    assert np.all(np.diff(key.astype(np.float64) if n > 2 ** 31 else key.astype(np.int64)) > 0), \
        "not strictly sorted / duplicate"
    if m is not None:
        assert len(u) == (m if directed else 2 * m)
    if not directed:
        fwd = set(zip(u.tolist(), v.tolist()))
        assert all((b, a) in fwd for a, b in fwd), "not symmetric"


# ---------------------------------------------------------------- G(n,m)

@pytest.mark.parametrize("n,m,P,k_leaf,k_max", [
    (4, 3, 1, 1024, 4096),
    (4, 3, 2, 1024, 4096),
    (4, 3, 4, 1024, 4096),
    (4, 5, 3, 2, 2),          # deep tile tree + re-split of full leaves
    (5, 4, 2, 1024, 4096),
])
def test_gnm_directed_uniform_over_all_graphs(orc, n, m, P, k_leaf, k_max):
    n_graphs = math.comb(n * (n - 1), m)
    S = 60 * n_graphs if n_graphs < 1000 else 40 * n_graphs
    counts = Counter()
    for seed in range(S):
        u, v = orc.gnm_directed(n, m, seed, P, k_leaf, k_max)
        counts[tuple(zip(u.tolist(), v.tolist()))] += 1
    for g in counts:
        assert len(set(g)) == m and all(a != b for a, b in g)
    assert len(counts) <= n_graphs
    assert chi2_uniform(counts, n_graphs) > P_MIN


@pytest.mark.parametrize("n,m,P,k_leaf,k_max", [
    (5, 4, 1, 1024, 4096),
    (5, 4, 2, 1024, 4096),
    (5, 4, 5, 1024, 4096),
    (5, 6, 3, 2, 3),
    (6, 3, 4, 2, 2),
])
def test_gnm_undirected_uniform_over_all_graphs(orc, n, m, P, k_leaf, k_max):
    n_graphs = math.comb(n * (n - 1) // 2, m)
    S = 60 * n_graphs
    counts = Counter()
    for seed in range(S):
        u, v = orc.gnm_undirected(n, m, seed, P, k_leaf, k_max)
        check_simple(u, v, n, directed=False, m=m)
        counts[tuple((a, b) for a, b in zip(u.tolist(), v.tolist()) if a > b)] += 1
    assert chi2_uniform(counts, n_graphs) > P_MIN


@pytest.mark.parametrize("n,m,P", [(65536, 1 << 20, 64), (1000, 999 * 1000 // 3, 7), (300, 89700, 300),
                                   (10, 90, 3), (2, 2, 2), (1, 0, 1), (100, 0, 5)])
def test_gnm_directed_invariants(orc, n, m, P):
    u, v = orc.gnm_directed(n, m, 1, P)
    check_simple(u, v, n, directed=True, m=m)
    cnt = orc.gnm_directed_chunk_counts(n, m, 1, P)
    assert int(cnt.sum()) == m
    bounds = [c * n // P for c in range(P + 1)]
    for c in range(P):
        rows = bounds[c + 1] - bounds[c]
        assert int(cnt[c]) <= rows * (n - 1)
        assert np.count_nonzero((u >= bounds[c]) & (u < bounds[c + 1])) == int(cnt[c])


@pytest.mark.parametrize("n,m,P", [(4000, 32000, 32), (1000, 999 * 1000 // 4, 5), (50, 1225, 7),
                                   (7, 10, 7), (2, 1, 2), (100, 0, 3)])
def test_gnm_undirected_invariants(orc, n, m, P):
    u, v = orc.gnm_undirected(n, m, 3, P)
    check_simple(u, v, n, directed=False, m=m)
    cnt = orc.gnm_undirected_chunk_counts(n, m, 3, P)
    assert int(np.tril(cnt).sum()) == m and int(np.triu(cnt, 1).sum()) == 0


def test_complete_graph(orc):
    n = 9
    u, v = orc.gnm_directed(n, n * (n - 1), 5, 3, 2, 2)
    assert len(u) == n * (n - 1)
    u, v = orc.gnm_undirected(n, n * (n - 1) // 2, 5, 4, 2, 2)
    assert len(u) == n * (n - 1)


def test_chunk_count_marginal_is_hypergeometric(orc):
    """Chunk 0 of a directed G(n,m) holds Hyp(n(n-1), rows_0 (n-1), m) samples."""
    n, m, P = 30, 200, 4
    rows0 = n // P + 0  # floor(1 * 30 / 4) = 7
    N, K = n * (n - 1), (n * 1 // P) * (n - 1)
    xs = [int(orc.gnm_directed_chunk_counts(n, m, seed, P)[0]) for seed in range(20000)]
    lg = math.lgamma

    def logpmf(k):
        return (lg(K + 1) - lg(k + 1) - lg(K - k + 1) + lg(N - K + 1) - lg(m - k + 1)
                - lg(N - K - m + k + 1) - lg(N + 1) + lg(m + 1) + lg(N - m + 1))
    ks = range(0, min(m, K) + 1)
    probs = np.array([math.exp(logpmf(k)) for k in ks])
    obs = np.bincount(xs, minlength=len(probs))[: len(probs)]
    mask = probs * len(xs) >= 5
    e = probs[mask] * len(xs)
    o = obs[mask]
    e = e * o.sum() / e.sum()
    assert stats.chi2.sf(float(((o - e) ** 2 / e).sum()), mask.sum() - 1) > P_MIN
    assert rows0 == 7


def test_law_does_not_depend_on_chunk_count(orc):
    """The degree sequence law is the same for P = 1 and P = 8 (Sec. 4.1)."""
    n, m = 64, 400
    d1 = np.concatenate([np.bincount(orc.gnm_directed(n, m, s, 1)[0].astype(np.int64), minlength=n)
                         for s in range(300)])
    d8 = np.concatenate([np.bincount(orc.gnm_directed(n, m, s, 8)[0].astype(np.int64), minlength=n)
                         for s in range(300)])
    assert stats.ks_2samp(d1, d8).pvalue > 1e-4


def test_floyd_leaf_uniform_over_subsets(orc):
    """Floyd's algorithm draws every k-subset of [0, L) with probability 1/C(L,k)."""
    for L, k in [(5, 2), (6, 3), (8, 4), (7, 7), (8, 1)]:
        n_sets = math.comb(L, k)
        S = 400 * n_sets
        counts = Counter(tuple(orc.floyd_leaf(L, k, 99, node).tolist()) for node in range(S))
        for s in counts:
            assert len(s) == k and list(s) == sorted(set(s)) and max(s) < L
        if n_sets == 1:
            assert len(counts) == 1
            continue
        assert chi2_uniform(counts, n_sets) > P_MIN


def test_floyd_leaf_large_universe(orc):
    L = (1 << 64) - 5
    out = orc.floyd_leaf(L, 3000, 1, 42)
    assert len(np.unique(out)) == 3000 and np.all(np.diff(out.astype(object)) > 0)


# ---------------------------------------------------------------- G(n,p)

@pytest.mark.parametrize("undirected,n,P", [(False, 4, 1), (False, 3, 3), (True, 4, 2), (True, 5, 5)])
def test_gnp_exact_graph_law(orc, undirected, n, P):
    p = 0.3
    pairs = [(a, b) for a in range(n) for b in range(n) if a != b and (not undirected or a > b)]
    S = 40000
    counts = Counter()
    for seed in range(S):
        u, v = orc.gnp(undirected, n, p, seed, P, 2)
        counts[tuple((a, b) for a, b in zip(u.tolist(), v.tolist()) if (not undirected or a > b))] += 1
    # pool by edge count: P(|E| = j) = C(N,j) p^j q^(N-j); then uniform within each count
    Np = len(pairs)
    by_size = Counter()
    for g, c in counts.items():
        by_size[len(g)] += c
    obs = np.array([by_size.get(j, 0) for j in range(Np + 1)], dtype=float)
    exp_ = np.array([math.comb(Np, j) * p ** j * (1 - p) ** (Np - j) for j in range(Np + 1)]) * S
    mask = exp_ >= 5
    chi2 = float(((obs[mask] - exp_[mask]) ** 2 / exp_[mask]).sum())
    assert stats.chi2.sf(chi2, mask.sum() - 1) > P_MIN
    # every pair appears with frequency p
    inc = Counter()
    for g, c in counts.items():
        for e in g:
            inc[e] += c
    for e in pairs:
        z = (inc[e] - S * p) / math.sqrt(S * p * (1 - p))
        assert abs(z) < 5, (e, z)


@pytest.mark.parametrize("undirected,n,p,P", [(False, 3000, 2e-3, 16), (True, 4096, 4 / 4095, 8),
                                              (True, 1 << 14, 16 / ((1 << 14) - 1), 32)])
def test_gnp_edge_count_and_degrees(orc, undirected, n, p, P):
    u, v = orc.gnp(undirected, n, p, 7, P)
    check_simple(u, v, n, directed=not undirected)
    Npairs = n * (n - 1) // (2 if undirected else 1)
    m = len(u) // (2 if undirected else 1)
    z = (m - Npairs * p) / math.sqrt(Npairs * p * (1 - p))
    assert abs(z) < 5, z
    deg = np.bincount(u.astype(np.int64), minlength=n)
    # (out-)degree ~ Binomial(n-1, p)
    kmax = int(deg.max())
    obs = np.bincount(deg, minlength=kmax + 1).astype(float)
    pm = stats.binom.pmf(np.arange(kmax + 1), n - 1, p)
    pm[-1] += stats.binom.sf(kmax, n - 1, p)
    e = pm * n
    mask = e >= 5
    o2, e2 = obs[mask], e[mask]
    e2 = e2 * o2.sum() / e2.sum()
    assert stats.chi2.sf(float(((o2 - e2) ** 2 / e2).sum()), mask.sum() - 1) > 1e-4


def test_gnp_pairs_on_tile_and_chunk_borders(orc):
    """Pairs at both ends of every tile and chunk appear with frequency p."""
    n, P, p, k_leaf = 12, 3, 0.25, 2   # tile length T = 8 pairs, chunks of 4 rows x 11
    S = 20000
    hits = np.zeros((n, n))
    for seed in range(S):
        u, v = orc.gnp(False, n, p, seed, P, k_leaf)
        hits[u.astype(np.int64), v.astype(np.int64)] += 1
    T = 8
    border = set()
    for c in range(P):
        r0 = c * n // P
        Uc = (c + 1) * n // P * (n - 1) - r0 * (n - 1)
        for lo in list(range(0, Uc, T)) + [Uc]:
            for off in (lo - 1, lo):
                if 0 <= off < Uc:
                    uu, w = r0 + off // (n - 1), off % (n - 1)
                    border.add((uu, w + (w >= uu)))
    assert len(border) > 20
    for (a, b) in border:
        z = (hits[a, b] - S * p) / math.sqrt(S * p * (1 - p))
        assert abs(z) < 5, (a, b, z)


def test_gnp_extremes(orc):
    u, v = orc.gnp(False, 50, 0.0, 1, 4)
    assert len(u) == 0
    u, v = orc.gnp(False, 7, 1.0, 1, 3)
    assert len(u) == 42
    u, v = orc.gnp(True, 7, 1.0, 1, 3)
    assert len(u) == 42
    check_simple(u, v, 7, directed=False)


@pytest.mark.parametrize("n,m,P,k_leaf,k_max,splits", [
    (40, 300, 5, 4, 6, [0, 2, 3, 5]),
    (1000, 20000, 7, 1024, 2048, [0, 1, 4, 7]),
    (5000, 5000 * 4999 // 4, 4, 1024, 2048, [0, 2, 4]),   # rows of ~2500 entries
    (333, 1000, 333, 8, 16, [0, 100, 101, 333]),          # one vertex per block
])
def test_undirected_row_blocks_concatenate_to_the_graph(orc, n, m, P, k_leaf, k_max, splits):
    """Sec. 4.2: a PE that regenerates the chunks of its row and column blocks
    produces exactly its rows of the one graph; the row ranges concatenate to
    the full list in both directions."""
    fu, fv = orc.gnm_undirected(n, m, 3, P, k_leaf, k_max)
    parts_u, parts_v = [], []
    for b0, b1 in zip(splits[:-1], splits[1:]):
        u, v = orc.gnm_undirected_rows(n, m, 3, P, b0, b1, k_leaf, k_max)
        lo, hi = b0 * n // P, b1 * n // P
        assert np.all((u >= lo) & (u < hi))
        parts_u.append(u)
        parts_v.append(v)
    assert np.array_equal(np.concatenate(parts_u), fu)
    assert np.array_equal(np.concatenate(parts_v), fv)


# ------------------------------------------- G(n,p) by binomial chunk counts

def _graph_law(orc_fn, undirected, n, p, S):
    pairs = [(a, b) for a in range(n) for b in range(n) if a != b and (not undirected or a > b)]
    counts = Counter()
    for seed in range(S):
        u, v = orc_fn(seed)
        counts[tuple((a, b) for a, b in zip(u.tolist(), v.tolist()) if (not undirected or a > b))] += 1
    Np = len(pairs)
    by_size = Counter()
    for g, c in counts.items():
        by_size[len(g)] += c
    obs = np.array([by_size.get(j, 0) for j in range(Np + 1)], dtype=float)
    exp_ = np.array([math.comb(Np, j) * p ** j * (1 - p) ** (Np - j) for j in range(Np + 1)]) * S
    mask = exp_ >= 5
    chi2 = float(((obs[mask] - exp_[mask]) ** 2 / exp_[mask]).sum())
    assert stats.chi2.sf(chi2, mask.sum() - 1) > P_MIN
    # within each edge count every graph is equally likely
    for j in range(Np + 1):
        graphs = {g: c for g, c in counts.items() if len(g) == j}
        cells = math.comb(Np, j)
        if cells > 1 and by_size.get(j, 0) >= 20 * cells:
            assert chi2_uniform(Counter(graphs), cells) > P_MIN, j


@pytest.mark.parametrize("undirected,n,P", [(False, 3, 1), (False, 3, 3), (True, 4, 2), (True, 4, 4)])
def test_gnp_binomial_exact_graph_law(orc, undirected, n, P):
    """Sec. 4.3 with binomial chunk counts: P(graph) = p^|E| (1-p)^(N-|E|),
    with leaves of two samples so the tile tree and Floyd are both used."""
    p = 0.35
    _graph_law(lambda seed: orc.gnp_binomial(undirected, n, p, seed, P, 2, 2), undirected, n, p,
               20000)


@pytest.mark.parametrize("mean", [4.0, 100.0])
def test_gnp_binomial_chunk_count_law_at_2e52_pairs(orc, mean):
    """One chunk of n(n-1) ~ 2^52 pairs: its count is Binomial(U, p), drawn by
    inversion (mean 4) or ratio of uniforms (mean 100) at a size beyond the
    G(n,m) limit."""
    n = 1 << 26
    U = n * (n - 1)
    p = mean / U
    S = 3000
    x = np.array([int(orc.gnp_binomial_counts(False, n, p, seed, 1)[0]) for seed in range(S)])
    kmax = int(x.max())
    obs = np.bincount(x, minlength=kmax + 1).astype(float)
    pm = stats.binom.pmf(np.arange(kmax + 1), U, p)
    pm[-1] += stats.binom.sf(kmax, U, p)
    e = pm * S
    mask = e >= 5
    o2, e2 = obs[mask], e[mask]
    rest_o, rest_e = obs[~mask].sum(), e[~mask].sum()
    chi2 = float(((o2 - e2) ** 2 / e2).sum()) + ((rest_o - rest_e) ** 2 / rest_e if rest_e > 0 else 0)
    assert stats.chi2.sf(chi2, mask.sum()) > P_MIN


@pytest.mark.parametrize("undirected,n,p,P", [(False, 3000, 2e-3, 16), (True, 1 << 14, 16 / ((1 << 14) - 1), 32)])
def test_gnp_binomial_edge_count_and_degrees(orc, undirected, n, p, P):
    u, v = orc.gnp_binomial(undirected, n, p, 11, P)
    check_simple(u, v, n, directed=not undirected)
    Npairs = n * (n - 1) // (2 if undirected else 1)
    m = len(u) // (2 if undirected else 1)
    assert abs((m - Npairs * p) / math.sqrt(Npairs * p * (1 - p))) < 5
    cnt = orc.gnp_binomial_counts(undirected, n, p, 11, P)
    assert int(cnt.sum()) == m      # the chunks hold exactly their binomial counts
    deg = np.bincount(u.astype(np.int64), minlength=n)
    kmax = int(deg.max())
    obs = np.bincount(deg, minlength=kmax + 1).astype(float)
    pm = stats.binom.pmf(np.arange(kmax + 1), n - 1, p)
    pm[-1] += stats.binom.sf(kmax, n - 1, p)
    e = pm * n
    mask = e >= 5
    o2, e2 = obs[mask], e[mask]
    e2 = e2 * o2.sum() / e2.sum()
    assert stats.chi2.sf(float(((o2 - e2) ** 2 / e2).sum()), mask.sum() - 1) > 1e-4


def test_gnp_binomial_extremes_and_limits(orc):
    u, v = orc.gnp_binomial(False, 50, 0.0, 1, 4)
    assert len(u) == 0
    u, v = orc.gnp_binomial(False, 7, 1.0, 1, 3)
    assert len(u) == 42
    u, v = orc.gnp_binomial(True, 9, 1.0, 1, 3)
    assert len(u) == 72
    check_simple(u, v, 9, directed=False)
    with pytest.raises(RuntimeError):
        orc.gnp_binomial_counts(False, 1 << 40, 1e-9, 1, 16)   # chunks of 2^66 pairs


# ---------------------------------------------------------------- digests

def test_checksum_is_order_independent_and_sensitive(orc):
    u, v = orc.gnm_directed(1000, 5000, 1, 4)
    c = orc.edge_checksum(u, v)
    perm = np.random.default_rng(0).permutation(len(u))
    assert orc.edge_checksum(u[perm], v[perm]) == c
    v2 = v.copy()
    v2[17] ^= 1
    assert orc.edge_checksum(u, v2) != c


def test_outdegree_hist(orc):
    u = np.array([3, 3, 5, 7, 7, 7], dtype=np.uint64)
    h = orc.outdegree_hist(u, 2, 10)
    assert h[0] == 5 and h[1] == 1 and h[2] == 1 and h[3] == 1 and h.sum() == 8
