"""CPU checks of the library's host-callable arithmetic (no GPU): the FP64
procedure, variates, Lemire draws, invariant division and the undirected chunk
geometry, compiled from the library headers for the host and compared with the
oracle.  The oracle shares no code with the library; agreement here is the
first evidence that both follow the same written procedure."""
import ctypes
import math

import numpy as np
import pytest

import host_shim


@pytest.fixture(scope="module")
def sh():
    return host_shim.load()


def test_fp64_functions_bit_equal(orc, sh):
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.uniform(0, 1, 20000), np.exp(rng.uniform(-700, 700, 20000)),
                         np.arange(1, 3000, dtype=float), [2.0 ** -1074, 5e-324 * 7]])
    for x in xs:
        x = float(x)
        if x <= 0:
            continue
        assert sh.sh_log(x) == orc.log(x), x
    for p in np.concatenate([10 ** rng.uniform(-300, -0.01, 10000), rng.uniform(0, 1, 5000)]):
        p = float(p)
        if 0 < p < 1:
            assert sh.sh_log1m(p) == orc.log1m(p), p
    for x in rng.uniform(-720, 720, 20000):
        assert sh.sh_exp(float(x)) == orc.exp(float(x)), x
    for k in list(range(200)) + [int(v) for v in rng.integers(0, 1 << 52, 5000)]:
        assert sh.sh_lnfact(float(k)) == orc.lnfact(k), k
    for _ in range(20000):
        a = float(int(rng.integers(0, 1 << int(rng.integers(1, 60)))))
        d = float(int(rng.integers(-min(a, 1e6), 1e6 + 1)))
        assert sh.sh_lnfact_diff(a, d) == orc.lnfact_diff(a, d), (a, d)


def test_u128_conversion_bit_equal(orc, sh):
    rng = np.random.default_rng(6)
    for _ in range(20000):
        hi = int(rng.integers(0, 1 << 63)) >> int(rng.integers(0, 63))
        lo = int(rng.integers(0, 1 << 63)) * 2 + int(rng.integers(0, 2))
        assert sh.sh_dbl128(lo, hi) == orc.u128_to_double((hi << 64) | lo)


def test_streams_bit_equal(orc, sh):
    rng = np.random.default_rng(7)
    for _ in range(5000):
        seed, node = int(rng.integers(0, 1 << 63)) * 2, int(rng.integers(0, 1 << 63))
        tag, i = int(rng.integers(0, 1 << 32)), int(rng.integers(0, 1 << 33))
        assert sh.sh_stream_u64(seed, node, tag, i) == orc.stream_u64(seed, node, tag, i)


def _hyper_cases():
    return [(40, 7, 13), (1000, 30, 100), (1000, 970, 100), (1000, 30, 900), (1000, 300, 400),
            (1000, 700, 800), (100000, 50000, 50000), (2 ** 40, int(0.3 * 2 ** 40), 4096),
            (2 ** 24, 2 ** 23, 4096), (2 ** 50, 2 ** 49, 2048), (2 ** 50, 2 ** 49, 127),
            (2 ** 60, 2 ** 59, 40000), (2 ** 60, 2 ** 60 // 100, 100000), (2 ** 72, 2 ** 52, 10 ** 6),
            (2 ** 72 - 5, 2 ** 71 + 3, 2 ** 33), (6, 3, 3), (10, 8, 9), (100, 100, 40), (100, 0, 3)]


def test_variates_bit_equal(orc, sh):
    out = ctypes.c_uint64()
    for N, K, t in _hyper_cases():
        for node in range(300):
            rc = sh.sh_hyper(N & (2 ** 64 - 1), N >> 64, K & (2 ** 64 - 1), K >> 64, t, 11, node, 3,
                             ctypes.byref(out))
            assert rc == 0
            assert out.value == orc.hypergeometric(N, K, t, 11, node, 3), (N, K, t, node)
    for n, p in [(50, 0.1), (10 ** 6, 3e-6), (1000, 0.3), (1000, 0.8), (2 ** 40, 1e-6),
                 (2 ** 44, 1e-13), (25, 0.5), (0, 0.5), (9, 1.0)]:
        for node in range(300):
            assert sh.sh_binom(n, p, 5, node, 9, ctypes.byref(out)) == 0
            assert out.value == orc.binomial(n, p, 5, node, 9), (n, p, node)


def test_lemire_matches_oracle_leaf(orc, sh):
    """Floyd draws: draw i of a leaf is Lemire-uniform on [0, L-k+i]."""
    rng = np.random.default_rng(8)
    for _ in range(200):
        L = int(rng.integers(1, 1 << 62)) if rng.random() < 0.7 else int(rng.integers(1, 50))
        k = int(rng.integers(1, min(L, 60) + 1))
        node = int(rng.integers(0, 1 << 40))
        draws = [sh.sh_lemire(3, node, i, L - k + i + 1) for i in range(k)]
        # replay Floyd on the draws and compare with the oracle's leaf
        S = set()
        for i, t in enumerate(draws):
            S.add(t if t not in S else L - k + i)
        assert sorted(S) == orc.floyd_leaf(L, k, 3, node).tolist()


@pytest.mark.parametrize("D", [1, 2, 3, 7, 255, 65535, 2 ** 32 - 1, 2 ** 36 - 1, 2 ** 63 - 25,
                               2 ** 63, 2 ** 64 - 1, 1000003])
def test_invariant_division(sh, D):
    rng = np.random.default_rng(D % 1000)
    xs = np.concatenate([rng.integers(0, 2 ** 63, 20000, dtype=np.uint64) * np.uint64(2)
                         + rng.integers(0, 2, 20000, dtype=np.uint64),
                         np.array([x & (2 ** 64 - 1) for x in
                                   (0, 1, D - 1, D, D + 1, 2 ** 64 - 1, (2 ** 64 - 1) // D * D)],
                                  dtype=np.uint64)])
    q = np.zeros_like(xs)
    P = ctypes.POINTER(ctypes.c_uint64)
    sh.sh_divq(D, xs.ctypes.data_as(P), q.ctypes.data_as(P), len(xs))
    for x, qq in zip(xs.tolist(), q.tolist()):
        assert qq == x // D, (x, D)


def test_undirected_geometry(sh):
    """Chunk index k <-> (i, j), universes and offset -> pair maps against brute force."""
    for n, P in [(10, 3), (33, 5), (7, 7), (100, 1), (17, 4)]:
        bounds = [c * n // P for c in range(P + 1)]
        k = 0
        for i in range(P):
            for j in range(i + 1):
                ri, si = bounds[i], bounds[i + 1] - bounds[i]
                rj, sj = bounds[j], bounds[j + 1] - bounds[j]
                if i == j:
                    pairs = [(u, v) for u in range(ri, ri + si) for v in range(ri, u)]
                else:
                    pairs = [(u, v) for u in range(ri, ri + si) for v in range(rj, rj + sj)]
                assert sh.sh_und_universe(n, P, k) == len(pairs)
                u, v = ctypes.c_uint64(), ctypes.c_uint64()
                for off, want in enumerate(pairs):
                    sh.sh_und_map(n, P, k, off, ctypes.byref(u), ctypes.byref(v))
                    assert (u.value, v.value) == want
                k += 1


def test_row_bounds_without_wide_division(sh):
    """r_c = floor(c n / P) through n = qP + r and an invariant multiplier."""
    import ctypes as C
    sh.sh_row_bound.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64]
    sh.sh_row_bound.restype = C.c_uint64
    rng = np.random.default_rng(9)
    for n, P in [(1 << 36, 1 << 16), (65536, 64), (12345, 31), (10, 3), (2 ** 63 + 11, 1 << 24),
                 (2 ** 64 - 1, 3), (7, 7), (1 << 20, 32)]:
        cs = set(range(0, min(P, 50) + 1)) | {P} | {int(x) for x in rng.integers(0, P + 1, 200)}
        for c in cs:
            assert sh.sh_row_bound(n, P, c) == c * n // P, (n, P, c)


def test_workload_generators_are_deterministic_and_in_range():
    from paper_1710_07565_gb300 import workloads
    a = workloads.batched_instances(4096)
    b = workloads.batched_instances(4096)
    assert a == b and len(a) == 4096
    for q in a:
        assert 256 <= q["n"] <= 1 << 20
        pairs = q["n"] * (q["n"] - 1) // (2 if q["undirected"] else 1)
        assert 0 <= q["m"] <= pairs
        assert 1 <= q["chunks"] <= (32 if q["undirected"] else 64) and q["chunks"] <= q["n"]
        deg = (2 * q["m"] if q["undirected"] else q["m"]) / q["n"]
        assert 1.9 <= deg <= 64.1 or q["m"] == pairs
    frac_und = sum(q["undirected"] for q in a) / len(a)
    assert 0.45 < frac_und < 0.55
    r = workloads.serving_requests(2000, 100.0)
    assert r == workloads.serving_requests(2000, 100.0)
    assert all(r[i]["arrival"] < r[i + 1]["arrival"] for i in range(len(r) - 1))
    assert all(1 << 10 <= q["n"] <= 1 << 26 for q in r)
