"""GPU parity of undirected G(n,m) (Sec. 4.2) and directed / undirected G(n,p)
(Sec. 4.3) with the oracle: bit-identical (u, v)-sorted lists."""
import numpy as np
import pytest

from gpu_util import assert_same_edges, edges_np, need_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kg():
    need_cuda()
    import paper_1710_07565_gb300 as kg
    kg.lib()
    return kg


UND_CASES = [
    # n, m, seed, P, id_bytes, k_leaf, k_max
    (5, 4, 1, 5, 4, 1024, 2048),
    (50, 1225, 3, 7, 4, 2, 2),              # complete graph, deep trees, re-splits
    (1000, 999 * 1000 // 4, 5, 5, 8, 1024, 2048),  # density 1/2: Floyd collisions
    (4000, 32000, 7, 32, 4, 1024, 2048),
    (100000, 800000, 9, 33, 4, 1024, 2048),  # odd chunk count, ragged blocks
    (3000, 40000, 11, 1, 8, 64, 100),        # one triangle chunk
    (777, 5000, 13, 777, 4, 3, 5),           # one vertex per block
    (2, 1, 15, 2, 4, 1024, 2048),
]


@pytest.mark.parametrize("n,m,seed,P,id_bytes,k_leaf,k_max", UND_CASES)
def test_gnm_undirected_bit_exact(kg, orc, n, m, seed, P, id_bytes, k_leaf, k_max):
    t = kg.gnm_undirected(n, m, seed, P, id_bytes=id_bytes, k_leaf=k_leaf, k_max=k_max)
    kg.check_device_error()
    gu, gv = edges_np(t, id_bytes)
    ou, ov = orc.gnm_undirected(n, m, seed, P, k_leaf, k_max)
    assert_same_edges(gu, gv, ou, ov, f"undirected n={n} m={m} P={P}")


def test_gnm_undirected_dense_rows(kg, orc):
    """Rows longer than 32, and degrees around the 4096-entry shared-memory
    sort limit (n = 8193, half of all pairs: degrees 4096 +- 32)."""
    n, m, P = 8193, 8193 * 8192 // 4, 3
    t = kg.gnm_undirected(n, m, 21, P, id_bytes=4)
    kg.check_device_error()
    gu, gv = edges_np(t, 4)
    ou, ov = orc.gnm_undirected(n, m, 21, P)
    assert_same_edges(gu, gv, ou, ov, "dense undirected")


def _gnp(kg, und, n, p, seed, P, id_bytes, k_leaf=1024, cap=None):
    out, cnt = kg.gnp(und, n, p, seed, P, id_bytes=id_bytes, k_leaf=k_leaf, cap=cap)
    kg.check_device_error()
    k = int(cnt.item())
    return edges_np(out[:k], id_bytes)


GNP_CASES = [
    # undirected, n, p, seed, P, id_bytes, k_leaf
    (False, 3000, 2e-3, 1, 16, 4, 1024),
    (False, 100, 0.3, 2, 7, 8, 2),           # tiny tiles
    (False, 50, 0.999, 3, 5, 4, 1024),
    (False, 64, 1.0, 4, 4, 4, 1024),          # every pair
    (False, (1 << 32) + 7, 1e-13, 5, 3, 8, 1024),  # n(n-1) > 2^64, tiles > 2^32 pairs
    (True, 4096, 4 / 4095, 6, 8, 4, 1024),
    (True, 5000, 0.01, 7, 31, 8, 16),
    (True, 300, 0.5, 8, 300, 4, 1024),        # one vertex per block
    (True, 40, 1.0, 9, 3, 4, 1024),
]


@pytest.mark.parametrize("und,n,p,seed,P,id_bytes,k_leaf", GNP_CASES)
def test_gnp_bit_exact(kg, orc, und, n, p, seed, P, id_bytes, k_leaf):
    gu, gv = _gnp(kg, und, n, p, seed, P, id_bytes, k_leaf)
    ou, ov = orc.gnp(und, n, p, seed, P, k_leaf)
    assert_same_edges(gu, gv, ou, ov, f"gnp und={und} n={n} p={p} P={P}")


def test_config2_undirected_gnp(kg, orc):
    """n = 2^20, p = 16/(n-1), 32 x 32 chunk grid, uint32 ids, both directions."""
    n = 1 << 20
    p = 16 / (n - 1)
    gu, gv = _gnp(kg, True, n, p, 1, 32, 4)
    ou, ov = orc.gnp(True, n, p, 1, 32, cap_hint=1 << 25)
    assert_same_edges(gu, gv, ou, ov, "config 2")
    # E[m] = p n(n-1)/2 = 8 n: the count is within 6 sd
    m = len(gu) // 2
    assert abs(m - 8 * n) < 6 * (8 * n) ** 0.5


def test_gnp_zero_and_capacity(kg):
    import torch
    s = kg._stream_ptr(None)
    out = torch.zeros((8, 2), dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), 77, dtype=torch.int64, device="cuda")
    kg.kg_gnp_ex(0, 1000, 0.0, 1, 4, 1024, 4, out.data_ptr(), 8, cnt.data_ptr(), s)
    kg.check_device_error()
    assert int(cnt.item()) == 0
    # too small an output buffer: count reported, capacity error, nothing past cap
    big = torch.zeros((1000, 2), dtype=torch.int32, device="cuda")
    kg.kg_gnp_ex(0, 2000, 0.01, 1, 4, 1024, 4, big.data_ptr(), 100, cnt.data_ptr(), s)
    assert kg.kg_last_error(s) == kg.KG_ERR_CAPACITY
    assert int(cnt.item()) > 100
    assert int(big[100:].abs().sum()) == 0
    L = kg.lib()
    assert L.kg_gnp_ex(0, 10, 1.5, 1, 2, 1024, 4, out.data_ptr(), 8, cnt.data_ptr(), s) == kg.KG_ERR_ARG
    assert L.kg_gnp_ex(1, 10, 0.5, 1, 11, 1024, 4, out.data_ptr(), 8, cnt.data_ptr(), s) == kg.KG_ERR_ARG
    assert L.kg_gnm_undirected(10, 46, 1, 2, 4, out.data_ptr(), 100, s) == kg.KG_ERR_ARG
    assert L.kg_gnm_undirected(10, 5, 1, 2, 4, out.data_ptr(), 9, s) == kg.KG_ERR_CAPACITY


# ---------------------------------------------------------------- G(n,p), binomial chunk counts

GNPB_CASES = [
    # undirected, n, p, seed, P, id_bytes
    (False, 1000, 0.01, 3, 7, 4),
    (False, 3000, 0.5, 4, 16, 4),              # dense: Floyd replacements in most leaves
    (False, 64, 1.0, 5, 4, 8),                 # every pair
    (False, 1 << 20, 4 / (1 << 20), 6, 64, 8),  # binomial at 2^34-pair chunks
    (True, 5000, 0.01, 7, 31, 4),
    (True, 300, 0.5, 8, 300, 4),               # one vertex per block
    (True, 1 << 20, 16 / ((1 << 20) - 1), 1, 32, 4),  # the n = 2^20, degree-16 instance
]


@pytest.mark.parametrize("und,n,p,seed,P,id_bytes", GNPB_CASES)
def test_gnp_binomial_bit_exact(kg, orc, und, n, p, seed, P, id_bytes):
    import torch
    t = kg.gnp_binomial(und, n, p, seed, P, id_bytes)
    kg.check_device_error()
    gu, gv = edges_np(t, id_bytes)
    mean = n * (n - 1) * p / (1 if not und else 2)
    ou, ov = orc.gnp_binomial(und, n, p, seed, P, cap_hint=int(2 * mean + 1024) * 2)
    assert_same_edges(gu, gv, ou, ov, f"gnp_binomial und={und} n={n} p={p} P={P}")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    kg.kg_gnp_binomial_count(und, n, p, seed, P, cnt.data_ptr(), kg._stream_ptr(None))
    assert int(cnt.item()) == len(ou)


def test_gnp_binomial_zero_capacity_and_range(kg):
    import torch
    s = kg._stream_ptr(None)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = torch.zeros((16, 2), dtype=torch.int32, device="cuda")
    kg.kg_gnp_binomial(False, 100, 0.0, 1, 4, 4, out.data_ptr(), 16, cnt.data_ptr(), s)
    kg.check_device_error()
    assert int(cnt.item()) == 0 and int(out.abs().sum()) == 0
    L = kg.lib()
    # 100 x 99 pairs at p = 1/2 do not fit 16 slots: the count is exact, the error recorded
    assert L.kg_gnp_binomial(0, 100, 0.5, 1, 4, 4, out.data_ptr(), 16, cnt.data_ptr(), s) == 0
    torch.cuda.synchronize()
    assert L.kg_last_error(s) == kg.KG_ERR_CAPACITY
    assert int(cnt.item()) > 16
    # chunks of 2^66 pairs are beyond the binomial's exact range
    assert L.kg_gnp_binomial(0, 1 << 40, 1e-9, 1, 16, 8, out.data_ptr(), 16, cnt.data_ptr(), s) \
        == kg.KG_ERR_RANGE
