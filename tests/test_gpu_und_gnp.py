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
    # rectangle tiles of 2^26 pairs (576 tiles of ~1000 draws): the sparse leaf
    # kernel, about one tile in 128 with a repeated draw (its fallback list)
    (1 << 18, 512000, 17, 8, 4, 1024, 2048),
    (1 << 18, 512000, 18, 8, 8, 1024, 2048),
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


# The emit pass walks a tile a second time when its kept pairs overflow its
# slots (k > slots), and walks every tile twice when the slots would pass
# 12 GB (slots = 0, what a large kg_gnp_directed call does).  Both branches
# are forced through the slot-count hook and compared with the oracle.
@pytest.mark.parametrize("slots", [0, 1, 3])
@pytest.mark.parametrize("und,n,p,seed,P,id_bytes,k_leaf", GNP_CASES)
def test_gnp_regenerate_path_bit_exact(kg, orc, slots, und, n, p, seed, P, id_bytes, k_leaf):
    out, cnt = kg.gnp(und, n, p, seed, P, id_bytes=id_bytes, k_leaf=k_leaf, slots_per_tile=slots)
    kg.check_device_error()
    k = int(cnt.item())
    gu, gv = edges_np(out[:k], id_bytes)
    ou, ov = orc.gnp(und, n, p, seed, P, k_leaf)
    assert_same_edges(gu, gv, ou, ov, f"gnp slots={slots} und={und} n={n} p={p} P={P}")


@pytest.mark.parametrize("slots", [0, 700])
def test_config2_regenerate_path(kg, orc, slots):
    """The n = 2^20, degree-16 instance with every tile walked twice (0 slots)
    and with 700 slots per tile, below the ~1024 kept pairs of most tiles."""
    n = 1 << 20
    p = 16 / (n - 1)
    out, cnt = kg.gnp(True, n, p, 1, 32, id_bytes=4, slots_per_tile=slots)
    kg.check_device_error()
    k = int(cnt.item())
    gu, gv = edges_np(out[:k], 4)
    ou, ov = orc.gnp(True, n, p, 1, 32, cap_hint=1 << 25)
    assert_same_edges(gu, gv, ou, ov, f"config 2, {slots} slots")


def test_gnp_directed_regenerate_large_tiles(kg, orc):
    """Directed, tiles of 2^20 pairs with ~1000 kept pairs each and a handful
    of slots: nearly every tile overflows and is regenerated."""
    n, p, P = 40000, 1e-3, 5
    out, cnt = kg.gnp(False, n, p, 3, P, id_bytes=8, slots_per_tile=5)
    kg.check_device_error()
    k = int(cnt.item())
    gu, gv = edges_np(out[:k], 8)
    ou, ov = orc.gnp(False, n, p, 3, P, cap_hint=1 << 22)
    assert_same_edges(gu, gv, ou, ov, "directed, 5 slots")


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


@pytest.mark.parametrize("und,n,p,P", [(False, 3000, 0.01, 7), (True, 5000, 0.003, 31),
                                        (True, 1, 0.5, 1), (False, 100, 0.0, 4)])
def test_gnp_size_is_what_the_default_generators_write(kg, und, n, p, P):
    """kg_gnp_size sizes kg_gnp_directed / kg_gnp_undirected exactly, and the
    output sized by it holds the whole list."""
    import torch
    s = kg._stream_ptr(None)
    size = torch.full((1,), 77, dtype=torch.int64, device="cuda")
    kg.kg_gnp_size(int(und), n, p, 9, P, size.data_ptr(), s)
    k = int(size.item())
    out = torch.zeros((max(k, 1), 2), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    f = kg.lib().kg_gnp_undirected if und else kg.lib().kg_gnp_directed
    assert f(n, p, 9, P, 4, out.data_ptr(), k, cnt.data_ptr(), s) == kg.KG_OK
    assert kg.kg_last_error(s) == kg.KG_OK
    assert int(cnt.item()) == k
    ref, rcnt = kg.gnp(und, n, p, 9, P, id_bytes=4)
    assert int(rcnt.item()) == k
    assert torch.equal(out[:k].cpu(), ref[:k].cpu())


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


# ---------------------------------------------------------------- undirected rows by row blocks

def _rows(kg, n, m, seed, P, b0, b1, id_bytes, cap, counts=None):
    import torch
    s = kg._stream_ptr(None)
    out = torch.zeros((max(cap, 1), 2), dtype=torch.int64 if id_bytes == 8 else torch.int32,
                      device="cuda")
    ent = torch.zeros(1, dtype=torch.int64, device="cuda")
    dig = torch.zeros(b1 - b0, dtype=torch.int64, device="cuda")
    hist = torch.zeros((b1 - b0, 65), dtype=torch.int64, device="cuda")
    kg.kg_gnm_undirected_rows(n, m, seed, P, b0, b1, counts.data_ptr() if counts is not None else 0,
                              id_bytes, out.data_ptr(), cap, ent.data_ptr(), dig.data_ptr(),
                              hist.data_ptr(), s)
    kg.check_device_error()
    k = int(ent.item())
    return (out[:k], dig.cpu().numpy().view(np.uint64), hist.cpu().numpy().view(np.uint64))


@pytest.mark.parametrize("n,m,seed,P,ranges,id_bytes", [
    (1000, 20000, 3, 7, [(0, 1), (1, 4), (4, 7)], 4),
    (5000, 5000 * 4999 // 4, 4, 4, [(1, 3)], 4),            # rows of ~2500 entries
    (333, 1000, 5, 333, [(0, 100), (100, 101), (101, 333)], 8),
    ((1 << 20) + 7, 1 << 22, 6, 32, [(5, 9), (31, 32)], 8),
])
def test_undirected_rows_bit_exact(kg, orc, n, m, seed, P, ranges, id_bytes):
    """Rows of a range of row blocks: equal to the oracle's rows, digest and
    degree histogram of every block equal to the oracle's."""
    for b0, b1 in ranges:
        ou, ov = orc.gnm_undirected_rows(n, m, seed, P, b0, b1)
        t, dig, hist = _rows(kg, n, m, seed, P, b0, b1, id_bytes, len(ou) + 16)
        gu, gv = edges_np(t, id_bytes)
        assert_same_edges(gu, gv, ou, ov, f"rows n={n} blocks [{b0},{b1})")
        for b in range(b0, b1):
            lo, hi = b * n // P, (b + 1) * n // P
            sel = (ou >= lo) & (ou < hi)
            assert int(dig[b - b0]) == orc.edge_checksum(ou[sel], ov[sel])
            assert np.array_equal(hist[b - b0], orc.outdegree_hist(ou[sel], lo, hi))


def test_undirected_rows_concatenate_to_the_whole_graph(kg):
    import torch
    n, m, P, seed = 30000, 400000, 9, 7
    whole = kg.gnm_undirected(n, m, seed, P).clone()
    parts = [_rows(kg, n, m, seed, P, b0, b1, 4, 2 * m)[0] for b0, b1 in [(0, 2), (2, 3), (3, 9)]]
    assert torch.equal(torch.cat(parts), whole)


def test_undirected_rows_at_scale_sampled_blocks(kg, orc):
    """n = 2^32 vertices (uint64 ids), m = 2^31, 1024 x 1024 chunk matrix: two
    sampled row blocks against the oracle (chunk counts drawn once on the GPU)."""
    import torch
    n, m, P, seed = 1 << 32, 1 << 31, 1024, 1
    counts = torch.zeros(P * (P + 1) // 2, dtype=torch.int64, device="cuda")
    kg.kg_gnm_undirected_chunk_counts(n, m, seed, P, counts.data_ptr(), kg._stream_ptr(None))
    assert int(counts.sum()) == m
    for b in (3, 700):
        ou, ov = orc.gnm_undirected_rows(n, m, seed, P, b, b + 1, cap_hint=1 << 24)
        t, dig, hist = _rows(kg, n, m, seed, P, b, b + 1, 8, len(ou) + 16, counts)
        gu, gv = edges_np(t, 8)
        assert_same_edges(gu, gv, ou, ov, f"block {b}")
        lo, hi = b * n // P, (b + 1) * n // P
        assert int(dig[0]) == orc.edge_checksum(ou, ov)
        assert np.array_equal(hist[0], orc.outdegree_hist(ou, lo, hi))


def test_bucketed_assembly_whole_graph(kg, orc):
    """n = 2^22, m = 2^22 (two entries per row): the whole list goes through
    the bucketed assembly (4096 buckets of 1024 rows, counting sort by row in
    shared memory) and equals the oracle's."""
    n, m, P = 1 << 22, 1 << 22, 64
    t = kg.gnm_undirected(n, m, 3, P, id_bytes=4)
    kg.check_device_error()
    gu, gv = edges_np(t, 4)
    ou, ov = orc.gnm_undirected(n, m, 3, P)
    assert_same_edges(gu, gv, ou, ov, "bucketed assembly")


def test_bucketed_assembly_widened_buckets(kg, orc):
    """A row window of 2^24 rows (n = 2^26, 64 row blocks, blocks [8, 24)) whose
    caller-given capacity allows 2.2 entries per row: at the target bucket
    width that needs 2^15 buckets, more than the shared-memory histogram holds,
    so the assembly widens them to 2^10 rows (2^14 buckets); the window's rows,
    digests and degree histograms equal the oracle's."""
    n, m, P, seed, b0, b1 = 1 << 26, 1 << 25, 64, 11, 8, 24
    cap = int(2.2 * (1 << 24))
    t, dig, hist = _rows(kg, n, m, seed, P, b0, b1, 4, cap)
    gu, gv = edges_np(t, 4)
    ou, ov = orc.gnm_undirected_rows(n, m, seed, P, b0, b1, cap_hint=cap)
    assert_same_edges(gu, gv, ou, ov, "widened buckets")
    for b in range(b0, b1):
        lo, hi = b * n // P, (b + 1) * n // P
        sel = (ou >= lo) & (ou < hi)
        assert int(dig[b - b0]) == orc.edge_checksum(ou[sel], ov[sel])
        assert np.array_equal(hist[b - b0], orc.outdegree_hist(ou[sel], lo, hi))
