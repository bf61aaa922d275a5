"""GPU parity of directed G(n,m) (Sec. 4.1) with the oracle: bit-identical
edge lists for the same (n, m, seed, chunks) through the C ABI."""
import ctypes

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


def run_directed(kg, n, m, seed, P, id_bytes=4, k_leaf=1024, k_max=2048):
    t = kg.gnm_directed(n, m, seed, P, id_bytes=id_bytes, k_leaf=k_leaf, k_max=k_max)
    kg.check_device_error()
    return edges_np(t, id_bytes)


def test_config1_bit_exact(kg, orc):
    """n = 2^16, m = 2^20, 64 chunks, seed 1, uint32 ids: the whole list."""
    n, m, P = 1 << 16, 1 << 20, 64
    gu, gv = run_directed(kg, n, m, 1, P, 4)
    ou, ov = orc.gnm_directed(n, m, 1, P)
    assert_same_edges(gu, gv, ou, ov, "config 1")


CASES = [
    # n, m, seed, P, id_bytes, k_leaf, k_max
    (10, 30, 3, 3, 4, 2, 2),                       # deep tile tree, re-split of full leaves
    (100, 5000, 5, 7, 8, 16, 24),                  # small leaves, dense
    (1000, 999000 // 2, 7, 13, 4, 1024, 2048),     # density 1/2: Floyd collisions everywhere
    (3, 6, 1, 3, 4, 2, 2),                         # complete graph
    (2, 1, 9, 1, 4, 1024, 2048),
    (12345, 777777, 11, 31, 4, 1024, 2048),        # ragged chunks and tiles
    (5000, 1 << 18, 13, 1, 8, 1024, 2048),         # one chunk
    ((1 << 20) + 3, 1 << 22, 17, 1000, 8, 1024, 2048),
    ((1 << 33) + 5, 1 << 20, 19, 17, 8, 1024, 2048),  # universe > 2^64: binomial regime, fair bits
    (4097, 300000, 23, 4097, 4, 64, 100),          # one row per chunk
    (600, 5000, 29, 600, 4, 3, 5),                 # many tiny tiles with re-splits
    (3037000501, 1000, 31, 1, 4, 1024, 2048),      # one tile just above 2^63 pairs: Lemire
                                                   # rejects about half of the draws
    (1 << 32, 1500, 37, 1, 8, 1024, 2048),         # one tile near 2^64: every draw takes the
                                                   # rejection test's slow branch
]


@pytest.mark.parametrize("n,m,seed,P,id_bytes,k_leaf,k_max", CASES)
def test_directed_bit_exact(kg, orc, n, m, seed, P, id_bytes, k_leaf, k_max):
    gu, gv = run_directed(kg, n, m, seed, P, id_bytes, k_leaf, k_max)
    ou, ov = orc.gnm_directed(n, m, seed, P, k_leaf, k_max)
    assert_same_edges(gu, gv, ou, ov, f"n={n} m={m} P={P}")


def test_zero_edges_and_single_vertex(kg):
    import torch
    out = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
    kg.kg_gnm_directed(1, 0, 1, 1, 4, out.data_ptr(), 0, kg._stream_ptr(None))
    kg.kg_gnm_directed(50, 0, 1, 5, 4, out.data_ptr(), 0, kg._stream_ptr(None))
    kg.check_device_error()
    assert int(out.abs().sum()) == 0


def test_argument_errors(kg):
    import torch
    s = kg._stream_ptr(None)
    out = torch.zeros((16, 2), dtype=torch.int32, device="cuda")
    p = out.data_ptr()
    L = kg.lib()
    assert L.kg_gnm_directed(10, 91, 1, 2, 4, p, 100, s) == kg.KG_ERR_ARG        # m > n(n-1)
    assert L.kg_gnm_directed(10, 20, 1, 11, 4, p, 100, s) == kg.KG_ERR_ARG       # P > n
    assert L.kg_gnm_directed(10, 20, 1, 0, 4, p, 100, s) == kg.KG_ERR_ARG        # P = 0
    assert L.kg_gnm_directed(10, 20, 1, 2, 3, p, 100, s) == kg.KG_ERR_ARG        # id_bytes
    assert L.kg_gnm_directed(10, 20, 1, 2, 4, p, 19, s) == kg.KG_ERR_CAPACITY    # cap < m
    assert L.kg_gnm_directed((1 << 32) + 1, 20, 1, 2, 4, p, 100, s) == kg.KG_ERR_RANGE
    assert L.kg_gnm_directed(1 << 40, (1 << 44) + 1, 1, 2, 8, p, 1 << 50, s) == kg.KG_ERR_RANGE
    assert L.kg_gnm_directed_ex(10, 20, 1, 2, 4096, 4096, 4, p, 100, s) == kg.KG_ERR_ARG
    assert L.kg_gnm_directed_ex(10, 20, 1, 2, 8, 4, 4, p, 100, s) == kg.KG_ERR_ARG
    kg.check_device_error()


def test_shutdown_releases_state_and_calls_still_work(kg):
    """kg_shutdown frees the error word and trims the cached scratch; a call
    after it makes that state again and returns the same graph."""
    import torch
    a = kg.gnm_directed(5000, 40000, 3, 8, id_bytes=4)
    kg.check_device_error()
    a = a.cpu()
    kg.kg_shutdown()
    b = kg.gnm_directed(5000, 40000, 3, 8, id_bytes=4)
    kg.check_device_error()
    assert torch.equal(a, b.cpu())
    kg.kg_shutdown()
    kg.kg_shutdown()  # idempotent
    # the error word is made again: a capacity error found on the device
    s = kg._stream_ptr(None)
    out = torch.zeros((100, 2), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    kg.kg_gnp_ex(0, 2000, 0.01, 1, 4, 1024, 4, out.data_ptr(), 100, cnt.data_ptr(), s)
    assert kg.kg_last_error(s) == kg.KG_ERR_CAPACITY
    assert kg.kg_last_error(s) == kg.KG_OK


def test_repeatable_and_stream_independent(kg):
    import torch
    n, m, P = 50000, 300000, 9
    a = kg.gnm_directed(n, m, 77, P).clone()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = kg.gnm_directed(n, m, 77, P, stream=s)
    s.synchronize()
    assert torch.equal(a, b)
    c = kg.gnm_directed(n, m, 78, P)
    assert not torch.equal(a, c)


CONFIG3 = (1 << 36, 1 << 33, 1 << 16)  # n, m, chunks


def test_config3_chunk_counts(kg, orc):
    import torch
    n, m, P = CONFIG3
    d = torch.zeros(P, dtype=torch.int64, device="cuda")
    kg.kg_gnm_directed_chunk_counts(n, m, 1, P, d.data_ptr(), kg._stream_ptr(None))
    kg.check_device_error()
    got = d.cpu().numpy().view(np.uint64)
    want = orc.gnm_directed_chunk_counts(n, m, 1, P)
    assert np.array_equal(got, want)
    assert int(got.sum()) == m


def test_config3_sampled_chunks(kg, orc):
    """Directed G(n,m) at scale (n = 2^36, m = 2^33, 2^16 chunks, uint64 ids):
    64 chunks chosen with seed 7 are generated through the chunk-range entry
    point; each chunk's edges are compared with the oracle's in full, together
    with the per-chunk digest and out-degree histogram."""
    import torch
    n, m, P = CONFIG3
    s = kg._stream_ptr(None)
    counts = torch.zeros(P, dtype=torch.int64, device="cuda")
    kg.kg_gnm_directed_chunk_counts(n, m, 1, P, counts.data_ptr(), s)
    cnt = counts.cpu().numpy().view(np.uint64)
    chunks = sorted(np.random.default_rng(7).choice(P, 64, replace=False).tolist())
    for c in chunks:
        kc = int(cnt[c])
        out = torch.empty((kc, 2), dtype=torch.int64, device="cuda")
        dig = torch.zeros(1, dtype=torch.int64, device="cuda")
        hist = torch.zeros(65, dtype=torch.int64, device="cuda")
        kg.kg_gnm_directed_range(n, m, 1, P, c, c + 1, counts.data_ptr(), 8, out.data_ptr(), kc,
                                 dig.data_ptr(), hist.data_ptr(), s)
        kg.check_device_error()
        gu, gv = edges_np(out, 8)
        ou, ov = orc.gnm_directed_chunk(n, m, 1, P, c, kc)
        assert_same_edges(gu, gv, ou, ov, f"chunk {c}")
        assert int(dig.cpu().numpy().view(np.uint64)[0]) == orc.edge_checksum(ou, ov)
        r0, r1 = c * n // P, (c + 1) * n // P
        assert np.array_equal(hist.cpu().numpy().view(np.uint64), orc.outdegree_hist(ou, r0, r1))


def test_range_concatenation_equals_whole(kg):
    """Chunk ranges generated separately (the paper's PEs) concatenate to the full list."""
    import torch
    n, m, P = 30000, 500000, 12
    s = kg._stream_ptr(None)
    whole = kg.gnm_directed(n, m, 5, P).clone()
    counts = torch.zeros(P, dtype=torch.int64, device="cuda")
    kg.kg_gnm_directed_chunk_counts(n, m, 5, P, counts.data_ptr(), s)
    cnt = counts.cpu().numpy()
    parts, pos = [], 0
    for c0, c1 in [(0, 5), (5, 6), (6, 12)]:
        k = int(cnt[c0:c1].sum())
        out = torch.empty((max(k, 1), 2), dtype=torch.int32, device="cuda")
        kg.kg_gnm_directed_range(n, m, 5, P, c0, c1, counts.data_ptr(), 4, out.data_ptr(), k, 0, 0, s)
        parts.append(out[:k])
    kg.check_device_error()
    assert torch.equal(torch.cat(parts), whole)


def test_edge_digest_matches_oracle(kg, orc):
    import torch
    n, m = 70000, 400000
    t = kg.gnm_directed(n, m, 3, 5, id_bytes=8)
    d = torch.zeros(1, dtype=torch.int64, device="cuda")
    kg.kg_edge_digest(t.data_ptr(), m, 8, d.data_ptr(), kg._stream_ptr(None))
    kg.check_device_error()
    u, v = edges_np(t, 8)
    assert int(d.cpu().numpy().view(np.uint64)[0]) == orc.edge_checksum(u, v)


@pytest.mark.parametrize("n,m,P,seed", [
    (2000, 2000 * 1999 // 3, 4, 21),       # rows of ~670 edges: runs across warps and tiles
    (1 << 16, 1 << 22, 16, 22),            # rows of ~64 edges
    (1 << 20, 1 << 21, 8, 23),             # rows of ~2 edges
    (5000, 5000 * 4999 // 2, 3, 24),       # density 1/2: replaced draws in every leaf
])
def test_fused_digest_and_histogram_per_chunk(kg, orc, n, m, P, seed):
    """The digest and out-degree histogram fused into the leaf kernel equal the
    oracle's checksum and histogram of each chunk, at row lengths from ~2 to
    ~2500 edges (runs of equal rows crossing warps, tiles and chunks)."""
    import torch
    s = kg._stream_ptr(None)
    counts = torch.zeros(P, dtype=torch.int64, device="cuda")
    kg.kg_gnm_directed_chunk_counts(n, m, seed, P, counts.data_ptr(), s)
    cnt = counts.cpu().numpy().view(np.uint64)
    k = int(cnt.sum())
    out = torch.empty((k, 2), dtype=torch.int64, device="cuda")
    dig = torch.zeros(P, dtype=torch.int64, device="cuda")
    hist = torch.zeros((P, 65), dtype=torch.int64, device="cuda")
    kg.kg_gnm_directed_range(n, m, seed, P, 0, P, counts.data_ptr(), 8, out.data_ptr(), k,
                             dig.data_ptr(), hist.data_ptr(), s)
    kg.check_device_error()
    gd = dig.cpu().numpy().view(np.uint64)
    gh = hist.cpu().numpy().view(np.uint64)
    for c in range(P):
        ou, ov = orc.gnm_directed_chunk(n, m, seed, P, c, int(cnt[c]))
        assert int(gd[c]) == orc.edge_checksum(ou, ov), c
        r0, r1 = c * n // P, (c + 1) * n // P
        assert np.array_equal(gh[c], orc.outdegree_hist(ou, r0, r1)), c
