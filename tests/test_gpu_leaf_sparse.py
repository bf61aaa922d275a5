"""GPU parity of the sparse leaf kernel (directed tiles of >= 2^26 pairs,
where Floyd's sampler almost never replaces a draw) with the oracle.  The
kernel leaves a tile to the general leaf kernel when it holds more than 1536
draws or when two draws are equal; these cases are forced here, next to long
rows (runs of one row across warps and tiles) for the fused digest."""
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


def test_repeated_draws_go_to_the_general_kernel(kg, orc):
    """n = 2^20, m = 2^24, 16 chunks: tiles of 2^26 pairs with ~1024 draws, so
    about one tile in 128 (some 128 of 16384) repeats a draw."""
    n, m, P = 1 << 20, 1 << 24, 16
    t = kg.gnm_directed(n, m, 41, P, id_bytes=8)
    kg.check_device_error()
    gu, gv = edges_np(t, 8)
    ou, ov = orc.gnm_directed(n, m, 41, P)
    assert_same_edges(gu, gv, ou, ov, "sparse tiles with repeats")


def test_tiles_over_1536_draws_are_routed_away(kg, orc):
    """k_leaf = 1600: tile counts around 1590 +- 40, most above the sparse
    kernel's 1536 (left to the general kernel), the rest sampled by it."""
    n, P = 1 << 22, 4
    m = 4 * 1590 * 1024
    t = kg.gnm_directed(n, m, 43, P, id_bytes=4, k_leaf=1600, k_max=2048)
    kg.check_device_error()
    gu, gv = edges_np(t, 4)
    ou, ov = orc.gnm_directed(n, m, 43, P, 1600, 2048)
    assert_same_edges(gu, gv, ou, ov, "k around 1590")


def _chunk(kg, n, m, seed, P, c, id_bytes, digest=True):
    import torch
    s = kg._stream_ptr(None)
    counts = torch.zeros(P, dtype=torch.int64, device="cuda")
    kg.kg_gnm_directed_chunk_counts(n, m, seed, P, counts.data_ptr(), s)
    kc = int(counts[c].item())
    dt = torch.int32 if id_bytes == 4 else torch.int64
    out = torch.empty((kc, 2), dtype=dt, device="cuda")
    dig = torch.zeros(1, dtype=torch.int64, device="cuda")
    hist = torch.zeros(65, dtype=torch.int64, device="cuda")
    kg.kg_gnm_directed_range(n, m, seed, P, c, c + 1, counts.data_ptr(), id_bytes, out.data_ptr(),
                             kc, dig.data_ptr() if digest else 0, hist.data_ptr() if digest else 0,
                             s)
    kg.check_device_error()
    return kc, out, int(dig.cpu().numpy().view(np.uint64)[0]), hist.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("c", [0, 9])
def test_long_rows_digest_and_histogram(kg, orc, c):
    """n = 2^24, m = 2^28, 16 chunks: tiles of 2^30 pairs span 64 rows of ~16
    edges, so runs of one row cross warps and tiles.  The chunk's edges, digest
    and out-degree histogram equal the oracle's."""
    n, m, P = 1 << 24, 1 << 28, 16
    kc, out, dig, hist = _chunk(kg, n, m, 5, P, c, 8)
    gu, gv = edges_np(out, 8)
    ou, ov = orc.gnm_directed_chunk(n, m, 5, P, c, kc)
    assert_same_edges(gu, gv, ou, ov, f"chunk {c}")
    assert dig == orc.edge_checksum(ou, ov)
    r0, r1 = c * n // P, (c + 1) * n // P
    assert np.array_equal(hist, orc.outdegree_hist(ou, r0, r1))


@pytest.mark.parametrize("c", [0, 63])
def test_uint32_ids(kg, orc, c):
    """n = 2^30, m = 2^26, 64 chunks, uint32 ids: tiles of 2^44 pairs."""
    n, m, P = 1 << 30, 1 << 26, 64
    kc, out, dig, hist = _chunk(kg, n, m, 7, P, c, 4, digest=False)
    gu, gv = edges_np(out, 4)
    ou, ov = orc.gnm_directed_chunk(n, m, 7, P, c, kc)
    assert_same_edges(gu, gv, ou, ov, f"chunk {c}")
