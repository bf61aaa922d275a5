"""GPU parity of the random geometric graph generator (Sec. 5) with the
oracle: bit-identical cell counts, coordinates and (u, v)-sorted edge lists."""
import math

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


def r_for_degree(dim, n, deg):
    """Radius whose ball holds `deg` expected neighbours (boundary ignored)."""
    vol = math.pi if dim == 2 else 4 * math.pi / 3
    return (deg / (vol * (n - 1))) ** (1 / dim)


CASES = [
    # dim, n, r, seed, id_bytes
    (2, 1, 0.3, 1, 4),
    (3, 2, 0.5, 2, 4),
    (2, 2000, 0.03, 3, 4),
    (3, 1500, 0.08, 4, 8),
    (2, 300, 0.5, 5, 4),          # 2 x 2 cells, the largest radius
    (3, 200, 0.5, 6, 4),
    (2, 4000, 0.001, 7, 4),       # cells bounded by n
    (2, 700, 0.25, 8, 8),         # cell side exactly R
    (2, 50, 0.0, 9, 4),           # r = 0
    (2, 200000, 0.003, 10, 8),
    (3, 100000, 0.02, 11, 4),
    (2, 1 << 20, r_for_degree(2, 1 << 20, 16), 12, 4),
    (3, 1 << 20, r_for_degree(3, 1 << 20, 16), 13, 4),
    (3, 6000, 0.5, 14, 4),        # 750 points per cell: FP64 splits above 1024, dense rows
    (3, 9000, 0.5, 15, 4),        # neighbourhood above the shared-memory stage: global reads
]


@pytest.mark.parametrize("dim,n,r,seed,id_bytes", CASES)
def test_rgg_bit_exact(kg, orc, dim, n, r, seed, id_bytes):
    if n * n * (r ** dim) > 6e8:
        pytest.skip("output too large for the oracle list")
    assert kg.rgg_grid(dim, n, r) == orc.rgg_grid_level(dim, n, r)
    cells = kg.rgg_cell_counts(dim, n, r, seed)
    kg.check_device_error()
    assert np.array_equal(cells.cpu().numpy().astype(np.uint64), orc.rgg_cell_counts(dim, n, r, seed))
    t, xy = kg.rgg(dim, n, r, seed, id_bytes=id_bytes, coords=True)
    kg.check_device_error()
    assert np.array_equal(xy.cpu().numpy().view(np.uint32), orc.rgg_points(dim, n, r, seed))
    gu, gv = edges_np(t, id_bytes)
    ou, ov = orc.rgg(dim, n, r, seed)
    assert_same_edges(gu, gv, ou, ov, f"rgg dim={dim} n={n} r={r}")


def test_rgg_zero_points_capacity_and_arguments(kg):
    import torch
    s = kg._stream_ptr(None)
    cnt = torch.full((1,), 77, dtype=torch.int64, device="cuda")
    out = torch.zeros((64, 2), dtype=torch.int32, device="cuda")
    kg.kg_rgg(2, 0, 0.1, 1, 4, out.data_ptr(), 64, cnt.data_ptr(), None, s)
    kg.check_device_error()
    assert int(cnt.item()) == 0
    # too small an output: capacity error, the count still exact, nothing past cap
    kg.kg_rgg_count(2, 3000, 0.05, 2, cnt.data_ptr(), s)
    need = int(cnt.item())
    assert need > 64
    big = torch.zeros((need, 2), dtype=torch.int32, device="cuda")
    kg.kg_rgg(2, 3000, 0.05, 2, 4, big.data_ptr(), 64, cnt.data_ptr(), None, s)
    assert kg.kg_last_error(s) == kg.KG_ERR_CAPACITY
    assert int(cnt.item()) == need
    assert int(big[64:].abs().sum()) == 0
    full = kg.rgg(2, 3000, 0.05, 2)
    assert torch.equal(big[:64], full[:64])
    L = kg.lib()
    p = out.data_ptr()
    assert L.kg_rgg(4, 10, 0.1, 1, 4, p, 64, cnt.data_ptr(), None, s) == kg.KG_ERR_ARG
    assert L.kg_rgg(2, 10, 0.6, 1, 4, p, 64, cnt.data_ptr(), None, s) == kg.KG_ERR_ARG
    assert L.kg_rgg(2, 10, float("nan"), 1, 4, p, 64, cnt.data_ptr(), None, s) == kg.KG_ERR_ARG
    assert L.kg_rgg(2, 10, 0.1, 1, 3, p, 64, cnt.data_ptr(), None, s) == kg.KG_ERR_ARG
    assert L.kg_rgg(2, 1 << 32, 0.1, 1, 4, p, 64, cnt.data_ptr(), None, s) == kg.KG_ERR_RANGE
    assert L.kg_rgg(2, 10, 0.1, 1, 4, p, 64, None, None, s) == kg.KG_ERR_ARG


def test_rgg_repeatable(kg):
    a = kg.rgg(3, 50000, 0.03, 5).cpu()
    b = kg.rgg(3, 50000, 0.03, 5).cpu()
    kg.check_device_error()
    assert a.shape == b.shape and bool((a == b).all())


@pytest.mark.parametrize("dim", [2, 3])
def test_rgg_at_scale_digest_and_sampled_rows(kg, orc, dim):
    """n = 2^24, average degree 16: entry count, digest and degree histogram
    of the whole graph, and two sampled vertex ranges entry by entry."""
    import torch
    n, seed = 1 << 24, 21
    r = r_for_degree(dim, n, 16)
    t = kg.rgg(dim, n, r, seed, id_bytes=4)
    kg.check_device_error()
    dig = torch.zeros(1, dtype=torch.int64, device="cuda")
    kg.kg_edge_digest(t.data_ptr(), t.shape[0], 4, dig.data_ptr(), kg._stream_ptr(None))
    entries, digest, hist = orc.rgg_digest(dim, n, r, seed)
    assert t.shape[0] == entries
    assert int(dig.item()) & ((1 << 64) - 1) == digest
    u = t[:, 0].to(torch.int64)
    deg = torch.bincount(u, minlength=n).clamp(max=64)
    assert np.array_equal(torch.bincount(deg, minlength=65).cpu().numpy().astype(np.uint64), hist)
    for lo in (0, n // 2 + 12345):
        hi = lo + 5000
        a, b = (int(x) for x in torch.searchsorted(u, torch.tensor([lo, hi], device="cuda")))
        gu, gv = edges_np(t[a:b], 4)
        ou, ov = orc.rgg_rows(dim, n, r, seed, lo, hi)
        assert_same_edges(gu, gv, ou, ov, f"rows [{lo}, {hi})")


def test_rgg_largest_ids_properties(kg):
    """n = 2^31 points (ids up to 2^31 - 1 in uint32 output, 2^30 cells): no
    oracle at this size, so what holds at any size: cell counts sum to n, rows
    strictly sorted without self-loops, the edge set symmetric (equal digests
    of the list and of its transpose), every entry within the radius."""
    import torch
    n, r, seed = 1 << 31, 1e-6, 3
    assert kg.rgg_grid(2, n, r) == 15
    cells = kg.rgg_cell_counts(2, n, r, seed)
    kg.check_device_error()
    assert int(cells.sum()) == n
    del cells
    t, xy = kg.rgg(2, n, r, seed, id_bytes=4, coords=True)
    kg.check_device_error()
    k = t.shape[0]
    assert k % 2 == 0 and k > 1000
    u = t[:, 0].to(torch.int64) & 0xffffffff
    v = t[:, 1].to(torch.int64) & 0xffffffff
    assert int(u.max()) >= 1 << 30
    assert bool((u != v).all())
    key = u * n + v
    assert bool((key[1:] > key[:-1]).all())
    s = kg._stream_ptr(None)
    d1 = torch.zeros(1, dtype=torch.int64, device="cuda")
    d2 = torch.zeros(1, dtype=torch.int64, device="cuda")
    tt = torch.stack((t[:, 1], t[:, 0]), dim=1).contiguous()
    kg.kg_edge_digest(t.data_ptr(), k, 4, d1.data_ptr(), s)
    kg.kg_edge_digest(tt.data_ptr(), k, 4, d2.data_ptr(), s)
    assert int(d1.item()) == int(d2.item())
    R = int(r * 2 ** 32)
    pu = xy[u].to(torch.int64) & 0xffffffff
    pv = xy[v].to(torch.int64) & 0xffffffff
    d = pu - pv
    assert int((d * d).sum(dim=1).max()) <= R * R
