"""Helpers for the GPU tests: device tensors <-> numpy edge arrays."""
import numpy as np
import pytest


def need_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def edges_np(t, id_bytes):
    """(k, 2) int32/int64 device tensor -> (u, v) uint64 numpy arrays."""
    a = t.cpu().numpy()
    if id_bytes == 4:
        a = a.view(np.uint32).astype(np.uint64)
    else:
        a = a.view(np.uint64)
    return a[:, 0].copy(), a[:, 1].copy()


def assert_same_edges(got_u, got_v, want_u, want_v, what=""):
    assert len(got_u) == len(want_u), f"{what}: {len(got_u)} edges, oracle {len(want_u)}"
    if len(want_u) == 0:
        return
    bad = np.nonzero((got_u != want_u) | (got_v != want_v))[0]
    assert bad.size == 0, (f"{what}: {bad.size} mismatches, first at {bad[0]}: "
                           f"got ({got_u[bad[0]]},{got_v[bad[0]]}) oracle ({want_u[bad[0]]},{want_v[bad[0]]})")
