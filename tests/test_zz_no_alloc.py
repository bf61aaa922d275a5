"""kg_gnm_directed_noalloc: the directed G(n,m) entry point for callers that
cannot let the library allocate device memory -- a framework whose caching
allocator already holds the GPU's memory, or a steady-state loop in which
allocation (which may synchronise the device and has no latency bound) is
forbidden.  Its scratch is a fixed array inside libkg.so.  It must return
exactly the bytes of kg_gnm_directed.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It calls the C ABI through
the ctypes binding; the output and status buffers are the caller's.
"""
import pytest

from gpu_util import need_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kg():
    need_cuda()
    import paper_1710_07565_gb300 as kg
    kg.lib()
    return kg


def _noalloc(kg, n, m, seed, P, id_bytes):
    import torch
    dt = torch.int32 if id_bytes == 4 else torch.int64
    out = torch.full((m, 2), -1, dtype=dt, device="cuda")
    status = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    s = kg._stream_ptr(None)
    kg.kg_gnm_directed_noalloc(n, m, seed, P, id_bytes, out.data_ptr(), m, status.data_ptr(), s)
    torch.cuda.synchronize()
    assert int(status.item()) == kg.KG_OK
    return out


def _reference(kg, n, m, seed, P, id_bytes):
    out = kg.gnm_directed(n, m, seed, P, id_bytes=id_bytes)
    kg.check_device_error()
    return out


def test_two_calls_in_a_row_match_the_allocating_entry_point(kg):
    import torch
    cases = [
        (1 << 16, 1 << 20, 1, 64, 4),        # n = 2^16, m = 2^20, 64 chunks, uint32 ids
        (12345, 777777, 11, 31, 8),          # ragged chunks and tiles, uint64 ids
    ]
    for n, m, seed, P, idb in cases:
        got = _noalloc(kg, n, m, seed, P, idb)
        want = _reference(kg, n, m, seed, P, idb)
        # integer output: equal bit for bit
        assert torch.equal(got, want), (n, m, P)


def _largest_fitting_chunks(kg, n, m):
    for P in range(256, 0, -1):
        if kg.kg_gnm_directed_noalloc_scratch(n, m, P) <= kg.NOALLOC_SCRATCH_BYTES:
            return P
    return 0


def test_largest_admitted_instance_matches(kg):
    """The largest chunk count whose scratch fits the array at tile depth 10
    (227 chunks of 2^10 tiles): the call runs and equals
    kg_gnm_directed."""
    import torch
    n, m = 1 << 20, 230_000_000
    P = _largest_fitting_chunks(kg, n, m)
    assert P > 128
    got = _noalloc(kg, n, m, 5, P, 4)
    want = _reference(kg, n, m, 5, P, 4)
    assert torch.equal(got, want)


def test_sizes_beyond_the_scratch_are_rejected_before_any_work(kg):
    import torch
    status = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    s = kg._stream_ptr(None)
    L = kg.lib()
    torch.cuda.synchronize()
    just_over = _largest_fitting_chunks(kg, 1 << 20, 230_000_000) + 1
    for n, m, P in [(1 << 20, 230_000_000, just_over),  # one chunk (2^10 tiles) too many
                    (1 << 26, 1 << 29, 64),             # 2^19 tiles
                    (1 << 36, 1 << 33, 1 << 16)]:       # 2^23 tiles
        assert kg.kg_gnm_directed_noalloc_scratch(n, m, P) > kg.NOALLOC_SCRATCH_BYTES
        st = L.kg_gnm_directed_noalloc(n, m, 1, P, 8, 0, m, status.data_ptr(), s)
        assert st == kg.KG_ERR_RANGE, (n, m, P)
    torch.cuda.synchronize()
    assert int(status.item()) == -7  # rejected synchronously: the status word is untouched
    st = L.kg_gnm_directed_noalloc(100, 50, 1, 4, 4, 0, 50, 0, s)  # no status word
    assert st == kg.KG_ERR_ARG
