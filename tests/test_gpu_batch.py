"""Batched G(n,m): one launch sequence for many instances must write exactly
what the per-instance entry points write, instance after instance."""
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


def _sequential(kg, insts, total):
    import torch
    out = torch.empty((total, 2), dtype=torch.int32, device="cuda")
    s = kg._stream_ptr(None)
    pos = 0
    for q in insts:
        k = 2 * q["m"] if q["undirected"] else q["m"]
        view = out[pos:pos + k]
        if q["undirected"]:
            kg.kg_gnm_undirected(q["n"], q["m"], q["seed"], q["chunks"], 4, view.data_ptr(), k, s)
        else:
            kg.kg_gnm_directed(q["n"], q["m"], q["seed"], q["chunks"], 4, view.data_ptr(), k, s)
        pos += k
    kg.check_device_error()
    return out


MIXED = [
    {"n": 5, "m": 4, "seed": 1, "chunks": 5, "undirected": True},
    {"n": 300, "m": 44850, "seed": 2, "chunks": 7, "undirected": True},     # complete graph
    {"n": 1000, "m": 500000, "seed": 3, "chunks": 13, "undirected": False},  # density 1/2
    {"n": 2, "m": 2, "seed": 4, "chunks": 2, "undirected": False},
    {"n": 70000, "m": 1 << 20, "seed": 5, "chunks": 64, "undirected": False},
    {"n": 50000, "m": 400000, "seed": 6, "chunks": 32, "undirected": True},
    {"n": 12345, "m": 0, "seed": 7, "chunks": 3, "undirected": True},
    {"n": 12345, "m": 77777, "seed": 8, "chunks": 1, "undirected": False},
    {"n": 9000, "m": 9000 * 8999 // 4, "seed": 9, "chunks": 3, "undirected": True},  # long rows
]


def test_batch_matches_per_instance_calls_and_oracle(kg, orc):
    import torch
    h = kg.kg_batch_create(MIXED)
    try:
        total = kg.kg_batch_entries(h)
        off = kg.kg_batch_offsets(h, len(MIXED))
        out = torch.zeros((total, 2), dtype=torch.int32, device="cuda")
        kg.kg_batch_run(h, out.data_ptr(), total, kg._stream_ptr(None))
        kg.check_device_error()
        seq = _sequential(kg, MIXED, total)
        assert torch.equal(out, seq)
        for i in (0, 1, 2, 5, 7):
            q = MIXED[i]
            u, v = edges_np(out[int(off[i]):int(off[i + 1])], 4)
            if q["undirected"]:
                ou, ov = orc.gnm_undirected(q["n"], q["m"], q["seed"], q["chunks"])
            else:
                ou, ov = orc.gnm_directed(q["n"], q["m"], q["seed"], q["chunks"])
            assert_same_edges(u, v, ou, ov, f"instance {i}")
    finally:
        kg.kg_batch_destroy(h)


def test_batch_of_generated_instances_graph_replay_and_tuning(kg):
    """256 instances of the batched workload (n log-uniform in [2^8, 2^20],
    degree in [2, 64], directed/undirected): captured in a CUDA graph and
    replayed, then tuned; every run equals the per-instance calls."""
    import torch
    from paper_1710_07565_gb300 import workloads
    insts = workloads.batched_instances(4096)[:256]
    h = kg.kg_batch_create(insts)
    try:
        total = kg.kg_batch_entries(h)
        seq = _sequential(kg, insts, total)
        out = torch.zeros((total, 2), dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        # first call on this stream outside capture (library set-up)
        kg.kg_batch_run(h, out.data_ptr(), total, s.cuda_stream)
        s.synchronize()
        assert torch.equal(out, seq)
        out.zero_()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            kg.kg_batch_run(h, out.data_ptr(), total, s.cuda_stream)
        g.replay()
        torch.cuda.synchronize()
        kg.check_device_error()
        assert torch.equal(out, seq)
        out.zero_()
        kg.kg_batch_tune(h, out.data_ptr(), total, 1, kg._stream_ptr(None))
        out.zero_()
        kg.kg_batch_run(h, out.data_ptr(), total, kg._stream_ptr(None))
        kg.check_device_error()
        assert torch.equal(out, seq)
    finally:
        kg.kg_batch_destroy(h)


def test_batch_argument_errors(kg):
    L = kg.lib()
    import ctypes
    bad = [{"n": 10, "m": 91, "seed": 1, "chunks": 2, "undirected": False}]
    with pytest.raises(kg.KGError):
        kg.kg_batch_create(bad)
    with pytest.raises(kg.KGError):
        kg.kg_batch_create([{"n": 100, "m": 10, "seed": 1, "chunks": 65, "undirected": False}])
    h = kg.kg_batch_create([{"n": 100, "m": 10, "seed": 1, "chunks": 4, "undirected": False}])
    try:
        assert L.kg_batch_run(h, 0, 5, kg._stream_ptr(None)) == kg.KG_ERR_CAPACITY
    finally:
        kg.kg_batch_destroy(h)


def test_tuning_is_cached_by_size_class(kg):
    """A second batch of the same size class on the same GPU takes the first
    one's tuned launch shapes without timing (its output unchanged), and every
    tiles-per-CTA choice writes the same bytes."""
    import time
    import torch
    from paper_1710_07565_gb300 import workloads
    insts = workloads.batched_instances(4096)[256:384]
    h1 = kg.kg_batch_create(insts)
    h2 = kg.kg_batch_create(insts)
    try:
        total = kg.kg_batch_entries(h1)
        seq = _sequential(kg, insts, total)
        out = torch.zeros((total, 2), dtype=torch.int32, device="cuda")
        s = kg._stream_ptr(None)
        kg.kg_batch_tune(h1, out.data_ptr(), total, 1, s)
        t0 = time.perf_counter()
        kg.kg_batch_tune(h2, out.data_ptr(), total, 1, s)
        t_cached = time.perf_counter() - t0
        assert kg.kg_batch_get_tuning(h1) == kg.kg_batch_get_tuning(h2)
        assert t_cached < 0.05  # no timing runs
        out.zero_()
        kg.kg_batch_run(h2, out.data_ptr(), total, s)
        kg.check_device_error()
        assert torch.equal(out, seq)
        tt, pc = kg.kg_batch_get_tuning(h1)
        assert tt in (64, 128, 256) and pc in (1, 2, 4, 8, 16)
    finally:
        kg.kg_batch_destroy(h1)
        kg.kg_batch_destroy(h2)
