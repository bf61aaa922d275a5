"""Multi-process replicas on CPU (gloo, world size 2): the benchmark's ranks
run independent replicas of the workload (distinct seeds, no data exchange),
the timed region is the slowest rank's, and the reported value is the units
of all ranks over that time.  The generator itself needs no collective: a
replica's chunk counts depend only on its own seed."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        seed = bench.replica_seed(rank)
        # each rank's own replica: the full chunk split tree of a small instance
        cnt = oracle.gnm_directed_chunk_counts(1 << 20, 1 << 22, seed, 64)
        ms = 100.0 + 50.0 * rank  # stand-in for the rank's measured time
        ms_max = bench.max_over_ranks(ms, torch.device("cpu"), world)
        rate = bench.aggregate_rate(1 << 22, 3, world, ms_max / 1e3)
        q.put((rank, seed, int(sum(int(c) for c in cnt)), [int(c) for c in cnt[:4]], ms_max, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    (r0, s0, m0, c0, t0, v0), (r1, s1, m1, c1, t1, v1) = res
    assert (r0, r1) == (0, 1)
    assert s0 != s1                       # independent replicas
    assert m0 == m1 == 1 << 22            # each replica holds exactly m edges
    assert c0 != c1                       # ... drawn from different streams
    assert t0 == t1 == 150.0              # the slowest rank's time on every rank
    assert v0 == v1 == pytest.approx((1 << 22) * 3 * 2 / 0.150)
