#!/usr/bin/env python3
"""Benchmark: directed G(n,m) at scale (Sec. 4.1 of the paper) on GB300.

Workload (one step): n = 2^36 vertices, m = 2^33 edges, P = 2^16 chunks,
seed 1, uint64 ids (16 B per edge).  The chunk split tree gives every chunk
its count; the edges are then generated in 16 slabs of 4096 chunks (about
2^29 edges = 8 GiB each) into one device slab buffer, and every slab is
reduced on the device, inside the same kernel, to a per-chunk order-
independent 64-bit digest and out-degree histogram.  128 GiB of edges are
written per step, far more than L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_VERT, M_EDGES, P_CHUNKS, SEED = 1 << 36, 1 << 33, 1 << 16, 1
SLABS = 16
CHUNKS_PER_SLAB = P_CHUNKS // SLABS
SLAB_CAP = (1 << 29) + (1 << 21)  # edges per slab buffer (mean 2^29, sd ~2^14.5)
ID_BYTES = 8
WORKLOAD = "directed G(n,m): n=2^36, m=2^33, 2^16 chunks, uint64 ids, 16 slabs of 8 GiB, per-chunk digest + out-degree histogram"
METRIC = "edges/s (directed G(n,m), n=2^36, m=2^33, 2^16 chunks, uint64 ids, on-device digest)"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "out", "").splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(seconds=10.0, min_chunks=16):
    """The oracle, single-threaded, on a bounded sample: whole chunks of the
    workload (chunk tree + chunk edges + digest + histogram), until ~seconds."""
    import oracle
    t0 = time.perf_counter()
    cnt = oracle.gnm_directed_chunk_counts(N_VERT, M_EDGES, SEED, P_CHUNKS)
    edges, chunks = 0, 0
    while chunks < min_chunks or time.perf_counter() - t0 < seconds:
        c = (chunks * 7919) % P_CHUNKS
        u, v = oracle.gnm_directed_chunk(N_VERT, M_EDGES, SEED, P_CHUNKS, c, int(cnt[c]))
        oracle.edge_checksum(u, v)
        oracle.outdegree_hist(u, c * N_VERT // P_CHUNKS, (c + 1) * N_VERT // P_CHUNKS)
        edges += len(u)
        chunks += 1
    dt = time.perf_counter() - t0
    return {"value": edges / dt, "unit": "edges/s", "cores": 1, "kind": "oracle",
            "sample": f"chunk split tree of all 2^16 chunks + {chunks} whole chunks "
                      f"({edges} edges) with digest and histogram, {dt:.1f} s single-threaded"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    steps = []
    for _ in range(args.warmup):
        cpu_baseline(seconds=2.0, min_chunks=4)
    for _ in range(args.steps):
        steps.append(cpu_baseline(seconds=args.ref_seconds, min_chunks=8))
    val = statistics.median(s["value"] for s in steps)
    cb = dict(steps[-1])
    cb["value"] = val
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "edges/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": M_EDGES / val * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": cb, "e2e": {"value": val, "unit": "edges/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kg", choices=["kg", "reference"])
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist

    import paper_1710_07565_gb300 as kg

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    seed = SEED + rank  # independent replicas (weak scaling, no data-path collective)
    dev = torch.device("cuda", local)
    s = torch.cuda.current_stream().cuda_stream
    buf = torch.empty((SLAB_CAP, 2), dtype=torch.int64, device=dev)
    counts = torch.zeros(P_CHUNKS, dtype=torch.int64, device=dev)
    digest = torch.zeros(P_CHUNKS, dtype=torch.int64, device=dev)
    hist = torch.zeros((P_CHUNKS, 65), dtype=torch.int64, device=dev)

    def step():
        kg.kg_gnm_directed_chunk_counts(N_VERT, M_EDGES, seed, P_CHUNKS, counts.data_ptr(), s)
        for i in range(SLABS):
            c0 = i * CHUNKS_PER_SLAB
            kg.kg_gnm_directed_range(N_VERT, M_EDGES, seed, P_CHUNKS, c0, c0 + CHUNKS_PER_SLAB,
                                     counts.data_ptr(), ID_BYTES, buf.data_ptr(), SLAB_CAP,
                                     digest.data_ptr() + 8 * c0, hist.data_ptr() + 8 * 65 * c0, s)

    # warm-up
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    kg.check_device_error()

    # timed region: CUDA events on the launching stream, per-kernel events on
    # the same stream through the library's profiling hook
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches0 = kg.kg_launch_count()
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        kg.kg_profile_begin()
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        barrier()
        prof = kg.kg_profile_end()
    launches = kg.kg_launch_count() - launches0
    ms = e0.elapsed_time(e1)
    kg.check_device_error()
    # sanity of the last step: exact counts, every vertex in one histogram bin
    tot = int(counts.sum())
    rows = N_VERT // P_CHUNKS
    if tot != M_EDGES or int(hist[:16].sum()) != 16 * rows:
        raise RuntimeError("inconsistent chunk counts or histogram")
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # end to end through the public entry points with host result buffers:
    # per step the per-chunk digests and histograms go to pinned host memory
    h_dig = torch.empty(P_CHUNKS, dtype=torch.int64, pin_memory=True)
    h_hist = torch.empty((P_CHUNKS, 65), dtype=torch.int64, pin_memory=True)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
        h_dig.copy_(digest, non_blocking=True)
        h_hist.copy_(hist, non_blocking=True)
        kg.check_device_error()  # synchronises the stream
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())

    total_edges = M_EDGES * args.steps * world
    value = total_edges / (ms / 1e3)
    e2e = total_edges / e2e_s
    peak, peak_kind = peaks()
    leaf_ms, leaf_n = prof["leaf"]
    per_launch_s = leaf_ms / 1e3 / max(leaf_n, 1)
    bytes_per_launch = M_EDGES * 16 / SLABS  # algorithmic: the edges written by one slab launch
    achieved = bytes_per_launch / per_launch_s / 1e9
    clocks = clk.summary()

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_VERT, "m": M_EDGES, "chunks": P_CHUNKS,
                   "slabs": SLABS, "id_bytes": ID_BYTES,
                   "l2": "no flush: 128 GiB of output per step, far above the 129 MB L2"},
        "write_GBps": M_EDGES * 16 * args.steps / (ms / 1e3) / 1e9,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "leaf_fast_kernel (Floyd draws, shared-memory sort, emit, digest)",
                     "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"},
        "kernel_ms": {k: round(v[0] / args.steps, 4) for k, v in prof.items() if v[1]},
        "kernel_launches_per_step": {k: v[1] // args.steps for k, v in prof.items() if v[1]},
        "e2e": {"value": e2e, "unit": "edges/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": P_CHUNKS * 8 * 66},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(seconds=args.ref_seconds)
        line["cpu_baseline"]["vs_value"] = value / line["cpu_baseline"]["value"]
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
