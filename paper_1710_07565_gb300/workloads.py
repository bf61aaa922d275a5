"""Seeded synthetic workloads (instance lists only; no sampling arithmetic).

Used by the tests and by bench.py; the random draws that pick instance sizes
come from numpy's Philox generator with a fixed key.

batched_instances(): 4096 independent G(n,m) instances, n log-uniform in
    [2^8, 2^20], average degree uniform in [2, 64], directed / undirected
    50/50, seed = instance index.  m = round(d n) for directed, round(d n / 2)
    for undirected instances; the chunk count is the largest power of two
    <= m / 2^16, clamped to [1, min(64, n)] (directed) or [1, min(32, n)].
serving_requests(): a Poisson stream of requests mixing directed /
    undirected G(n,m) and G(n,p), n log-uniform in [2^10, 2^26], average
    degree uniform in [4, 32]; G(n,p) requests use the sampler named by
    gnp_model ("gnp_binomial": binomial chunk counts, "gnp": geometric skips).
"""
from __future__ import annotations

import math

import numpy as np

KEY_BATCH = 0x5EED
KEY_SERVE = 0x5E4E


def _chunks(m: int, n: int, cap: int) -> int:
    p = 1
    while p * 2 <= m / 2 ** 16:
        p *= 2
    return max(1, min(p, cap, n))


def batched_instances(count: int = 4096, key: int = KEY_BATCH):
    rng = np.random.Generator(np.random.Philox(key=key))
    out = []
    for i in range(count):
        u_n, u_d, u_kind = rng.random(3)
        n = int(round(2.0 ** (8 + 12 * u_n)))
        d = 2 + 62 * u_d
        undirected = bool(u_kind >= 0.5)
        if undirected:
            m = int(round(d * n / 2))
            m = min(m, n * (n - 1) // 2)
            P = _chunks(m, n, 32)
        else:
            m = int(round(d * n))
            m = min(m, n * (n - 1))
            P = _chunks(m, n, 64)
        out.append({"n": n, "m": m, "seed": i, "chunks": P, "undirected": undirected})
    return out


def instance_entries(inst) -> int:
    return 2 * inst["m"] if inst["undirected"] else inst["m"]


def serving_requests(count: int, rate_per_s: float, key: int = KEY_SERVE,
                     gnp_model: str = "gnp_binomial"):
    """Requests with Poisson arrival times (seconds from 0)."""
    rng = np.random.Generator(np.random.Philox(key=key))
    t = 0.0
    out = []
    for i in range(count):
        u_gap, u_n, u_d, u_kind = rng.random(4)
        t += -math.log(1.0 - u_gap) / rate_per_s
        n = int(round(2.0 ** (10 + 16 * u_n)))
        d = 4 + 28 * u_d
        kind = int(u_kind * 4)  # 0 gnm dir, 1 gnm und, 2 gnp dir, 3 gnp und
        und = kind in (1, 3)
        req = {"id": i, "arrival": t, "n": n, "seed": 1000 + i, "undirected": und,
               "model": "gnm" if kind < 2 else gnp_model}
        if kind < 2:
            req["m"] = int(round(d * n / 2)) if und else int(round(d * n))
        else:
            req["p"] = (d / (n - 1)) if n > 1 else 0.0
        cap = 32 if und else 64
        req["chunks"] = _chunks(req.get("m", int(d * n)), n, cap)
        out.append(req)
    return out
