"""Serving loop: requests admitted by exact output bytes against a budget,
overlapping on several streams; each result must be the same alone and in
the mix (integer digests: equal, tolerance zero)."""
import numpy as np
import pytest

from gpu_util import need_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kg():
    need_cuda()
    import paper_1710_07565_gb300 as kg
    kg.lib()
    return kg


def _small_requests(count, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(2 ** rng.uniform(8, 16))
        d = float(rng.uniform(4, 32))
        kind = int(rng.integers(0, 6))
        und = kind in (1, 3, 5)
        model = "gnm" if kind < 2 else ("gnp" if kind < 4 else "gnp_binomial")
        req = {"n": n, "seed": 100 + i, "undirected": und, "model": model,
               "chunks": int(min(n, 1 + rng.integers(0, 16))), "arrival": 0.0}
        if model == "gnm":
            pairs = n * (n - 1) // (2 if und else 1)
            req["m"] = min(pairs, int(d * n / (2 if und else 1)))
        else:
            req["p"] = d / (n - 1)
        out.append(req)
    return out


def _alone(kg, req):
    """The request generated by itself through the plain entry points."""
    import torch
    s = kg._stream_ptr(None)
    dig = torch.zeros(1, dtype=torch.int64, device="cuda")
    if req["model"] == "gnm":
        k = 2 * req["m"] if req["undirected"] else req["m"]
        out = torch.empty((max(k, 1), 2), dtype=torch.int32, device="cuda")
        f = kg.kg_gnm_undirected if req["undirected"] else kg.kg_gnm_directed
        f(req["n"], req["m"], req["seed"], req["chunks"], 4, out.data_ptr(), k, s)
    elif req["model"] == "gnp_binomial":
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        kg.kg_gnp_binomial_count(req["undirected"], req["n"], req["p"], req["seed"], req["chunks"],
                                 cnt.data_ptr(), s)
        k = int(cnt.item())
        out = torch.empty((max(k, 1), 2), dtype=torch.int32, device="cuda")
        kg.kg_gnp_binomial(req["undirected"], req["n"], req["p"], req["seed"], req["chunks"], 4,
                           out.data_ptr(), k, cnt.data_ptr(), s)
        assert int(cnt.item()) == k
    else:
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        kg.kg_gnp_count(req["undirected"], req["n"], req["p"], req["seed"], req["chunks"], 1024,
                        cnt.data_ptr(), s)
        k = int(cnt.item())
        out = torch.empty((max(k, 1), 2), dtype=torch.int32, device="cuda")
        kg.kg_gnp_ex(req["undirected"], req["n"], req["p"], req["seed"], req["chunks"], 1024, 4,
                     out.data_ptr(), k, cnt.data_ptr(), s)
        assert int(cnt.item()) == k
    kg.kg_edge_digest(out.data_ptr(), k, 4, dig.data_ptr(), s)
    kg.check_device_error()
    return k, int(dig.cpu().numpy().view(np.uint64)[0])


def test_alone_equals_in_mix_under_a_tight_budget(kg):
    """200 requests served together under a budget far below their total
    output, each equal (entry count and digest) to the same request alone."""
    reqs = _small_requests(200)
    sizes = [_alone(kg, r) for r in reqs]
    biggest = max(k for k, _ in sizes) * 8
    budget = max(biggest * 3, 1 << 20)            # far below the total: admission must wait
    assert budget < sum(k for k, _ in sizes) * 8
    res = kg.serve(reqs, budget, streams=4, realtime=False)
    kg.check_device_error()
    for r, (k, dig), got in zip(reqs, sizes, res):
        assert got["status"] == kg.KG_OK
        assert got["entries"] == k, r
        assert got["digest"] == dig, r
        assert got["t_submit_ms"] <= got["t_admit_ms"] <= got["t_done_ms"]


def test_request_larger_than_budget_is_refused(kg):
    req = {"n": 5000, "m": 200000, "seed": 1, "undirected": False, "model": "gnm", "chunks": 4,
           "arrival": 0.0}
    res = kg.serve([req], 1 << 20, streams=2, realtime=False)  # 1.6 MB of output > 1 MiB
    assert res[0]["status"] == kg.KG_ERR_CAPACITY


def test_realtime_poisson_arrivals(kg):
    from paper_1710_07565_gb300 import workloads
    reqs = [r for r in workloads.serving_requests(400, 400.0) if r["n"] <= 1 << 18][:40]
    res = kg.serve(reqs, 8 << 30, streams=8, realtime=True)
    kg.check_device_error()
    assert all(r["status"] == kg.KG_OK for r in res)
    # in-order submission times follow the arrivals
    sub = [r["t_submit_ms"] for r in res]
    assert sub == sorted(sub)
    for req, got in zip(reqs[:10], res[:10]):
        k, dig = _alone(kg, req)
        assert (got["entries"], got["digest"]) == (k, dig)
