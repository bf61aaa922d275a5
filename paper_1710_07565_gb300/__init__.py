"""GB300-native communication-free Erdos-Renyi generators (directed / undirected
G(n,m) and G(n,p)) -- Python binding of the C ABI in include/kg.h.

Every function named ``kg_*`` here is argument marshalling for the C entry
point of the same name in libkg.so: device pointers and streams are passed as
integers, the work runs in the CUDA kernels.  The convenience wrappers
(``gnm_directed`` ...) allocate the output with PyTorch (device memory only)
and call the same entry points.  There is no CPU path: if the library cannot
be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build_lib

KG_OK, KG_ERR_ARG, KG_ERR_RANGE, KG_ERR_CAPACITY, KG_ERR_CUDA, KG_ERR_TIMEOUT, KG_ERR_INTERNAL = range(7)
K_LEAF_DEFAULT = 1024
K_MAX_DEFAULT = 2048

_lock = threading.Lock()
_lib = None


class KGError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_str(status)} (status {status})")


def build(force: bool = False) -> str:
    """Compile libkg.so for sm_103a in-tree."""
    return _build_lib.build(force=force)


def lib_path() -> str:
    return _build_lib.LIB


def lib() -> ctypes.CDLL:
    """The loaded CUDA library (built on first use if the toolchain is present)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build_lib.LIB
            if not os.path.exists(path):
                path = _build_lib.build()
            L = ctypes.CDLL(path)
            u64, u32, i32, dbl, vp = (ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_void_p)
            sigs = {
                "kg_gnm_directed": [u64, u64, u64, u32, i32, vp, u64, vp],
                "kg_gnm_directed_ex": [u64, u64, u64, u32, u32, u32, i32, vp, u64, vp],
                "kg_gnm_directed_chunk_counts": [u64, u64, u64, u32, vp, vp],
                "kg_gnm_directed_range": [u64, u64, u64, u32, u32, u32, vp, i32, vp, u64, vp, vp, vp],
                "kg_gnm_undirected": [u64, u64, u64, u32, i32, vp, u64, vp],
                "kg_gnm_undirected_ex": [u64, u64, u64, u32, u32, u32, i32, vp, u64, vp],
                "kg_gnp_directed": [u64, dbl, u64, u32, i32, vp, u64, vp, vp],
                "kg_gnp_undirected": [u64, dbl, u64, u32, i32, vp, u64, vp, vp],
                "kg_gnp_ex": [i32, u64, dbl, u64, u32, u32, i32, vp, u64, vp, vp],
                "kg_gnp_binomial": [i32, u64, dbl, u64, u32, i32, vp, u64, vp, vp],
                "kg_gnm_undirected_chunk_counts": [u64, u64, u64, u32, vp, vp],
                "kg_gnm_undirected_rows": [u64, u64, u64, u32, u32, u32, vp, i32, vp, u64, vp, vp,
                                           vp, vp],
                "kg_gnp_binomial_count": [i32, u64, dbl, u64, u32, vp, vp],
                "kg_edge_digest": [vp, u64, i32, vp, vp],
                "kg_last_error": [vp],
                "kg_gnp_size": [i32, u64, dbl, u64, u32, vp, vp],
                "kg_rgg": [i32, u64, dbl, u64, i32, vp, u64, vp, vp, vp],
                "kg_rgg_count": [i32, u64, dbl, u64, vp, vp],
                "kg_rgg_cell_counts": [i32, u64, dbl, u64, vp, vp],
                "kg_rgg_grid": [i32, u64, dbl, ctypes.POINTER(ctypes.c_int)],
                "kg_shutdown": [],
                "kg_gnm_directed_noalloc": [u64, u64, u64, u32, i32, vp, u64, vp, vp],
                "kg_gnm_directed_noalloc_scratch": [u64, u64, u32, ctypes.POINTER(u64)],
                "kg_gnp_ex_slots": [i32, u64, dbl, u64, u32, u32, i32, i32, vp, u64, vp, vp],
                "kg_peak_store": [vp, u64, i32, vp],
                "kg_peak_fp64": [vp, u32, u32, vp],
            }
            for name, args in sigs.items():
                f = getattr(L, name, None)
                if f is None:
                    continue
                f.argtypes = args
                f.restype = ctypes.c_int
            L.kg_batch_create.argtypes = [vp, u32, i32, ctypes.POINTER(vp)]
            L.kg_batch_create.restype = ctypes.c_int
            L.kg_batch_entries.argtypes = [vp]
            L.kg_batch_entries.restype = u64
            L.kg_batch_offsets.argtypes = [vp, vp]
            L.kg_batch_offsets.restype = ctypes.c_int
            L.kg_batch_run.argtypes = [vp, vp, u64, vp]
            L.kg_batch_run.restype = ctypes.c_int
            L.kg_batch_tune.argtypes = [vp, vp, u64, i32, vp]
            L.kg_batch_tune.restype = ctypes.c_int
            L.kg_batch_get_tuning.argtypes = [vp, vp, vp]
            L.kg_batch_get_tuning.restype = ctypes.c_int
            L.kg_batch_destroy.argtypes = [vp]
            L.kg_batch_destroy.restype = ctypes.c_int
            L.kg_gnp_count.argtypes = [i32, u64, dbl, u64, u32, u32, vp, vp]
            L.kg_gnp_count.restype = ctypes.c_int
            L.kg_server_create.argtypes = [u64, u32, ctypes.POINTER(vp)]
            L.kg_server_create.restype = ctypes.c_int
            L.kg_server_submit.argtypes = [vp, vp, ctypes.POINTER(u64)]
            L.kg_server_submit.restype = ctypes.c_int
            L.kg_server_poll.argtypes = [vp, vp, u32, ctypes.POINTER(u32)]
            L.kg_server_poll.restype = ctypes.c_int
            L.kg_server_pending.argtypes = [vp, vp, vp, vp, vp]
            L.kg_server_pending.restype = ctypes.c_int
            L.kg_server_destroy.argtypes = [vp]
            L.kg_server_destroy.restype = ctypes.c_int
            L.kg_status_str.argtypes = [ctypes.c_int]
            L.kg_status_str.restype = ctypes.c_char_p
            L.kg_launch_count.argtypes = []
            L.kg_launch_count.restype = ctypes.c_ulonglong
            L.kg_profile_begin.argtypes = []
            L.kg_profile_begin.restype = ctypes.c_int
            L.kg_profile_end.argtypes = [ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_ulonglong)]
            L.kg_profile_end.restype = ctypes.c_int
            _lib = L
    return _lib


def status_str(status: int) -> str:
    try:
        return lib().kg_status_str(status).decode()
    except OSError:
        return f"status {status}"


def _call(name, *args):
    st = getattr(lib(), name)(*args)
    if st != KG_OK:
        raise KGError(st, name)
    return st


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------- raw entry points

def kg_gnm_directed(n, m, seed, chunks, id_bytes, d_out, cap_edges, stream):
    return _call("kg_gnm_directed", n, m, seed, chunks, id_bytes, d_out, cap_edges, stream)


def kg_gnm_directed_ex(n, m, seed, chunks, k_leaf, k_max, id_bytes, d_out, cap_edges, stream):
    return _call("kg_gnm_directed_ex", n, m, seed, chunks, k_leaf, k_max, id_bytes, d_out,
                 cap_edges, stream)


def kg_gnm_directed_chunk_counts(n, m, seed, chunks, d_counts, stream):
    return _call("kg_gnm_directed_chunk_counts", n, m, seed, chunks, d_counts, stream)


def kg_gnm_directed_range(n, m, seed, chunks, c_begin, c_end, d_counts, id_bytes, d_out,
                          cap_edges, d_chunk_digest, d_chunk_hist, stream):
    return _call("kg_gnm_directed_range", n, m, seed, chunks, c_begin, c_end, d_counts, id_bytes,
                 d_out, cap_edges, d_chunk_digest, d_chunk_hist, stream)


def kg_gnm_undirected(n, m, seed, chunks, id_bytes, d_out, cap_edges, stream):
    return _call("kg_gnm_undirected", n, m, seed, chunks, id_bytes, d_out, cap_edges, stream)


def kg_gnm_undirected_ex(n, m, seed, chunks, k_leaf, k_max, id_bytes, d_out, cap_edges, stream):
    return _call("kg_gnm_undirected_ex", n, m, seed, chunks, k_leaf, k_max, id_bytes, d_out,
                 cap_edges, stream)


def kg_gnp_directed(n, p, seed, chunks, id_bytes, d_out, cap_edges, d_count, stream):
    return _call("kg_gnp_directed", n, p, seed, chunks, id_bytes, d_out, cap_edges, d_count, stream)


def kg_gnp_undirected(n, p, seed, chunks, id_bytes, d_out, cap_edges, d_count, stream):
    return _call("kg_gnp_undirected", n, p, seed, chunks, id_bytes, d_out, cap_edges, d_count,
                 stream)


def kg_gnp_ex(undirected, n, p, seed, chunks, k_leaf, id_bytes, d_out, cap_edges, d_count, stream):
    return _call("kg_gnp_ex", int(undirected), n, p, seed, chunks, k_leaf, id_bytes, d_out,
                 cap_edges, d_count, stream)


def kg_gnp_ex_slots(undirected, n, p, seed, chunks, k_leaf, slots_per_tile, id_bytes, d_out,
                    cap_edges, d_count, stream):
    """kg_gnp_ex with the per-tile slot count set (a test hook: 0 walks every
    tile twice, a small count makes tiles overflow their slots)."""
    return _call("kg_gnp_ex_slots", int(undirected), n, p, seed, chunks, k_leaf, slots_per_tile,
                 id_bytes, d_out, cap_edges, d_count, stream)


def kg_gnm_undirected_chunk_counts(n, m, seed, chunks, d_counts, stream):
    return _call("kg_gnm_undirected_chunk_counts", n, m, seed, chunks, d_counts, stream)


def kg_gnm_undirected_rows(n, m, seed, chunks, b_begin, b_end, d_counts, id_bytes, d_out,
                           cap_edges, d_entries, d_block_digest, d_block_hist, stream):
    return _call("kg_gnm_undirected_rows", n, m, seed, chunks, b_begin, b_end, d_counts, id_bytes,
                 d_out, cap_edges, d_entries, d_block_digest, d_block_hist, stream)


def kg_gnp_binomial(undirected, n, p, seed, chunks, id_bytes, d_out, cap_edges, d_count, stream):
    return _call("kg_gnp_binomial", int(undirected), n, p, seed, chunks, id_bytes, d_out,
                 cap_edges, d_count, stream)


def kg_gnp_binomial_count(undirected, n, p, seed, chunks, d_count, stream):
    return _call("kg_gnp_binomial_count", int(undirected), n, p, seed, chunks, d_count, stream)


def kg_gnm_directed_noalloc(n, m, seed, chunks, id_bytes, d_out, cap_edges, d_status, stream):
    """Directed G(n,m) that allocates nothing: scratch is a fixed array inside
    the library (see include/kg.h for the size limit and the sharing rules)."""
    return _call("kg_gnm_directed_noalloc", n, m, seed, chunks, id_bytes, d_out, cap_edges,
                 d_status, stream)


def kg_gnm_directed_noalloc_scratch(n, m, chunks) -> int:
    """Bytes of the library's fixed array that kg_gnm_directed_noalloc would
    use for (n, m, chunks) (host only)."""
    b = ctypes.c_uint64(0)
    _call("kg_gnm_directed_noalloc_scratch", n, m, chunks, ctypes.byref(b))
    return b.value


NOALLOC_SCRATCH_BYTES = 32 << 20  # KG_NOALLOC_SCRATCH_BYTES of include/kg.h


def kg_peak_store(d_buf, nbytes, mode, stream):
    return _call("kg_peak_store", d_buf, nbytes, mode, stream)


def kg_peak_fp64(d_out, blocks, iters, stream):
    return _call("kg_peak_fp64", d_out, blocks, iters, stream)


def kg_edge_digest(d_edges, count, id_bytes, d_digest, stream):
    return _call("kg_edge_digest", d_edges, count, id_bytes, d_digest, stream)


def kg_last_error(stream) -> int:
    return lib().kg_last_error(stream)


PROF_CLASSES = ("chunk_tree", "tile_tree", "scan", "leaf", "digest", "gnp_tile", "assembly", "other",
                "rgg")


def kg_launch_count() -> int:
    return lib().kg_launch_count()


def kg_profile_begin():
    return _call("kg_profile_begin")


def kg_profile_end():
    """{class: (milliseconds, launches)} of the launches since kg_profile_begin."""
    ms = (ctypes.c_double * len(PROF_CLASSES))()
    n = (ctypes.c_ulonglong * len(PROF_CLASSES))()
    st = lib().kg_profile_end(ms, n)
    if st != KG_OK:
        raise KGError(st, "kg_profile_end")
    return {c: (ms[i], n[i]) for i, c in enumerate(PROF_CLASSES)}


class kg_instance(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("m", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("chunks", ctypes.c_uint32), ("undirected", ctypes.c_int32)]


def kg_batch_create(instances, id_bytes=4):
    """instances: sequence of dicts with n, m, seed, chunks, undirected.  Returns a handle."""
    arr = (kg_instance * max(len(instances), 1))()
    for i, q in enumerate(instances):
        arr[i] = kg_instance(q["n"], q["m"], q["seed"], q["chunks"], 1 if q["undirected"] else 0)
    h = ctypes.c_void_p()
    _call("kg_batch_create", ctypes.cast(arr, ctypes.c_void_p), len(instances), id_bytes,
          ctypes.byref(h))
    return h


def kg_batch_entries(h) -> int:
    return lib().kg_batch_entries(h)


def kg_batch_offsets(h, count):
    import numpy as np
    off = np.zeros(count + 1, dtype=np.uint64)
    _call("kg_batch_offsets", h, off.ctypes.data_as(ctypes.c_void_p))
    return off


def kg_batch_run(h, d_out, cap_entries, stream):
    return _call("kg_batch_run", h, d_out, cap_entries, stream)


def kg_batch_tune(h, d_out, cap_entries, reps, stream):
    return _call("kg_batch_tune", h, d_out, cap_entries, reps, stream)


def kg_batch_get_tuning(h):
    a, b = ctypes.c_uint32(), ctypes.c_uint32()
    _call("kg_batch_get_tuning", h, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def kg_batch_destroy(h):
    return _call("kg_batch_destroy", h)


def kg_gnp_count(undirected, n, p, seed, chunks, k_leaf, d_count, stream):
    return _call("kg_gnp_count", int(undirected), n, p, seed, chunks, k_leaf, d_count, stream)


def kg_gnp_size(undirected, n, p, seed, chunks, d_count, stream):
    return _call("kg_gnp_size", int(undirected), n, p, seed, chunks, d_count, stream)


def kg_rgg(dim, n, r, seed, id_bytes, d_out, cap_entries, d_count, d_coords, stream):
    return _call("kg_rgg", dim, n, r, seed, id_bytes, d_out, cap_entries, d_count, d_coords,
                 stream)


def kg_rgg_count(dim, n, r, seed, d_count, stream):
    return _call("kg_rgg_count", dim, n, r, seed, d_count, stream)


def kg_rgg_cell_counts(dim, n, r, seed, d_counts, stream):
    return _call("kg_rgg_cell_counts", dim, n, r, seed, d_counts, stream)


def rgg_grid(dim, n, r) -> int:
    """g of the 2^g-per-dimension cell grid of RGG(n, r) (Sec. 5)."""
    g = ctypes.c_int()
    _call("kg_rgg_grid", dim, n, r, ctypes.byref(g))
    return g.value


def rgg_cell_counts(dim, n, r, seed=1, stream=None, device="cuda"):
    """Points per cell (row-major cells) as an int64 tensor."""
    import torch
    out = torch.zeros(1 << (dim * rgg_grid(dim, n, r)), dtype=torch.int64, device=device)
    kg_rgg_cell_counts(dim, n, r, seed, out.data_ptr(), _stream_ptr(stream))
    return out


def rgg(dim, n, r, seed=1, id_bytes=4, coords=False, stream=None, device="cuda"):
    """RGG(n, r) (Sec. 5): the (entries, 2) tensor of both directions sorted by
    (u, v), sized exactly by a count pass first; with coords=True also the
    (n, dim) int32 tensor holding the uint32 fixed-point coordinates."""
    import torch
    s = _stream_ptr(stream)
    cnt = torch.zeros(1, dtype=torch.int64, device=device)
    kg_rgg_count(dim, n, r, seed, cnt.data_ptr(), s)
    k = int(cnt.item())
    out = _empty_edges(max(k, 1), id_bytes, device)
    xy = torch.zeros((max(n, 1), dim), dtype=torch.int32, device=device) if coords else None
    kg_rgg(dim, n, r, seed, id_bytes, out.data_ptr(), k, cnt.data_ptr(),
           xy.data_ptr() if coords else None, s)
    if coords:
        return out[:k], xy[:n]
    return out[:k]


def kg_shutdown():
    return _call("kg_shutdown")


# request models: G(n,m); G(n,p) by geometric skips; G(n,p) by binomial chunk counts
_MODELS = {"gnm": 0, "gnp": 1, "gnp_binomial": 2}


class kg_request(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("undirected", ctypes.c_int32), ("n", ctypes.c_uint64),
                ("m", ctypes.c_uint64), ("p", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("chunks", ctypes.c_uint32), ("id_bytes", ctypes.c_int32)]


class kg_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("entries", ctypes.c_uint64), ("digest", ctypes.c_uint64),
                ("t_submit_ms", ctypes.c_double), ("t_admit_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double), ("status", ctypes.c_int32), ("pad", ctypes.c_int32)]


def kg_server_create(budget_bytes, streams):
    h = ctypes.c_void_p()
    _call("kg_server_create", budget_bytes, streams, ctypes.byref(h))
    return h


def kg_server_submit(h, req: dict, id_bytes=4) -> int:
    r = kg_request(_MODELS[req["model"]], 1 if req["undirected"] else 0, req["n"],
                   req.get("m", 0), req.get("p", 0.0), req["seed"], req["chunks"], id_bytes)
    out = ctypes.c_uint64()
    _call("kg_server_submit", h, ctypes.byref(r), ctypes.byref(out))
    return out.value


def kg_server_poll(h, max_results=4096):
    buf = (kg_result * max_results)()
    n = ctypes.c_uint32()
    _call("kg_server_poll", h, ctypes.cast(buf, ctypes.c_void_p), max_results, ctypes.byref(n))
    return [{"id": buf[i].id, "entries": buf[i].entries, "digest": buf[i].digest,
             "t_submit_ms": buf[i].t_submit_ms, "t_admit_ms": buf[i].t_admit_ms,
             "t_done_ms": buf[i].t_done_ms, "status": buf[i].status} for i in range(n.value)]


def kg_server_pending(h):
    a, b, c, d = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint64()
    _call("kg_server_pending", h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d))
    return {"sizing": a.value, "waiting": b.value, "running": c.value, "bytes_in_use": d.value}


def kg_server_destroy(h):
    return _call("kg_server_destroy", h)


def serve(requests, budget_bytes, streams=8, id_bytes=4, realtime=True, clock=None, server=None):
    """Drive a server over `requests` (dicts with an 'arrival' time in seconds):
    submit each at its arrival (realtime) or all at once, poll until all are
    done.  Returns the per-request results (by id order of submission).  With
    `server` (a kg_server_create handle) that server is used and kept;
    otherwise one is created for the call and destroyed after it."""
    import time
    h = server if server is not None else kg_server_create(budget_bytes, streams)
    results = {}
    try:
        t0 = time.perf_counter()
        i = 0
        idmap = {}
        while len(results) < len(requests):
            now = time.perf_counter() - t0
            while i < len(requests) and (not realtime or requests[i]["arrival"] <= now):
                idmap[kg_server_submit(h, requests[i], id_bytes)] = i
                i += 1
            for r in kg_server_poll(h):
                results[idmap[r["id"]]] = r
            if i < len(requests) and realtime:
                time.sleep(0)
    finally:
        if server is None:
            kg_server_destroy(h)
    return [results[k] for k in range(len(requests))]


# ---------------------------------------------------------------- torch helpers

def _empty_edges(count, id_bytes, device):
    import torch
    dt = torch.int32 if id_bytes == 4 else torch.int64
    return torch.empty((max(count, 1), 2), dtype=dt, device=device)


def check_device_error(stream=None):
    st = kg_last_error(_stream_ptr(stream))
    if st != KG_OK:
        raise KGError(st, "device")


def gnm_directed(n, m, seed=1, chunks=1, id_bytes=4, k_leaf=K_LEAF_DEFAULT, k_max=K_MAX_DEFAULT,
                 out=None, stream=None, device="cuda"):
    """Directed G(n,m) as an (m, 2) int32/int64 tensor of (u, v) (int32 holds uint32 bits)."""
    if out is None:
        out = _empty_edges(m, id_bytes, device)
    kg_gnm_directed_ex(n, m, seed, chunks, k_leaf, k_max, id_bytes, out.data_ptr(), m,
                       _stream_ptr(stream))
    return out[:m]


def gnm_undirected(n, m, seed=1, chunks=1, id_bytes=4, k_leaf=K_LEAF_DEFAULT, k_max=K_MAX_DEFAULT,
                   out=None, stream=None, device="cuda"):
    """Undirected G(n,m) as a (2m, 2) tensor: both directions, sorted by (u, v)."""
    if out is None:
        out = _empty_edges(2 * m, id_bytes, device)
    kg_gnm_undirected_ex(n, m, seed, chunks, k_leaf, k_max, id_bytes, out.data_ptr(), 2 * m,
                         _stream_ptr(stream))
    return out[:2 * m]


def gnp(undirected, n, p, seed=1, chunks=1, id_bytes=4, k_leaf=K_LEAF_DEFAULT, cap=None,
        stream=None, device="cuda", slots_per_tile=-1):
    """G(n,p) edge list; returns (edges tensor view, device count tensor).
    slots_per_tile >= 0 sets the skip walk's per-tile slot count
    (kg_gnp_ex_slots); the output does not depend on it."""
    import torch
    if cap is None:
        pairs = n * (n - 1) // (2 if undirected else 1)
        mean = pairs * p
        cap = int(min(pairs, mean + 12 * (mean ** 0.5) + 64)) * (2 if undirected else 1)
    out = _empty_edges(cap, id_bytes, device)
    cnt = torch.zeros(1, dtype=torch.int64, device=device)
    kg_gnp_ex_slots(undirected, n, p, seed, chunks, k_leaf, slots_per_tile, id_bytes,
                    out.data_ptr(), cap, cnt.data_ptr(), _stream_ptr(stream))
    return out, cnt


def gnp_binomial(undirected, n, p, seed=1, chunks=1, id_bytes=4, stream=None, device="cuda"):
    """G(n,p) by binomial chunk counts (Sec. 4.3): sized exactly first, then
    generated; returns the edges tensor."""
    import torch
    s = _stream_ptr(stream)
    cnt = torch.zeros(1, dtype=torch.int64, device=device)
    kg_gnp_binomial_count(undirected, n, p, seed, chunks, cnt.data_ptr(), s)
    k = int(cnt.item())
    out = _empty_edges(max(k, 1), id_bytes, device)
    kg_gnp_binomial(undirected, n, p, seed, chunks, id_bytes, out.data_ptr(), k, cnt.data_ptr(), s)
    return out[:k]
