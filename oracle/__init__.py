"""CPU oracle for the communication-free Erdos-Renyi generators.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package; the product path (``paper_1710_07565_gb300``) never does.

The oracle is plain single-threaded C (``oracle/*.c``) compiled with
``-O2 -ffp-contract=off`` and loaded through ctypes.  It restates the sampling
procedure of the paper (Sec. 2.2, 4.1, 4.2, 4.3) step by step and shares no
code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["or_rng.c", "or_math.c", "or_variates.c", "or_er.c", "or_rgg.c"]
_lock = threading.Lock()
_lib = None

# Defaults of the procedure's leaf parameters (expected samples per leaf and
# the count above which a leaf is split once more).
K_LEAF = 1024
K_MAX = 2048

ERR_NAMES = {0: "ok", 1: "bad argument", 2: "out of range", 3: "capacity", 6: "internal"}


class OracleError(RuntimeError):
    def __init__(self, rc, what):
        super().__init__(f"oracle {what}: {ERR_NAMES.get(rc, rc)} (code {rc})")
        self.rc = rc


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, no fused multiply-add)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    hdrs = [os.path.join(_HERE, h) for h in ("oracle.h", "or_internal.h")]
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(f) <= t for f in srcs + hdrs):
            return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-Wall", "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    """Load (building if needed) the oracle shared library."""
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u64, u32, dbl, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_int
            p64 = ctypes.POINTER(ctypes.c_uint64)
            p32 = ctypes.POINTER(ctypes.c_uint32)
            L.or_philox4x32_10.argtypes = [p32, p32, p32]
            L.or_philox4x32_10.restype = None
            L.or_stream_u64.argtypes = [u64, u64, u32, u64]
            L.or_stream_u64.restype = u64
            for f in ("or_log", "or_log1m", "or_exp", "or_lnfact"):
                getattr(L, f).argtypes = [dbl]
                getattr(L, f).restype = dbl
            L.or_lnfact_diff.argtypes = [dbl, dbl]
            L.or_lnfact_diff.restype = dbl
            L.or_u128_to_double.argtypes = [u64, u64]
            L.or_u128_to_double.restype = dbl
            L.or_hypergeometric.argtypes = [u64, u64, u64, u64, u64, u64, u64, u32, p64]
            L.or_hypergeometric.restype = i32
            L.or_binomial.argtypes = [u64, dbl, u64, u64, u32, p64]
            L.or_binomial.restype = i32
            L.or_floyd_leaf.argtypes = [u64, u64, u64, u64, p64]
            L.or_floyd_leaf.restype = i32
            L.or_gnm_directed_chunk_counts.argtypes = [u64, u64, u64, u32, p64]
            L.or_gnm_directed_chunk_counts.restype = i32
            L.or_gnm_directed_chunk.argtypes = [u64, u64, u64, u32, u32, u32, u32, u64, p64, p64]
            L.or_gnm_directed_chunk.restype = i32
            L.or_gnm_directed.argtypes = [u64, u64, u64, u32, u32, u32, p64, p64]
            L.or_gnm_directed.restype = i32
            L.or_gnm_undirected_chunk_counts.argtypes = [u64, u64, u64, u32, p64]
            L.or_gnm_undirected_chunk_counts.restype = i32
            L.or_gnm_undirected.argtypes = [u64, u64, u64, u32, u32, u32, p64, p64]
            L.or_gnm_undirected.restype = i32
            L.or_gnp.argtypes = [i32, u64, dbl, u64, u32, u32, p64, p64, u64, p64]
            L.or_gnp.restype = i32
            L.or_gnm_undirected_rows.argtypes = [u64, u64, u64, u32, u32, u32, u32, u32, p64, p64,
                                                 u64, p64]
            L.or_gnm_undirected_rows.restype = i32
            L.or_gnp_binomial_counts.argtypes = [i32, u64, dbl, u64, u32, p64]
            L.or_gnp_binomial_counts.restype = i32
            L.or_gnp_binomial.argtypes = [i32, u64, dbl, u64, u32, u32, u32, p64, p64, u64, p64]
            L.or_gnp_binomial.restype = i32
            pi32 = ctypes.POINTER(ctypes.c_int)
            L.or_rgg_grid_level.argtypes = [i32, u64, dbl, pi32]
            L.or_rgg_grid_level.restype = i32
            L.or_rgg_cell_counts.argtypes = [i32, u64, dbl, u64, p64]
            L.or_rgg_cell_counts.restype = i32
            L.or_rgg_points.argtypes = [i32, u64, dbl, u64, p32]
            L.or_rgg_points.restype = i32
            L.or_rgg.argtypes = [i32, u64, dbl, u64, p64, p64, u64, p64]
            L.or_rgg.restype = i32
            L.or_rgg_rows.argtypes = [i32, u64, dbl, u64, u64, u64, p64, p64, u64, p64]
            L.or_rgg_rows.restype = i32
            L.or_rgg_digest.argtypes = [i32, u64, dbl, u64, p64, p64, p64]
            L.or_rgg_digest.restype = i32
            L.or_edge_checksum.argtypes = [p64, p64, u64]
            L.or_edge_checksum.restype = u64
            L.or_outdegree_hist.argtypes = [p64, u64, u64, u64, p64]
            L.or_outdegree_hist.restype = i32
            _lib = L
    return _lib


def _p64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _check(rc, what):
    if rc != 0:
        raise OracleError(rc, what)


def _split128(x: int):
    return x & ((1 << 64) - 1), x >> 64


# ---------------------------------------------------------------- primitives

def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return tuple(o)


def stream_u64(seed, node, tag, index):
    return lib().or_stream_u64(seed, node, tag, index)


def log(x):
    return lib().or_log(x)


def log1m(p):
    return lib().or_log1m(p)


def exp(x):
    return lib().or_exp(x)


def lnfact(k):
    return lib().or_lnfact(float(k))


def lnfact_diff(a, d):
    return lib().or_lnfact_diff(float(a), float(d))


def u128_to_double(x: int) -> float:
    lo, hi = _split128(x)
    return lib().or_u128_to_double(lo, hi)


def hypergeometric(N: int, K: int, t: int, seed: int, node: int, tag: int) -> int:
    out = ctypes.c_uint64()
    nl, nh = _split128(N)
    kl, kh = _split128(K)
    _check(lib().or_hypergeometric(nl, nh, kl, kh, t, seed, node, tag, ctypes.byref(out)),
           "hypergeometric")
    return out.value


def binomial(n: int, p: float, seed: int, node: int, tag: int) -> int:
    out = ctypes.c_uint64()
    _check(lib().or_binomial(n, p, seed, node, tag, ctypes.byref(out)), "binomial")
    return out.value


def floyd_leaf(L: int, k: int, seed: int, node: int) -> np.ndarray:
    out = np.zeros(max(k, 1), dtype=np.uint64)
    _check(lib().or_floyd_leaf(L, k, seed, node, _p64(out)), "floyd_leaf")
    return out[:k]


# ---------------------------------------------------------------- generators

def gnm_directed_chunk_counts(n, m, seed, P):
    cnt = np.zeros(P, dtype=np.uint64)
    _check(lib().or_gnm_directed_chunk_counts(n, m, seed, P, _p64(cnt)), "chunk counts")
    return cnt


def gnm_directed_chunk(n, m, seed, P, c, k_c, k_leaf=K_LEAF, k_max=K_MAX):
    u = np.zeros(max(k_c, 1), dtype=np.uint64)
    v = np.zeros(max(k_c, 1), dtype=np.uint64)
    _check(lib().or_gnm_directed_chunk(n, m, seed, P, k_leaf, k_max, c, k_c, _p64(u), _p64(v)),
           "directed chunk")
    return u[:k_c], v[:k_c]


def gnm_directed(n, m, seed, P, k_leaf=K_LEAF, k_max=K_MAX):
    u = np.zeros(max(m, 1), dtype=np.uint64)
    v = np.zeros(max(m, 1), dtype=np.uint64)
    _check(lib().or_gnm_directed(n, m, seed, P, k_leaf, k_max, _p64(u), _p64(v)), "gnm_directed")
    return u[:m], v[:m]


def gnm_undirected_chunk_counts(n, m, seed, P):
    cnt = np.zeros(P * P, dtype=np.uint64)
    _check(lib().or_gnm_undirected_chunk_counts(n, m, seed, P, _p64(cnt)), "quad counts")
    return cnt.reshape(P, P)


def gnm_undirected(n, m, seed, P, k_leaf=K_LEAF, k_max=K_MAX):
    u = np.zeros(max(2 * m, 1), dtype=np.uint64)
    v = np.zeros(max(2 * m, 1), dtype=np.uint64)
    _check(lib().or_gnm_undirected(n, m, seed, P, k_leaf, k_max, _p64(u), _p64(v)),
           "gnm_undirected")
    return u[:2 * m], v[:2 * m]


def gnp(undirected, n, p, seed, P, k_leaf=K_LEAF, cap_hint=None):
    """G(n,p) edge list (both directions when undirected)."""
    L = lib()
    cap = cap_hint if cap_hint is not None else 1 << 16
    while True:
        u = np.zeros(max(cap, 1), dtype=np.uint64)
        v = np.zeros(max(cap, 1), dtype=np.uint64)
        cnt = ctypes.c_uint64()
        rc = L.or_gnp(1 if undirected else 0, n, p, seed, P, k_leaf, _p64(u), _p64(v), cap,
                      ctypes.byref(cnt))
        if rc == 3:
            cap = cnt.value
            continue
        _check(rc, "gnp")
        return u[:cnt.value], v[:cnt.value]


def gnm_undirected_rows(n, m, seed, P, b0, b1, k_leaf=K_LEAF, k_max=K_MAX, cap_hint=None):
    """Rows of row blocks [b0, b1) of undirected G(n,m), both directions (Sec. 4.2)."""
    L = lib()
    cap = cap_hint if cap_hint is not None else 1 << 16
    while True:
        u = np.zeros(max(cap, 1), dtype=np.uint64)
        v = np.zeros(max(cap, 1), dtype=np.uint64)
        cnt = ctypes.c_uint64()
        rc = L.or_gnm_undirected_rows(n, m, seed, P, k_leaf, k_max, b0, b1, _p64(u), _p64(v), cap,
                                      ctypes.byref(cnt))
        if rc == 3:
            cap = cnt.value
            continue
        _check(rc, "gnm_undirected_rows")
        return u[:cnt.value], v[:cnt.value]


def gnp_binomial_counts(undirected, n, p, seed, P):
    """Sec. 4.3 chunk counts: P (directed) or P(P+1)/2 (undirected) binomials."""
    C = P * (P + 1) // 2 if undirected else P
    cnt = np.zeros(C, dtype=np.uint64)
    _check(lib().or_gnp_binomial_counts(1 if undirected else 0, n, p, seed, P, _p64(cnt)),
           "gnp_binomial_counts")
    return cnt


def gnp_binomial(undirected, n, p, seed, P, k_leaf=K_LEAF, k_max=K_MAX, cap_hint=None):
    """G(n,p) by binomial chunk counts and the G(n,m) sampler (Sec. 4.3)."""
    L = lib()
    cap = cap_hint if cap_hint is not None else 1 << 16
    while True:
        u = np.zeros(max(cap, 1), dtype=np.uint64)
        v = np.zeros(max(cap, 1), dtype=np.uint64)
        cnt = ctypes.c_uint64()
        rc = L.or_gnp_binomial(1 if undirected else 0, n, p, seed, P, k_leaf, k_max, _p64(u),
                               _p64(v), cap, ctypes.byref(cnt))
        if rc == 3:
            cap = cnt.value
            continue
        _check(rc, "gnp_binomial")
        return u[:cnt.value], v[:cnt.value]


# ---------------------------------------------------------------- RGG, Sec. 5

def rgg_grid_level(dim, n, r) -> int:
    """g of the 2^g-per-dimension cell grid."""
    g = ctypes.c_int()
    _check(lib().or_rgg_grid_level(dim, n, r, ctypes.byref(g)), "rgg_grid_level")
    return g.value


def rgg_cell_counts(dim, n, r, seed) -> np.ndarray:
    """Points per cell, row-major cell order (dimension 0 fastest)."""
    cnt = np.zeros(1 << (dim * rgg_grid_level(dim, n, r)), dtype=np.uint64)
    _check(lib().or_rgg_cell_counts(dim, n, r, seed, _p64(cnt)), "rgg_cell_counts")
    return cnt


def rgg_points(dim, n, r, seed) -> np.ndarray:
    """(n, dim) uint32 fixed-point coordinates (x 2^-32)."""
    x = np.zeros((max(n, 1), dim), dtype=np.uint32)
    _check(lib().or_rgg_points(dim, n, r, seed,
                               x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))), "rgg_points")
    return x[:n]


def rgg_rows(dim, n, r, seed, u_lo, u_hi, cap_hint=None):
    """Entries of the rows of vertices [u_lo, u_hi), sorted by (u, v)."""
    L = lib()
    cap = cap_hint if cap_hint is not None else 1 << 16
    while True:
        u = np.zeros(max(cap, 1), dtype=np.uint64)
        v = np.zeros(max(cap, 1), dtype=np.uint64)
        cnt = ctypes.c_uint64()
        rc = L.or_rgg_rows(dim, n, r, seed, u_lo, u_hi, _p64(u), _p64(v), cap, ctypes.byref(cnt))
        if rc == 3:
            cap = cnt.value
            continue
        _check(rc, "rgg_rows")
        return u[:cnt.value], v[:cnt.value]


def rgg(dim, n, r, seed, cap_hint=None):
    """All entries of RGG(n, r) (both directions), sorted by (u, v)."""
    return rgg_rows(dim, n, r, seed, 0, n, cap_hint)


def rgg_digest(dim, n, r, seed):
    """(entries, digest, degree histogram[65]) without storing the edges."""
    e = ctypes.c_uint64()
    d = ctypes.c_uint64()
    h = np.zeros(65, dtype=np.uint64)
    _check(lib().or_rgg_digest(dim, n, r, seed, ctypes.byref(e), ctypes.byref(d), _p64(h)),
           "rgg_digest")
    return e.value, d.value, h


def edge_checksum(u, v) -> int:
    u = np.ascontiguousarray(u, dtype=np.uint64)
    v = np.ascontiguousarray(v, dtype=np.uint64)
    return lib().or_edge_checksum(_p64(u), _p64(v), len(u))


def outdegree_hist(u, row_lo, row_hi) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.uint64)
    h = np.zeros(65, dtype=np.uint64)
    _check(lib().or_outdegree_hist(_p64(u), len(u), row_lo, row_hi, _p64(h)), "hist")
    return h
