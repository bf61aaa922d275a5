"""The C-ABI library builds for sm_103a, loads, and exports every function
include/kg.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "kg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)  # comments
    names = re.findall(r"^[A-Za-z_][\w \t]*?\**[ \t]*\b(kg_[a-z0-9_]+)[ \t]*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("kg_gnm_directed", "kg_gnm_undirected", "kg_gnp_directed", "kg_gnp_undirected",
                 "kg_gnm_directed_range", "kg_gnm_undirected_rows", "kg_gnp_binomial",
                 "kg_batch_run", "kg_server_poll", "kg_edge_digest", "kg_last_error",
                 "kg_status_str", "kg_gnm_directed_noalloc", "kg_rgg", "kg_rgg_count",
                 "kg_rgg_cell_counts", "kg_rgg_grid", "kg_gnp_size", "kg_shutdown"):
        assert must in names, must


def test_library_exports_every_declared_function():
    import paper_1710_07565_gb300 as kg
    path = kg.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # host-only calls that need no device
    lib.kg_status_str.restype = ctypes.c_char_p
    lib.kg_status_str.argtypes = [ctypes.c_int]
    assert lib.kg_status_str(0) and lib.kg_status_str(3)


def test_rgg_grid_level_matches_the_oracle(orc):
    """kg_rgg_grid is host logic (no device): the library's grid rule and the
    oracle's, written separately, agree over sizes, radii and both limits."""
    import paper_1710_07565_gb300 as kg
    lib = ctypes.CDLL(kg.build())
    lib.kg_rgg_grid.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_double,
                                ctypes.POINTER(ctypes.c_int)]
    lib.kg_rgg_grid.restype = ctypes.c_int
    g = ctypes.c_int()
    radii = [0.0, 1e-9, 1e-6, 2 ** -17, 1e-4, 0.001, 0.01, 0.03, 0.1, 0.2, 0.25, 0.3, 0.5]
    sizes = [0, 1, 3, 4, 7, 8, 63, 64, 1000, 4095, 4096, 10 ** 6, 1 << 26, (1 << 32) - 1]
    for dim in (2, 3):
        for n in sizes:
            for r in radii:
                assert lib.kg_rgg_grid(dim, n, r, ctypes.byref(g)) == 0
                assert g.value == orc.rgg_grid_level(dim, n, r), (dim, n, r)
    assert lib.kg_rgg_grid(4, 10, 0.1, ctypes.byref(g)) == kg.KG_ERR_ARG
    assert lib.kg_rgg_grid(2, 10, 0.51, ctypes.byref(g)) == kg.KG_ERR_ARG
    assert lib.kg_rgg_grid(2, 1 << 32, 0.1, ctypes.byref(g)) == kg.KG_ERR_RANGE


def _largest_fitting_chunks(kg, n, m, lim, top=512):
    """Largest chunk count <= top whose no-allocation scratch fits `lim`."""
    for P in range(top, 0, -1):
        if kg.kg_gnm_directed_noalloc_scratch(n, m, P) <= lim:
            return P
    return 0


def test_noalloc_scratch_need_per_tile():
    """kg_gnm_directed_noalloc_scratch is host logic (the measuring pass of
    the carve that the no-allocation call runs).  Its need grows by ~144 B
    per tile (counts of two tile-tree levels, the scanned offsets, the tile
    lists and the 112-byte descriptor), so the 32 MiB array holds about
    233,000 tiles, and the boundary between fitting and not fitting moves one
    chunk at a time at a fixed tile depth."""
    import paper_1710_07565_gb300 as kg
    kg.lib()
    lim = kg.NOALLOC_SCRATCH_BYTES
    n = 1 << 20
    # tile depth d: m ceil(n/P) / n <= 1024 * 2^d; doubling m doubles the tiles
    a = kg.kg_gnm_directed_noalloc_scratch(n, 1 << 24, 64)   # 64 * 2^8 tiles
    b = kg.kg_gnm_directed_noalloc_scratch(n, 1 << 25, 64)   # 64 * 2^9 tiles
    per_tile = (b - a) / (64 * (1 << 8))
    assert 140 <= per_tile <= 148, per_tile
    # at m = 2.3e8 the tile depth is 10 for 220 <= P <= 256: the largest
    # fitting chunk count carries about lim / per_tile / 2^10 chunks
    m = 230_000_000
    P = _largest_fitting_chunks(kg, n, m, lim, 256)
    assert abs(P - lim / per_tile / 1024) < 2, P
    assert kg.kg_gnm_directed_noalloc_scratch(n, m, P + 1) > lim
    # the instance the old estimate admitted but whose descriptors did not fit
    assert kg.kg_gnm_directed_noalloc_scratch(1 << 26, 1 << 29, 64) > lim
