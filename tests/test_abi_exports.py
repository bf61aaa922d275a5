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
                 "kg_status_str", "kg_gnm_directed_noalloc"):
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
