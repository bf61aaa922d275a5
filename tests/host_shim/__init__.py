"""Builds tests/host_shim/shim.cu (the library's host-callable primitives) for the CPU tests."""
import ctypes
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CSRC = os.path.join(ROOT, "paper_1710_07565_gb300", "csrc")
OUT = os.path.join(HERE, "_build", "libshim.so")


def load():
    deps = [os.path.join(HERE, "shim.cu")] + [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    if not os.path.exists(OUT) or any(os.path.getmtime(d) > os.path.getmtime(OUT) for d in deps):
        os.makedirs(os.path.dirname(OUT), exist_ok=True)
        nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
        tmp = OUT + f".tmp{os.getpid()}"
        subprocess.run([nvcc, "-std=c++17", "-O2", "-Xcompiler", "-fPIC,-ffp-contract=off",
                        "-shared", "-I", CSRC, "-o", tmp, os.path.join(HERE, "shim.cu")], check=True)
        os.replace(tmp, OUT)
    L = ctypes.CDLL(OUT)
    u64, u32, dbl, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_int
    p64 = ctypes.POINTER(ctypes.c_uint64)
    for f in ("sh_log", "sh_log1m", "sh_exp", "sh_lnfact"):
        getattr(L, f).argtypes = [dbl]
        getattr(L, f).restype = dbl
    L.sh_lnfact_diff.argtypes = [dbl, dbl]
    L.sh_lnfact_diff.restype = dbl
    L.sh_dbl128.argtypes = [u64, u64]
    L.sh_dbl128.restype = dbl
    L.sh_stream_u64.argtypes = [u64, u64, u32, u64]
    L.sh_stream_u64.restype = u64
    L.sh_hyper.argtypes = [u64, u64, u64, u64, u64, u64, u64, u32, p64]
    L.sh_hyper.restype = i32
    L.sh_binom.argtypes = [u64, dbl, u64, u64, u32, p64]
    L.sh_binom.restype = i32
    L.sh_lemire.argtypes = [u64, u64, u64, u64]
    L.sh_lemire.restype = u64
    L.sh_divq.argtypes = [u64, p64, p64, u64]
    L.sh_divq.restype = None
    L.sh_und_map.argtypes = [u64, u32, u64, u64, p64, p64]
    L.sh_und_map.restype = None
    L.sh_und_universe.argtypes = [u64, u32, u64]
    L.sh_und_universe.restype = u64
    return L
