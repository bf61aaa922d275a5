"""Pins of the oracle's pseudorandomisation (Sec. 2.2 of the paper: per-subtree
seeds from a hash of (global seed, subtree id); here Philox4x32-10 keyed by the
seed with the subtree named in the counter).

Philox4x32-10 is pinned to an independent implementation: cuRAND's host-side
generator (a CPU library routine; no GPU needed).  Its default ordering emits
output block b from the counter (b // 65536, 0, b % 65536, 0) with the seed as
key, and a generator offset of 4*b starts at block b, so counter words 0, 1 and
2 and both key words are exercised.
"""
import ctypes
import os

import numpy as np
import pytest

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    pytest.skip("libcurand not available")


def _curand_blocks(cr, seed, first_block, nblocks):
    gen = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert cr.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * first_block)) == 0
        out = np.zeros(4 * nblocks, dtype=np.uint32)
        assert cr.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.c_size_t(out.size)) == 0
    finally:
        cr.curandDestroyGenerator(gen)
    return out.reshape(nblocks, 4)


@pytest.mark.parametrize("seed", [0, 1, 0x5EED, 0x123456789ABCDEF0, (1 << 64) - 1])
@pytest.mark.parametrize("first_block", [0, 65530, 65536 * 7 + 3, (1 << 40) + 12345 * 65536 + 17])
def test_philox_matches_curand_host_generator(orc, seed, first_block):
    cr = _curand()
    blocks = _curand_blocks(cr, seed, first_block, 12)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for i in range(blocks.shape[0]):
        b = first_block + i
        pos, thread = divmod(b, 65536)
        ctr = (pos & 0xFFFFFFFF, pos >> 32, thread, 0)
        assert orc.philox4x32_10(ctr, key) == tuple(int(x) for x in blocks[i]), (seed, b)


def test_stream_word_layout(orc):
    """u64 #i of a stream is half (i & 1) of the Philox block i >> 1 whose
    counter is (i >> 1, lo32(node), hi32(node), tag); each half is wA<<32|wB."""
    seed, node, tag = 0xDEADBEEFCAFEF00D, (7 << 32) | 0x1234, 4 | (3 << 8)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for i in range(10):
        w = orc.philox4x32_10((i >> 1, node & 0xFFFFFFFF, node >> 32, tag), key)
        want = (w[0] << 32 | w[1]) if i % 2 == 0 else (w[2] << 32 | w[3])
        assert orc.stream_u64(seed, node, tag, i) == want


def test_streams_differ_by_tag_and_node(orc):
    a = [orc.stream_u64(1, 5, 1, i) for i in range(8)]
    b = [orc.stream_u64(1, 5, 2, i) for i in range(8)]
    c = [orc.stream_u64(1, 6, 1, i) for i in range(8)]
    assert len(set(a) | set(b) | set(c)) == 24


def test_u128_to_double_is_correctly_rounded(orc):
    """Conversion of 128-bit universe sizes: nearest-even, as Python's int->float."""
    rng = np.random.default_rng(3)
    vals = [0, 1, (1 << 53) + 1, (1 << 64) - 1, (1 << 64) + (1 << 11), (1 << 72) + (1 << 19),
            (1 << 72) + (1 << 19) + 1, (1 << 127) + (1 << 74)]
    for _ in range(2000):
        bits = int(rng.integers(1, 128))
        vals.append(int(rng.integers(0, 1 << 62)) << max(0, bits - 62) | int(rng.integers(0, 1 << 20)))
    for x in vals:
        x &= (1 << 128) - 1
        assert orc.u128_to_double(x) == float(x), x
