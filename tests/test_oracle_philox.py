"""Pins the oracle's Philox4x32-10 against an independent implementation:
cuRAND's host-side PHILOX4_32_10 generator (run on the CPU, no GPU needed).

cuRAND's host generator lays block j of its output stream at counter
(j // 65536, 0, j % 65536, 0) with key = (seed lo, seed hi); an offset of o
32-bit words starts the stream at block o // 4.  Block indices >= 65536 reach
counter word 0, offsets >= 2^50 words reach word 1, and the key is exercised
by the seeds.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

import oracle

_CURAND = None


def _curand():
    global _CURAND
    if _CURAND is None:
        cands = []
        cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
        for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"),
                  os.path.join(cuda, "targets", "sbsa-linux", "lib"),
                  os.path.join(cuda, "targets", "x86_64-linux", "lib")):
            cands += [os.path.join(d, "libcurand.so"), os.path.join(d, "libcurand.so.10")]
        found = ctypes.util.find_library("curand")
        if found:
            cands.append(found)
        for c in cands:
            try:
                _CURAND = ctypes.CDLL(c)
                break
            except OSError:
                continue
    if _CURAND is None:
        pytest.skip("libcurand not found")
    return _CURAND


def curand_host_philox(seed: int, offset_words: int, n_words: int):
    L = _curand()
    gen = ctypes.c_void_p()
    assert L.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert L.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert L.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset_words)) == 0
        out = np.zeros(n_words, dtype=np.uint32)
        assert L.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                ctypes.c_size_t(n_words)) == 0
    finally:
        L.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 20230825])
def test_philox_matches_curand_host_word2(seed):
    out = curand_host_philox(seed, 0, 4 * 64)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for j in range(64):
        assert oracle.philox4x32_10((0, 0, j, 0), key) == [int(v) for v in out[4 * j:4 * j + 4]]


def test_philox_matches_curand_host_word0():
    seed = 0xDEADBEEFCAFEF00D
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for blk in (65536, 65536 * 3 + 17, 65536 * 1000 + 65535):
        out = curand_host_philox(seed, 4 * blk, 4)
        ctr = (blk // 65536, 0, blk % 65536, 0)
        assert oracle.philox4x32_10(ctr, key) == [int(v) for v in out]


def test_philox_matches_curand_host_word1():
    seed = 77
    key = (seed, 0)
    for hi, lo_blk in ((1, 0), (1, 5), (3, 12345)):
        blk = (hi << 48) + lo_blk
        out = curand_host_philox(seed, 4 * blk, 4)
        ctr = ((blk // 65536) & 0xFFFFFFFF, (blk // 65536) >> 32, blk % 65536, 0)
        assert oracle.philox4x32_10(ctr, key) == [int(v) for v in out]


def test_philox_is_a_bijection_sample():
    # distinct counters give distinct outputs (a dropped counter word would
    # collapse some of them)
    key = (12345, 678)
    outs = set()
    for w in range(4):
        for v in range(1, 200):
            ctr = [0, 0, 0, 0]
            ctr[w] = v
            outs.add(tuple(oracle.philox4x32_10(ctr, key)))
    assert len(outs) == 4 * 199


def test_child_id_distinct():
    ids = {oracle.child_id(p, s, t) for p in range(200) for s in (0, 1, 999) for t in (1, 2)}
    assert len(ids) == 200 * 3 * 2
