"""Pins of the oracle's Philox4x32-10 against a library generator.

cuRAND's host-side Philox4_32_10 generator (a CPU implementation shipped with
the CUDA toolkit) emits, for seed s, the words of Philox4x32-10 with key
(lo32(s), hi32(s)) and counter (0, 0, i, 0) for its i-th group of four. The
oracle's generator is written from Salmon et al. (SC'11); agreement with an
independent implementation on several keys and counters pins it.
"""
import ctypes
import os

import numpy as np
import pytest

CURAND = "/usr/local/cuda/lib64/libcurand.so"


def _curand_stream(seed, n):
    try:
        lib = ctypes.CDLL(CURAND)
    except OSError:
        pytest.skip("cuRAND host library not available")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:  # PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(n, np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host(oracle_mod, seed):
    if not os.path.exists(CURAND):
        pytest.skip("cuRAND host library not available")
    ref = _curand_stream(seed, 32)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(8):
        got = oracle_mod.philox4x32_10([0, 0, i, 0], key)
        assert got.tolist() == ref[4 * i:4 * i + 4].tolist(), i


def test_philox_counter_words_all_matter(oracle_mod):
    base = oracle_mod.philox4x32_10([5, 6, 7, 8], [9, 10]).tolist()
    for k in range(4):
        c = [5, 6, 7, 8]
        c[k] += 1
        assert oracle_mod.philox4x32_10(c, [9, 10]).tolist() != base
    for k in range(2):
        key = [9, 10]
        key[k] += 1
        assert oracle_mod.philox4x32_10([5, 6, 7, 8], key).tolist() != base


def test_philox_uniformity(oracle_mod):
    # 4096 blocks: the top-24-bit uniforms have mean 1/2 and variance 1/12
    u = np.concatenate([oracle_mod.philox4x32_10([i, 3, 0, 0], [17, 0]) for i in range(4096)])
    u = (u >> 8).astype(np.float64) * 2.0 ** -24
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 0.005
