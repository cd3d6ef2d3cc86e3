"""Pins the oracle's Philox4x32-10 (Salmon et al., SC'11) to an independent
implementation: cuRAND's host-side PHILOX4_32_10 generator, run as a library
on the CPU.  That generator emits block b of its stream as Philox of the
counter (b >> 16 as a 64-bit value in words 0-1, b & 0xFFFF in word 2, 0) under
the key (seed lo32, seed hi32), which exercises the key and counter words 0-2.
Word 3 is pinned on the GPU against cuRAND's device API (tests/test_gpu_rng.py).
"""
import ctypes
import os

import numpy as np
import pytest

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for name in ("libcurand.so", "libcurand.so.10"):
        for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
                  "/usr/local/cuda/targets/x86_64-linux/lib", ""):
            path = os.path.join(d, name) if d else name
            try:
                return ctypes.CDLL(path)
            except OSError:
                continue
    pytest.skip("libcurand not found")


def _curand_stream(seed: int, offset: int, count: int) -> np.ndarray:
    lib = _curand()
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(count, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(count)) == 0
        return out
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 1508078281])
def test_philox_matches_curand_host(orc, seed):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    out = _curand_stream(seed, 0, 4 * 70)
    for b in range(70):
        mine = orc.philox4x32_10([0, 0, b, 0], key)
        assert list(mine) == list(out[4 * b:4 * b + 4]), b


@pytest.mark.parametrize("block0", [1 << 16, 5 << 16 | 3, (1 << 48) | 7, (0x1234 << 48) | (99 << 16) | 2])
def test_philox_matches_curand_high_counter_words(orc, block0):
    seed = 0x0FEDCBA987654321
    key = [seed & 0xFFFFFFFF, seed >> 32]
    out = _curand_stream(seed, 4 * block0, 8)
    for q in range(2):
        b = block0 + q
        hi, lo = b >> 16, b & 0xFFFF
        ctr = [hi & 0xFFFFFFFF, hi >> 32, lo, 0]
        assert list(orc.philox4x32_10(ctr, key)) == list(out[4 * q:4 * q + 4])
