"""Pins of the oracle's Philox4x32-10 against an outside implementation.

The paper names no generator; the build reads it as Philox4x32-10 (Salmon et al.,
SC'11). cuRAND's host-side PHILOX4_32_10 generator is an independent
implementation of the same published function. With seed s it uses key
(lo32(s), hi32(s)); its default ordering emits output block
b = ((c1 << 32) | c0) * 65536 + c2 from counter (c0, c1, c2, 0) (a mapping
established by matching outputs), and an offset of 4*b starts at block b.
Counter word 3 is out of its reach; the test below at least shows it enters.
"""
import ctypes

import numpy as np
import pytest

import oracle as O

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for name in ("libcurand.so", "libcurand.so.10", "/usr/local/cuda/lib64/libcurand.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def _curand_blocks(seed, first_block, n_blocks):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available on this host")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * first_block)) == 0
        out = np.zeros(4 * n_blocks, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out.reshape(n_blocks, 4)


def _block_index(c0, c1, c2):
    return (((c1 << 32) | c0) << 16) + c2


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 2**64 - 1])
def test_philox_matches_curand_counter_word2(seed):
    ref = _curand_blocks(seed, 0, 8)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for i in range(8):
        got = O.philox((0, 0, i, 0), key)
        assert np.array_equal(got, ref[i]), (seed, i, got, ref[i])


@pytest.mark.parametrize("ctr", [(1, 0, 0), (7, 0, 65535), (0xFFFFFFFF, 0, 12), (7, 5, 3), (2, 0x3FFF, 9)])
def test_philox_matches_curand_counter_words01(ctr):
    seed = 0xDEADBEEF00000042
    c0, c1, c2 = ctr
    ref = _curand_blocks(seed, _block_index(c0, c1, c2), 1)
    got = O.philox((c0, c1, c2, 0), (seed & 0xFFFFFFFF, seed >> 32))
    assert np.array_equal(got, ref[0]), (ctr, got, ref[0])


def test_philox_counter_word3_enters():
    key = (9, 10)
    base = O.philox((1, 2, 3, 0), key)
    assert not np.array_equal(base, O.philox((1, 2, 3, 1), key))
    assert not np.array_equal(O.philox((1, 2, 3, 1), key), O.philox((1, 2, 3, 2), key))


def test_uniform_mapping_is_uniform():
    # (x >> 8) * 2^-24 of Philox words: chi-square over 64 bins.
    vals = []
    for i in range(4096):
        vals.extend(O.philox((i, 3, 7, 11), (123, 456)))
    u = (np.array(vals, dtype=np.uint64) >> 8).astype(np.float64) / 2**24
    assert u.min() >= 0.0 and u.max() < 1.0
    hist, _ = np.histogram(u, bins=64, range=(0, 1))
    expected = len(u) / 64
    chi2 = ((hist - expected) ** 2 / expected).sum()
    assert chi2 < 120.0  # 63 degrees of freedom
