"""Pins of the oracle's Philox4x32-10 (Salmon et al., SC'11).

The cuRAND host generator CURAND_RNG_PSEUDO_PHILOX4_32_10 runs on the CPU
without a GPU.  In its default ordering, output block n (four words) is the
Philox block for key = (seed_lo, seed_hi) and counter
(n >> 16, 0, n & 0xFFFF, 0); a stream offset of 2^50 words moves the counter's
second word to 1.  The oracle must reproduce those words bit for bit.
"""
import ctypes as C
import os

import numpy as np
import pytest

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for p in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return C.CDLL(p)
        except OSError:
            continue
    pytest.skip("libcurand not available")


def _curand_words(seed, n_words, offset=0):
    lib = _curand()
    g = C.c_void_p()
    if lib.curandCreateGeneratorHost(C.byref(g), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(g, C.c_ulonglong(seed)) == 0
        if offset:
            assert lib.curandSetGeneratorOffset(g, C.c_ulonglong(offset)) == 0
        out = np.zeros(n_words, np.uint32)
        assert lib.curandGenerate(g, out.ctypes.data_as(C.c_void_p), C.c_size_t(n_words)) == 0
    finally:
        lib.curandDestroyGenerator(g)
    return out.reshape(-1, 4)


@pytest.mark.parametrize("seed", [0, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 987654321])
def test_philox_matches_curand_host(orc, seed):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    blocks = _curand_words(seed, 4 * (65536 * 3))
    rng = np.random.default_rng(seed & 0xFFFF)
    picks = np.concatenate([np.arange(8), [65535, 65536, 65537, 131072 + 17],
                            rng.integers(0, blocks.shape[0], 300)])
    for n in picks:
        n = int(n)
        ctr = [n >> 16, 0, n & 0xFFFF, 0]
        assert (orc.philox4x32_10(ctr, key) == blocks[n]).all(), (seed, n)


def test_philox_second_counter_word_matches_curand(orc):
    seed = 0x0123456789ABCDEF
    key = [seed & 0xFFFFFFFF, seed >> 32]
    off = (1 << 50) + 4 * (7 * 65536 + 3)
    blocks = _curand_words(seed, 64, offset=off)
    for n in range(16):
        ctr = [7, 1, 3 + n, 0]
        assert (orc.philox4x32_10(ctr, key) == blocks[n]).all()


def test_rng_words_layout(orc):
    """key = (seed_lo, seed_hi ^ sample); ctr = (c0, c1, step_lo, purpose<<24 | step_hi)."""
    seed, sample, c0, c1, step, purpose = 0xDEADBEEF12345678, 7, 123, 45, (5 << 32) + 99, 3
    w = orc.rng_words(seed, sample, c0, c1, step, purpose)
    key = [seed & 0xFFFFFFFF, (seed >> 32) ^ sample]
    ctr = [c0, c1, step & 0xFFFFFFFF, (purpose << 24) | (step >> 32)]
    assert (w == orc.philox4x32_10(ctr, key)).all()


def test_philox_uniformity(orc):
    """Frequency chi^2 of the 24-bit uniforms over 64 bins, and a serial test
    on consecutive (w0, w1) pairs over an 8x8 grid."""
    n = 40000
    w = np.array([orc.rng_words(42, 0, x, 0, 0, 0) for x in range(n)], dtype=np.uint64)
    for col in range(4):
        bins = np.bincount((w[:, col] >> 26).astype(np.int64), minlength=64)
        chi2 = ((bins - n / 64) ** 2 / (n / 64)).sum()
        assert chi2 < 63 + 5 * np.sqrt(2 * 63), chi2
    g = ((w[:, 0] >> 29) * 8 + (w[:, 1] >> 29)).astype(np.int64)
    bins = np.bincount(g, minlength=64)
    chi2 = ((bins - n / 64) ** 2 / (n / 64)).sum()
    assert chi2 < 63 + 5 * np.sqrt(2 * 63), chi2
