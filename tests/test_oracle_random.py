"""Pins for the oracle's random draws: Philox4x32-10 against cuRAND's host
generator (an independent implementation, run, not read), and the Gaussian
transform against numpy's libm-backed log/sin/cos and the normal law."""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O


def _curand():
    cands = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64",
                          "libcurand.so"), ctypes.util.find_library("curand")]
    for c in cands:
        if not c:
            continue
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 2**64 - 1])
def test_philox_matches_curand_host(seed):
    L = _curand()
    if L is None:
        pytest.skip("libcurand not present")
    g = ctypes.c_void_p()
    assert L.curandCreateGeneratorHost(ctypes.byref(g), 161) == 0  # PHILOX4_32_10
    assert L.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
    assert L.curandSetGeneratorOrdering(g, 103) == 0  # PSEUDO_LEGACY
    nblk = 64
    out = np.zeros(4 * nblk, np.uint32)
    assert L.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p),
                            ctypes.c_size_t(out.size)) == 0
    L.curandDestroyGenerator(g)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    # cuRAND's legacy host stream walks counter word 2 (its subsequence word)
    for i in range(nblk):
        np.testing.assert_array_equal(O.philox4x32_10([0, 0, i, 0], key), out[4 * i:4 * i + 4])


def test_philox_counter_words_all_matter():
    base = O.philox4x32_10([5, 6, 7, 8], [9, 10])
    for w in range(4):
        c = [5, 6, 7, 8]
        c[w] ^= 1
        assert not np.array_equal(O.philox4x32_10(c, [9, 10]), base)
    for w in range(2):
        k = [9, 10]
        k[w] ^= 1 << 31
        assert not np.array_equal(O.philox4x32_10([5, 6, 7, 8], k), base)


def test_philox_bits_balanced():
    words = np.concatenate([O.philox4x32_10([c, 3, 4, 0], [1, 2]) for c in range(4000)])
    bits = np.unpackbits(words.view(np.uint8))
    # 512000 fair bits: mean within 5 sigma
    assert abs(bits.mean() - 0.5) < 5 * 0.5 / np.sqrt(bits.size)
    u = (words >> 8).astype(np.float64) / 2**24
    assert stats.kstest(u, "uniform").pvalue > 1e-4


def test_log_f32_against_libm():
    rng = np.random.default_rng(0)
    r = rng.integers(0, 2**24, 20000)
    us = ((r + 1).astype(np.float64) * 2.0**-24).astype(np.float32)
    us = np.r_[us, np.float32(2.0**-24), np.float32(1.0), np.float32(0.5),
               np.float32(np.sqrt(0.5)), np.float32(np.sqrt(2.0) / 2 * 1.0000001)]
    for u in us:
        got = O.log_f32(float(u))
        ref = np.log(np.float64(u))
        assert abs(got - ref) <= 3e-7 * max(1.0, abs(ref)), (u, got, ref)
    assert O.log_f32(1.0) == 0.0


def test_sincos_against_libm():
    rng = np.random.default_rng(1)
    r24 = np.r_[rng.integers(0, 2**24, 20000), np.arange(8) << 21,
                (np.arange(8) << 21) + (1 << 21) - 1]
    for r in r24:
        s, c = O.sincos_2pi(int(r))
        th = 2 * np.pi * int(r) / 2**24
        assert abs(s - np.sin(th)) < 4e-7 and abs(c - np.cos(th)) < 4e-7, (r, s, c)


def test_box_muller_against_exact_transform_and_normal_law():
    rng = np.random.default_rng(2)
    ra = rng.integers(0, 2**32, 40000, dtype=np.uint64)
    rb = rng.integers(0, 2**32, 40000, dtype=np.uint64)
    z = []
    for a, b in zip(ra, rb):
        z0, z1 = O.box_muller(int(a), int(b))
        u1 = ((int(a) >> 8) + 1) * 2.0**-24
        u2 = (int(b) >> 8) * 2.0**-24
        rad = np.sqrt(-2 * np.log(u1))
        assert abs(z0 - rad * np.cos(2 * np.pi * u2)) < 2e-6 * max(1, rad)
        assert abs(z1 - rad * np.sin(2 * np.pi * u2)) < 2e-6 * max(1, rad)
        z += [z0, z1]
    z = np.array(z)
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 0.02
    assert stats.kstest(z, "norm").pvalue > 1e-4
