"""Pins of the oracle's Philox4x32-10 stream (Salmon et al., SC'11).

The oracle's generator is checked against an implementation it shares
nothing with: cuRAND's host-side Philox4x32-10 generator, whose j-th block of
four outputs for seed s is Philox(counter=(0, 0, j, 0), key=(s lo, s hi)).
Then the uniform conversion and the uniformity of the keyed draws."""
import ctypes as C
import ctypes.util
import os

import numpy as np
import pytest

from oracle import oracle as O


def _curand():
    for p in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if p and (os.path.exists(p) or not p.startswith("/")):
            try:
                return C.CDLL(p)
            except OSError:
                pass
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(seed):
    L = _curand()
    if L is None:
        pytest.skip("libcurand not available")
    g = C.c_void_p()
    assert L.curandCreateGeneratorHost(C.byref(g), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    try:
        assert L.curandSetPseudoRandomGeneratorSeed(g, C.c_uint64(seed)) == 0
        n_blocks = 2048
        out = np.zeros(4 * n_blocks, np.uint32)
        assert L.curandGenerate(g, out.ctypes.data_as(C.c_void_p), C.c_size_t(out.size)) == 0
    finally:
        L.curandDestroyGenerator(g)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in list(range(64)) + list(range(64, n_blocks, 97)):
        assert np.array_equal(O.philox4x32_10([0, 0, j, 0], key), out[4 * j:4 * j + 4]), j


def test_uniform_is_top_53_bits_of_first_two_words():
    for seed, shot, op in [(1, 0, 0), (7, 12345, 99), (2 ** 40 + 3, 2 ** 33 + 5, 511)]:
        x = O.philox4x32_10([shot & 0xFFFFFFFF, shot >> 32, op, 0], [seed & 0xFFFFFFFF, seed >> 32])
        bits = (int(x[0]) << 32) | int(x[1])
        assert O.uniform(seed, shot, op) == (bits >> 11) / 2.0 ** 53


def test_uniform_draws_are_uniform():
    stats = pytest.importorskip("scipy.stats")
    u = np.array([O.uniform(3, s, op) for s in range(400) for op in range(250)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    hist, _ = np.histogram(u, bins=64, range=(0, 1))
    assert stats.chisquare(hist).pvalue > 1e-3
    # neighbouring shots and ops are not correlated
    a = u.reshape(400, 250)
    assert abs(np.corrcoef(a[:, 0], a[:, 1])[0, 1]) < 0.2
    assert abs(np.corrcoef(a[:-1, 5], a[1:, 5])[0, 1]) < 0.2
