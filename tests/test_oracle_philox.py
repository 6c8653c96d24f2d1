"""Pins of the oracle's Philox4x32-10 uniform stream (Section 3.1 (i): the
program-and-event-occurrence-specific uniform z_(Prog,E)).

The oracle's block function is written from Salmon et al. (SC'11).  It is
pinned here against cuRAND's host-side Philox4_32_10 generator, run as a
library (its k-th output block is the Philox block of counter (0, 0, k, 0)
under key (seed mod 2^32, seed >> 32)), and by statistical tests of the
uniform mapping.
"""

import ctypes
import os

import numpy as np
import pytest
from scipy import stats

import oracle

_CURAND_PHILOX4_32_10 = 161


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    return None


def _curand_blocks(lib, seed, n_blocks):
    g = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(g), _CURAND_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(4 * n_blocks, dtype=np.uint32)
        assert lib.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    finally:
        lib.curandDestroyGenerator(g)
    return out.reshape(n_blocks, 4)


@pytest.mark.parametrize("seed", [0, 1, 0x9ABCDEF012345678, 20150126])
def test_philox_block_matches_curand(seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    n = 2048
    ref = _curand_blocks(lib, seed, n)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for k in list(range(64)) + list(range(64, n, 37)):
        got = oracle.philox4x32_10([0, 0, k, 0], key)
        assert np.array_equal(got, ref[k]), (seed, k)


def test_uniform_is_word0_mapped_to_open_interval():
    # every grid value (j + 1/2) 2^-23 is exact in FP32; (j + 1/2) 2^-24 would not be above 1/2
    j = np.arange(0, 1 << 23, 997, dtype=np.int64)
    grid = (j + 0.5) / 2.0**23
    assert np.array_equal(grid.astype(np.float32).astype(np.float64), grid)
    assert np.array_equal((1.0 - grid).astype(np.float32).astype(np.float64), 1.0 - grid)
    for (t, k, e, s) in [(0, 0, 0, 0), (5, 17, 3, 0), (999_999, 1200, 63, 7), ((1 << 33) + 5, 2, 9, 1 << 40)]:
        w = oracle.philox4x32_10([t & 0xFFFFFFFF, k, e, t >> 32], [s & 0xFFFFFFFF, s >> 32])
        u = oracle.uniform(s, t, k, e)
        assert u == ((int(w[0]) >> 9) + 0.5) / 2.0**23
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u  # exact in FP32, so FP32 and FP64 invert the same z


def test_uniform_extremes_are_exact_complements():
    # the smallest and largest values of the mapping and their complements
    lo = 0.5 / 2.0**23
    hi = (2.0**23 - 0.5) / 2.0**23
    assert float(np.float32(1.0 - hi)) == 1.0 - hi == lo


def test_uniform_statistics():
    rng = np.random.default_rng(5)
    n = 400_000
    trials = rng.integers(0, 1_000_000, size=n)
    ks = rng.integers(0, 1500, size=n).astype(np.int32)
    elts = rng.integers(0, 64, size=n).astype(np.int32)
    u = oracle.uniform_batch(0, trials, ks, elts)
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    counts = np.histogram(u, bins=256, range=(0.0, 1.0))[0]
    assert stats.chisquare(counts).pvalue > 1e-4
    # neighbouring ELT keys and neighbouring event indices are uncorrelated
    u0 = oracle.uniform_batch(0, trials, ks, np.zeros(n, np.int32))
    u1 = oracle.uniform_batch(0, trials, ks, np.ones(n, np.int32))
    u2 = oracle.uniform_batch(0, trials, ks + 1, np.zeros(n, np.int32))
    u3 = oracle.uniform_batch(1, trials, ks, np.zeros(n, np.int32))
    bound = 5.0 / np.sqrt(n)
    for other in (u1, u2, u3):
        assert abs(np.corrcoef(u0, other)[0, 1]) < bound


def test_uniform_depends_on_every_key_component():
    base = oracle.uniform(3, 10, 4, 2)
    assert oracle.uniform(4, 10, 4, 2) != base
    assert oracle.uniform(3, 11, 4, 2) != base
    assert oracle.uniform(3, 10, 5, 2) != base
    assert oracle.uniform(3, 10, 4, 3) != base
    assert oracle.uniform(3, 10 + (1 << 32), 4, 2) != base
    assert oracle.uniform(3 + (1 << 32), 10, 4, 2) != base
