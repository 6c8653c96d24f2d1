"""Pins of the oracle's two-sigma secondary uncertainty (Section 3.1 inputs,
Section 3.2 five-step combination): the normal CDF and quantile, the two
extreme cases the model names (sigma_C = 0: z = z_(Prog,E); sigma_I = 0:
z = z_(E), shared by all ELTs of an occurrence), and the distribution of the
combined normal (Monte Carlo)."""

import math

import numpy as np
import pytest

import oracle
from paper_1501_06326_gb300 import synth


def test_normal_cdf_closed_values():
    assert oracle.normcdf(0.0) == 0.5
    assert abs(oracle.normcdf(1.959963984540054) - 0.975) < 1e-15
    assert abs(oracle.normcdf(-1.0) - 0.15865525393145707) < 1e-16
    for v in (-5.0, -1.3, 0.7, 4.2):
        assert abs(oracle.normcdf(v) + oracle.normcdf(-v) - 1.0) < 1e-15


def test_normal_quantile_round_trip_and_library_pin():
    # the lower half round-trips to FP64 resolution (above 1/2, 1 - Phi(v) is not
    # representable near 1, which is why the oracle carries the complement Phi(-v))
    v = np.linspace(-5.3, 0.0, 201)
    p = np.array([oracle.normcdf(x) for x in v])
    back = oracle.normcdfinv_batch(p)
    assert np.max(np.abs(back - v)) < 1e-12
    # on the uniform grid 1 - p is exact, and the quantile is odd about 1/2
    g = (np.arange(0, 1 << 23, 4099) + 0.5) / 2.0**23
    assert np.array_equal(oracle.normcdfinv_batch(1.0 - g), -oracle.normcdfinv_batch(g))
    special = pytest.importorskip("scipy.special")
    z = (np.arange(1, 2000) + 0.5) / 2000.0
    assert np.allclose(oracle.normcdfinv_batch(z), special.ndtri(z), rtol=1e-13, atol=1e-13)


def _tiny(corr_split):
    yet = synth.make_yet(300, 40.0, 2000, 91)
    pool = synth.make_elt_pool(2, 600, 2000, 92, correlated=0.5)
    if corr_split == "independent":
        pool.sigma_c = np.zeros_like(pool.sigma_c)
    return yet, pool


def test_sigma_c_zero_is_the_independent_model():
    yet, pool = _tiny("independent")
    terms = (0.0, math.inf, 0.0, math.inf)
    plain = synth.ELTPool(pool.elt_ids, pool.rec_offsets, pool.event_ids, pool.mean, pool.sigma, pool.exposure,
                          pool.terms)
    a = oracle.run_layer(yet, pool, terms, seed=4)
    b = oracle.run_layer(yet, plain, terms, seed=4)
    assert np.array_equal(a["ylt"], b["ylt"])


def test_sigma_i_zero_makes_the_elts_of_an_occurrence_share_their_uniform():
    # two ELTs with identical records and sigma_I = 0: every occurrence draws the
    # same z_(E) for both, so each event's loss is exactly twice one ELT's
    yet = synth.make_yet(300, 40.0, 2000, 93)
    one = synth.make_elt_pool(1, 600, 2000, 94)
    sc = one.sigma.copy()
    zero = np.zeros_like(sc)
    cat = lambda a: np.concatenate([a, a])
    two = synth.ELTPool(np.array([0, 1], np.int32), np.array([0, 600, 1200], np.int64), cat(one.event_ids),
                        cat(one.mean), cat(zero), cat(one.exposure), np.tile(one.terms, (2, 1)), cat(sc))
    single = synth.ELTPool(one.elt_ids, one.rec_offsets, one.event_ids, one.mean, zero, one.exposure, one.terms, sc)
    terms = (0.0, math.inf, 0.0, math.inf)
    y2 = oracle.run_layer(yet, two, terms, seed=8)["ylt"]
    y1 = oracle.run_layer(yet, single, terms, seed=8)["ylt"]
    assert np.array_equal(y2, 2.0 * y1)
    # with sigma_C = 0 instead, the two ELTs draw independently
    indep = synth.ELTPool(two.elt_ids, two.rec_offsets, two.event_ids, two.mean, cat(sc), two.exposure, two.terms)
    assert not np.array_equal(oracle.run_layer(yet, indep, terms, seed=8)["ylt"], 2.0 * y1)


@pytest.mark.parametrize("s_i,s_c", [(1.0, 1.0), (0.6, 0.8), (0.3, 0.05)])
def test_combined_normal_distribution(s_i, s_c):
    n = 200_000
    rng = np.random.default_rng(5)
    t = rng.integers(0, 1 << 40, n)
    k = rng.integers(0, 5000, n).astype(np.int32)
    v1, z1 = oracle.combined_normal_batch(11, t, k, np.full(n, 3, np.int32), s_i, s_c)
    v2, _ = oracle.combined_normal_batch(11, t, k, np.full(n, 7, np.int32), s_i, s_c)
    se = 1.0 / math.sqrt(n)
    assert abs(v1.mean()) < 5 * se and abs(v1.var() - 1.0) < 10 * se
    rho = s_c * s_c / (s_i * s_i + s_c * s_c)  # shared z_(E), independent z_(Prog,E)
    assert abs(np.corrcoef(v1, v2)[0, 1] - rho) < 5 * se
    # z = Phi(v) is uniform (Kolmogorov-Smirnov distance)
    zs = np.sort(z1)
    ks = np.max(np.abs(zs - (np.arange(1, n + 1) - 0.5) / n))
    assert ks < 1.63 / math.sqrt(n)


def test_event_uniform_is_a_separate_stream():
    zs = [oracle.uniform_event(2, t, k) for t in range(40) for k in range(5)]
    zp = [oracle.uniform(2, t, k, 0) for t in range(40) for k in range(5)]
    assert len(set(zs)) == len(zs) and not set(zs) & set(zp)


Q_GRID = (0.9, 0.5, 0.1, 1e-3, 1e-7, 1e-12)


@pytest.mark.parametrize("q", Q_GRID)
def test_upper_tail_quantile_closed_forms(q):
    # 1 - I_x(a, 1) = 1 - x^a = q  =>  x = (1 - q)^(1/a)
    for a in (0.3, 1.0, 7.5):
        assert abs(oracle.betaincinv_upper(q, a, 1.0) - math.exp(math.log1p(-q) / a)) <= 1e-12
    # 1 - I_x(1, b) = (1 - x)^b = q  =>  x = 1 - q^(1/b)
    for b in (0.3, 1.0, 7.5):
        assert abs(oracle.betaincinv_upper(q, 1.0, b) + math.expm1(math.log(q) / b)) <= 1e-12
    # arcsine law: I_x(1/2, 1/2) = (2 / pi) asin(sqrt(x))  =>  x = cos^2(pi q / 2)
    assert abs(oracle.betaincinv_upper(q, 0.5, 0.5) - math.cos(math.pi * q / 2.0) ** 2) <= 1e-12


@pytest.mark.parametrize("s_i,s_c", [(300.0, 100.0), (200.0, 200.0), (0.0, 400.0), (50.0, 350.0)])
def test_correlated_record_loss_against_library_routines(s_i, s_c):
    # one record (mean 1000, exposure 4000, sigma = s_i + s_c) hit once per trial:
    # each year loss is max_l InvCDF_beta(Phi(v)), v the combined normal of the
    # record's and the occurrence's uniforms (Section 3.2), here from SciPy's
    # normal and Beta inverses (the upper half by the complemented inverse)
    special = pytest.importorskip("scipy.special")
    n, seed = 3000, 17
    yet = synth.YET(np.arange(n + 1, dtype=np.int64), np.zeros(n, np.int32), 4)
    pool = synth.ELTPool(np.array([5], np.int32), np.array([0, 1], np.int64), np.array([0], np.int32),
                         np.array([1000.0], np.float32), np.array([s_i], np.float32), np.array([4000.0], np.float32),
                         np.array([[0.0, np.inf, 1.0]], np.float32), np.array([s_c], np.float32))
    got = oracle.run_layer(yet, pool, (0.0, math.inf, 0.0, math.inf), seed=seed)["ylt"]
    t = np.arange(n, dtype=np.int64)
    k = np.zeros(n, np.int32)
    vp = special.ndtri(oracle.uniform_batch(seed, t, k, np.full(n, 5, np.int32)))
    ve = special.ndtri(oracle.uniform_batch(seed, t, k, np.full(n, -1, np.int32)))
    v = (s_i * vp + s_c * ve) / math.hypot(s_i, s_c)
    _, a, b = oracle.beta_params(1000.0, s_i + s_c, 4000.0)
    x = np.where(v <= 0.0, special.betaincinv(a, b, special.ndtr(v)), special.betainccinv(a, b, special.ndtr(-v)))
    assert np.sum(v > 0.0) > n // 3 and np.sum(v < 0.0) > n // 3
    assert np.allclose(got, 4000.0 * x, rtol=1e-9, atol=0.0)


def test_shared_z_keys_every_elt_by_the_occurrence():
    # Beta(1,1) records (mu/max = 1/2, sigma^2/max^2 = 1/12) have Loss = max z: with one
    # event per trial the year loss is max z, and z is the occurrence's shared draw
    n, seed = 200, 9
    max_l = 1000.0
    yet = synth.YET(np.arange(n + 1, dtype=np.int64), np.full(n, 2, np.int32), 4)
    pool = synth.ELTPool(np.array([3, 8], np.int32), np.array([0, 1, 2], np.int64), np.array([2, 2], np.int32),
                         np.full(2, 500.0, np.float32), np.full(2, max_l / math.sqrt(12.0), np.float32),
                         np.full(2, max_l, np.float32), np.tile(np.array([0.0, np.inf, 1.0], np.float32), (2, 1)))
    terms = (0.0, math.inf, 0.0, math.inf)
    z = oracle.uniform_batch(seed, np.arange(n, dtype=np.int64), np.zeros(n, np.int32),
                             np.full(n, oracle.SHARED_Z_WORD, np.int32))
    one = oracle.run_layer(yet, pool.subset([0]), terms, seed=seed, shared_z=True)["ylt"]
    assert np.allclose(one, max_l * z, rtol=1e-6, atol=0.0)  # shapes 1 up to the FP32 sigma
    # both ELTs draw the same z: the year loss doubles exactly; without the flag it does not
    two = oracle.run_layer(yet, pool, terms, seed=seed, shared_z=True)["ylt"]
    assert np.array_equal(two, 2.0 * one)
    indep = oracle.run_layer(yet, pool, terms, seed=seed)["ylt"]
    assert not np.allclose(indep, two, rtol=1e-3)
    # the shared word is outside the pool-id range and apart from the occurrence stream of sigma_C
    assert oracle.SHARED_Z_WORD < 0
    assert oracle.uniform(seed, 5, 0, oracle.SHARED_Z_WORD) != oracle.uniform_event(seed, 5, 0)
