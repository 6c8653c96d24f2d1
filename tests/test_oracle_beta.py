"""Pins of the oracle's Beta machinery (Section 3.3: Beta parameters from the
XELT record, the sigma clip, and Loss = max_l * InvCDF_beta(z; alpha, beta)).

Closed forms of the Beta quantile, integer-shape binomial sums of the
regularised incomplete Beta, round trips, SciPy's betaincinv (a library pin,
test-only) and Monte Carlo moments of the secondary-uncertainty loss.
"""

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

P_GRID = [0.5 / 2**23, 1e-6, 1e-3, 0.01, 0.1, 0.25, 0.5, 0.75, 0.9, 0.99, 1 - 1e-6, 1 - 0.5 / 2**23]
SHAPES = [0.05, 0.2, 0.5, 0.9, 2.0, 7.5, 50.0, 400.0]


def _close(x, y, rel):
    return abs(x - y) <= rel * max(abs(y), 1e-300)


@pytest.mark.parametrize("p", P_GRID)
def test_uniform_beta_is_identity(p):
    assert _close(oracle.betaincinv(p, 1.0, 1.0), p, 1e-13)


@pytest.mark.parametrize("a", SHAPES)
@pytest.mark.parametrize("p", P_GRID)
def test_beta_a1_closed_form(a, p):
    # I_x(a, 1) = x^a, so the quantile is p^(1/a)
    want = p ** (1.0 / a)
    got = oracle.betaincinv(p, a, 1.0)
    if want > 0.5:  # compare the small side: 1 - x
        assert _close(oracle.betaincinv_complement(p, a, 1.0), -math.expm1(math.log(p) / a), 1e-10)
    else:
        assert _close(got, want, 1e-10)


@pytest.mark.parametrize("b", SHAPES)
@pytest.mark.parametrize("p", P_GRID)
def test_beta_1b_closed_form(b, p):
    # I_x(1, b) = 1 - (1 - x)^b, so the quantile is 1 - (1 - p)^(1/b)
    want = -math.expm1(math.log1p(-p) / b)
    got = oracle.betaincinv(p, 1.0, b)
    if want > 0.5:
        assert _close(oracle.betaincinv_complement(p, 1.0, b), (1.0 - p) ** (1.0 / b), 1e-10)
    else:
        assert _close(got, want, 1e-10)


@pytest.mark.parametrize("p", P_GRID)
def test_arcsine_closed_form(p):
    # Beta(1/2, 1/2) is the arcsine law: I_x = (2/pi) asin(sqrt(x)), quantile sin^2(pi p / 2)
    want = math.sin(math.pi * p / 2.0) ** 2
    got = oracle.betaincinv(p, 0.5, 0.5)
    if want > 0.5:
        # 1 - sin^2(pi p / 2) = sin^2(pi (1 - p) / 2), evaluated without cancellation
        assert _close(oracle.betaincinv_complement(p, 0.5, 0.5), math.sin(math.pi * (1.0 - p) / 2.0) ** 2, 1e-10)
    else:
        assert _close(got, want, 1e-10)


@pytest.mark.parametrize("a,b", [(1, 1), (2, 3), (5, 2), (7, 7), (1, 9), (12, 4), (20, 30)])
@pytest.mark.parametrize("x", ["1/1000", "1/7", "1/2", "3/5", "9/10", "999/1000"])
def test_integer_shapes_binomial_sum(a, b, x):
    # For integer a, b: I_x(a, b) = sum_{j=a}^{a+b-1} C(a+b-1, j) x^j (1-x)^(a+b-1-j)
    xf = Fraction(x)
    n = a + b - 1
    exact = sum(math.comb(n, j) * xf**j * (1 - xf) ** (n - j) for j in range(a, n + 1))
    got = oracle.betainc(float(xf), float(a), float(b))
    assert _close(got, float(exact), 1e-12)


def test_betainc_symmetry_and_limits():
    for a, b in [(0.3, 4.0), (2.5, 0.7), (40.0, 60.0)]:
        for x in [1e-4, 0.3, 0.5, 0.8, 0.9999]:
            assert abs(oracle.betainc(x, a, b) + oracle.betainc(1 - x, b, a) - 1.0) < 1e-13
        assert oracle.betainc(0.0, a, b) == 0.0
        assert oracle.betainc(1.0, a, b) == 1.0


def test_round_trip():
    rng = np.random.default_rng(11)
    n = 4000
    a = np.exp(rng.uniform(math.log(0.05), math.log(2000), n))
    b = np.exp(rng.uniform(math.log(0.05), math.log(2000), n))
    p = (rng.integers(0, 1 << 23, n) + 0.5) / 2**23
    x = oracle.betaincinv_batch(p, a, b)
    for i in range(n):
        if x[i] <= 0.5:
            back, target = oracle.betainc(x[i], a[i], b[i]), p[i]
        else:  # roots above 1/2 are checked on their complement: I_{1-x}(b, a) = 1 - p
            y = oracle.betaincinv_complement(p[i], a[i], b[i])
            back, target = oracle.betainc(y, b[i], a[i]), 1.0 - p[i]
        # the forward evaluation carries the lgamma cancellation of ln B(a, b) (~1e-12 at shape 2000)
        assert abs(back - target) <= 1e-10 * target, (a[i], b[i], p[i])


def test_scipy_betaincinv_library_pin():
    special = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(3)
    n = 6000
    a = np.exp(rng.uniform(math.log(0.05), math.log(2000), n))
    b = np.exp(rng.uniform(math.log(0.05), math.log(2000), n))
    p = (rng.integers(0, 1 << 23, n) + 0.5) / 2**23
    x = oracle.betaincinv_batch(p, a, b)
    ref = special.betaincinv(a, b, p)
    lower = ref <= 0.5
    # roots below 1/2: relative agreement; above 1/2 both sides are doubles near 1
    assert np.all(np.abs(x[lower] - ref[lower]) <= 1e-8 * ref[lower])
    assert np.all(np.abs(x[~lower] - ref[~lower]) <= 1e-8 * (1.0 - ref[~lower]) + 4e-16)


# --------------------------------------------------------------- Beta parameters
def test_beta_params_uniform_special_case():
    # mu_b = 1/2 and sigma_b^2 = 1/12 give alpha = beta = 1 (the uniform law)
    max_l = 1000.0
    kind, a, b = oracle.beta_params(500.0, max_l / math.sqrt(12.0), max_l)
    assert kind == 0
    assert _close(a, 1.0, 1e-12) and _close(b, 1.0, 1e-12)


@pytest.mark.parametrize("mu,sigma,max_l", [(10.0, 3.0, 40.0), (1e5, 2e4, 1.5e6), (2.0, 0.1, 2.5)])
def test_beta_params_reproduce_mean_and_variance(mu, sigma, max_l):
    kind, a, b = oracle.beta_params(mu, sigma, max_l)
    assert kind == 0
    m = a / (a + b)
    v = a * b / ((a + b) ** 2 * (a + b + 1.0))
    assert _close(max_l * m, mu, 1e-13)
    assert _close(max_l * math.sqrt(v), sigma, 1e-12)


def test_beta_params_sigma_clip():
    mu, max_l = 30.0, 100.0
    s_max = max_l * math.sqrt(0.3 * 0.7)
    kind, a, b = oracle.beta_params(mu, 2.0 * s_max, max_l)
    assert kind == 0
    k = 1.0 / (1.0 - 1e-6) ** 2 - 1.0
    assert _close(a + b, k, 1e-8) and _close(a / (a + b), 0.3, 1e-12)


def test_beta_params_degenerate_and_invalid():
    assert oracle.beta_params(0.0, 5.0, 10.0)[0] == 1
    assert oracle.beta_params(5.0, 0.0, 10.0)[0] == 1
    assert oracle.beta_params(10.0, 1.0, 10.0)[0] == -1  # max_l must exceed mu
    assert oracle.beta_params(-1.0, 1.0, 10.0)[0] == -1
    assert oracle.beta_params(float("nan"), 1.0, 10.0)[0] == -1


@pytest.mark.parametrize("mu,sigma,max_l", [(100.0, 40.0, 400.0), (50.0, 45.0, 120.0)])
def test_monte_carlo_moments_of_the_loss(mu, sigma, max_l):
    # Loss = max_l * InvCDF(z; alpha, beta) with z ~ U(0,1) has mean mu and s.d. sigma
    kind, a, b = oracle.beta_params(mu, sigma, max_l)
    assert kind == 0
    n = 40_000
    rng = np.random.default_rng(17)
    z = (rng.integers(0, 1 << 23, n) + 0.5) / 2**23
    loss = max_l * oracle.betaincinv_batch(z, a, b)
    se = sigma / math.sqrt(n)
    assert abs(loss.mean() - mu) < 4.0 * se
    # variance of the sample variance ~ (m4 - s^4) / n; a 5% band is > 4 s.e. here
    assert abs(loss.std() / sigma - 1.0) < 0.05
