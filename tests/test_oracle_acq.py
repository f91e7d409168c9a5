"""Pins of the oracle's acquisition functions (Sec. III-C) and lambda (Sec. III-F)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import (contextual_variance_lambda, expected_improvement, masked_argmax,
                    masked_topk, negative_lcb, probability_of_improvement)
from golden_values import load

G = load("closed_forms.txt")


def test_closed_form_values():
    ei = lambda d, s: float(expected_improvement(0.0, s, d, 0.0))
    pi = lambda d, s: float(probability_of_improvement(0.0, s, d, 0.0))
    assert ei(0.0, 1.0) == pytest.approx(float(G["ei_delta0_sigma1"]), rel=1e-15)
    assert pi(0.0, 1.0) == float(G["pi_delta0_sigma1"])
    assert ei(1.0, 1.0) == pytest.approx(float(G["ei_delta1_sigma1"]), rel=1e-15)
    assert pi(1.0, 1.0) == pytest.approx(float(G["pi_delta1_sigma1"]), rel=1e-15)
    assert ei(0.5, 2.0) == pytest.approx(float(G["ei_delta0.5_sigma2"]), rel=1e-15)


@pytest.mark.parametrize("mu,sigma,fplus,lam", [(0.3, 0.7, 0.1, 0.05), (-1.2, 0.2, -1.0, 0.0),
                                                (2.0, 1.5, -0.5, 0.3), (0.0, 0.05, 0.02, 0.01)])
def test_definitions_by_integration(mu, sigma, fplus, lam):
    """EI = E[max(f+ - lam - g, 0)], PI = P(g <= f+ - lam), g ~ N(mu, sigma^2)."""
    pdf = lambda g: math.exp(-0.5 * ((g - mu) / sigma) ** 2) / (sigma * math.sqrt(2 * math.pi))
    thr = fplus - lam
    ei_q, _ = integrate.quad(lambda g: (thr - g) * pdf(g), mu - 40 * sigma, thr,
                             epsabs=1e-14, epsrel=1e-12)
    pi_q, _ = integrate.quad(pdf, mu - 40 * sigma, thr, epsabs=1e-14, epsrel=1e-12)
    assert float(expected_improvement(mu, sigma, fplus, lam)) == pytest.approx(max(ei_q, 0), rel=1e-8, abs=1e-14)
    assert float(probability_of_improvement(mu, sigma, fplus, lam)) == pytest.approx(max(pi_q, 0), rel=1e-8, abs=1e-14)


def test_exploration_offset_and_limits():
    mu, s = np.array([0.1, -0.4, 0.9]), np.array([0.3, 0.5, 0.01])
    np.testing.assert_allclose(expected_improvement(mu, s, 0.2, 0.15),
                               expected_improvement(mu + 0.15, s, 0.2, 0.0), rtol=1e-14)
    # sigma -> 0: EI -> max(delta, 0), PI -> step
    assert float(expected_improvement(0.0, 0.0, 0.3, 0.1)) == pytest.approx(0.2)
    assert float(expected_improvement(0.0, 0.0, 0.1, 0.3)) == 0.0
    assert float(probability_of_improvement(0.0, 0.0, 0.3, 0.1)) == 1.0
    assert float(probability_of_improvement(0.0, 0.0, 0.1, 0.3)) == 0.0
    assert float(expected_improvement(0.0, 1e-9, 0.3, 0.1)) == pytest.approx(0.2, rel=1e-9)
    # larger exploration offset never raises EI or PI
    for lam in (0.0, 0.1, 1.0):
        assert np.all(expected_improvement(mu, s, 0.2, lam + 0.1) <= expected_improvement(mu, s, 0.2, lam))


def test_negative_lcb():
    np.testing.assert_allclose(negative_lcb([1.0, -2.0], [0.5, 2.0], 0.3), [-0.85, 2.6], rtol=1e-15)


def test_contextual_variance():
    # at the first pass the mean variance equals its baseline: lambda = f+/mu_s
    assert contextual_variance_lambda(0.37, 2.0, 5.0, 0.37) == pytest.approx(0.4, rel=1e-15)
    base = contextual_variance_lambda(0.2, 1.5, 3.0, 0.5)
    assert contextual_variance_lambda(0.4, 1.5, 3.0, 0.5) == pytest.approx(2 * base)
    assert contextual_variance_lambda(0.2, 3.0, 3.0, 0.5) == pytest.approx(2 * base)
    assert contextual_variance_lambda(0.2, 1.5, 6.0, 0.5) == pytest.approx(base / 2)
    with pytest.raises(ValueError):
        contextual_variance_lambda(0.2, -1.0, 3.0, 0.5)
    with pytest.raises(ValueError):
        contextual_variance_lambda(0.2, 1.0, 0.0, 0.5)


def test_masked_argmax_and_topk_brute_force():
    rng = np.random.default_rng(5)
    for trial in range(200):
        n = int(rng.integers(1, 40))
        s = rng.integers(0, 6, size=n).astype(float)       # many ties
        m = rng.uniform(size=n) < 0.7
        best, bi = -math.inf, -1
        for i in range(n):
            if m[i] and s[i] > best:
                best, bi = s[i], i
        assert masked_argmax(s, m) == bi
        ref = sorted([(-s[i], i) for i in range(n) if m[i]])[:3]
        assert masked_topk(s, m, 3) == [(i, -v) for v, i in ref]
