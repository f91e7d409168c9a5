"""Pins of the oracle's Matern covariance (paper Sec. III-B)."""
import math

import numpy as np
import pytest
from scipy.special import gamma, kv

from oracle import matern
from golden_values import load

G = load("closed_forms.txt")


@pytest.mark.parametrize("nu,l", [(1.5, 1.5), (1.5, 2.0), (2.5, 0.7), (2.5, 1.5)])
def test_unit_variance_at_zero(nu, l):
    assert matern(0.0, nu, l) == 1.0


def test_closed_form_points():
    l = 1.5
    assert matern(l / math.sqrt(3), 1.5, l) == pytest.approx(float(G["matern32_t1"]), rel=1e-15)
    assert matern(l / math.sqrt(5), 2.5, l) == pytest.approx(float(G["matern52_t1"]), rel=1e-15)
    assert matern(2 * l / math.sqrt(3), 1.5, l) == pytest.approx(float(G["matern32_t2"]), rel=1e-15)
    assert matern(3 * l / math.sqrt(5), 2.5, l) == pytest.approx(float(G["matern52_t3"]), rel=1e-15)


def bessel_matern(r, nu, l):
    """General Matern family, k(r) = 2^(1-nu)/Gamma(nu) t^nu K_nu(t), t = sqrt(2 nu) r / l."""
    t = math.sqrt(2 * nu) * np.asarray(r) / l
    return 2 ** (1 - nu) / gamma(nu) * t ** nu * kv(nu, t)


@pytest.mark.parametrize("nu", [1.5, 2.5])
@pytest.mark.parametrize("l", [0.5, 1.5, 2.0])
def test_equals_bessel_form(nu, l):
    r = np.linspace(1e-3, 6.0, 400)
    np.testing.assert_allclose(matern(r, nu, l), bessel_matern(r, nu, l), rtol=1e-12, atol=1e-300)


def test_monotone_decreasing_and_positive():
    r = np.linspace(0, 10, 1001)
    for nu in (1.5, 2.5):
        k = matern(r, nu, 1.5)
        assert np.all(np.diff(k) < 0) and np.all(k > 0)


def test_matches_sklearn_kernel():
    skl = pytest.importorskip("sklearn.gaussian_process.kernels")
    rng = np.random.default_rng(3)
    X = rng.uniform(size=(9, 4))
    for nu, l in ((1.5, 1.5), (2.5, 0.8)):
        Ksk = skl.Matern(length_scale=l, nu=nu)(X)
        d = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
        np.testing.assert_allclose(matern(d, nu, l), Ksk, rtol=1e-13, atol=1e-15)


def test_rejects_other_nu():
    with pytest.raises(ValueError):
        matern(1.0, 0.5, 1.0)
