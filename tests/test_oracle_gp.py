"""Pins of the oracle's GP posterior (paper Sec. III-B, III-G)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import gp_fit, gp_posterior, matern, predict, standardize


def exact_inverse(A):
    """Gauss-Jordan elimination over the rationals (exact for fp64 inputs)."""
    n = len(A)
    M = [[Fraction(float(A[i][j])) for j in range(n)] + [Fraction(int(i == j)) for j in range(n)]
         for i in range(n)]
    for c in range(n):
        p = max(range(c, n), key=lambda r: abs(M[r][c]))
        M[c], M[p] = M[p], M[c]
        piv = M[c][c]
        M[c] = [v / piv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return [row[n:] for row in M]


def brute_posterior(X, yt, Xc, nu, l, jitter):
    """mu = k*^T K^-1 y~, var = 1 - k*^T K^-1 k*, K^-1 exact, sums in rationals."""
    n = len(X)
    dist = lambda a, b: float(np.sqrt(np.sum((a - b) ** 2)))
    K = [[float(matern(dist(X[i], X[j]), nu, l)) + (jitter if i == j else 0.0)
          for j in range(n)] for i in range(n)]
    Ki = exact_inverse(K)
    ytq = [Fraction(float(v)) for v in yt]
    mus, vars_ = [], []
    for c in Xc:
        ks = [Fraction(float(matern(dist(c, X[j]), nu, l))) for j in range(n)]
        w = [sum(Ki[i][j] * ks[j] for j in range(n)) for i in range(n)]   # K^-1 k*
        mus.append(float(sum(w[i] * ytq[i] for i in range(n))))
        vars_.append(float(1 - sum(w[i] * ks[i] for i in range(n))))
    return np.array(mus), np.array(vars_)


@pytest.mark.parametrize("d,n,nu,l,seed", [(2, 5, 1.5, 1.5, 0), (3, 7, 2.5, 0.8, 1),
                                           (1, 4, 1.5, 2.0, 2), (3, 8, 1.5, 1.5, 3)])
def test_matches_exact_rational_inverse(d, n, nu, l, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(size=(n, d))
    y = rng.uniform(1, 3, size=n)
    Xc = rng.uniform(size=(12, d))
    jitter = 1e-6
    mu, var, fit = predict(X, y, Xc, nu, l, jitter)
    bmu, bvar = brute_posterior(X, fit.ytilde, Xc, nu, l, jitter)
    np.testing.assert_allclose(mu, bmu, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(var, np.maximum(bvar, 0), rtol=1e-7, atol=1e-10)


def test_matches_sklearn_gpr():
    gpm = pytest.importorskip("sklearn.gaussian_process")
    kern = pytest.importorskip("sklearn.gaussian_process.kernels")
    rng = np.random.default_rng(7)
    X = rng.uniform(size=(30, 4))
    y = rng.uniform(1, 5, size=30)
    Xc = rng.uniform(size=(200, 4))
    for nu, l, jit in ((1.5, 1.5, 1e-10), (2.5, 0.9, 1e-8)):
        mu, var, fit = predict(X, y, Xc, nu, l, jit)
        gpr = gpm.GaussianProcessRegressor(
            kernel=kern.Matern(length_scale=l, nu=nu, length_scale_bounds="fixed"),
            alpha=jit, optimizer=None, normalize_y=False)
        gpr.fit(X, fit.ytilde)
        smu, sstd = gpr.predict(Xc, return_std=True)
        np.testing.assert_allclose(mu, smu, rtol=1e-7, atol=1e-8)
        np.testing.assert_allclose(np.sqrt(var), sstd, rtol=1e-6, atol=1e-7)


def test_interpolates_noiseless_observations():
    rng = np.random.default_rng(11)
    X = rng.uniform(size=(25, 3))
    y = rng.uniform(1, 2, size=25)
    mu, var, fit = predict(X, y, X, 1.5, 1.5, 1e-10)
    np.testing.assert_allclose(mu, fit.ytilde, atol=1e-6)
    assert np.all(var <= 1e-6)


def test_variance_bounds_and_shrinks_with_data():
    rng = np.random.default_rng(12)
    X = rng.uniform(size=(20, 3))
    y = rng.uniform(1, 2, size=20)
    Xc = rng.uniform(size=(300, 3))
    _, v1, _ = predict(X[:10], y[:10], Xc)
    _, v2, _ = predict(X, y, Xc)
    assert np.all((v1 >= 0) & (v1 <= 1)) and np.all((v2 >= 0) & (v2 <= 1))
    assert np.all(v2 <= v1 + 1e-9)


def test_far_from_data_reverts_to_prior():
    X = np.array([[0.0, 0.0]])
    y = np.array([3.0])
    fit = gp_fit(X, y, 1.5, 0.05, 1e-10, normalize_y=False)
    mu, var = gp_posterior(fit, np.array([[1.0, 1.0]]))
    assert abs(mu[0]) < 1e-9 and abs(var[0] - 1.0) < 1e-9


def test_standardize():
    yt, m, s = standardize([1.0, 2.0, 3.0, 6.0])
    assert m == 3.0 and s == pytest.approx(np.sqrt(3.5))
    assert np.mean(yt) == pytest.approx(0.0, abs=1e-15) and np.std(yt) == pytest.approx(1.0)
    yt, m, s = standardize([2.0, 2.0])
    assert s == 1.0 and np.all(yt == 0)


def test_single_observation_posterior():
    """One point: mu(c) = k(r) y~, var(c) = 1 - k(r)^2 / (1 + jitter)."""
    X = np.array([[0.2, 0.4]])
    y = np.array([5.0])
    jit = 1e-4
    fit = gp_fit(X, y, 2.5, 1.0, jit, normalize_y=False)
    Xc = np.array([[0.5, 0.1], [0.2, 0.4]])
    mu, var = gp_posterior(fit, Xc)
    r = np.sqrt(((Xc - X) ** 2).sum(1))
    t = np.sqrt(5) * r
    k = (1 + t + t * t / 3) * np.exp(-t)
    np.testing.assert_allclose(mu, k * 5.0 / (1 + jit), rtol=1e-12)
    np.testing.assert_allclose(var, 1 - k * k / (1 + jit), rtol=1e-10, atol=1e-15)
