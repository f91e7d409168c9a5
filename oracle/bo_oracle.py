"""FP64 oracle: search space, Matern covariance, GP posterior, acquisition.

Test infrastructure only (see the package docstring).  Everything here is the
plain definition written out; library primitives (numpy/scipy Cholesky,
triangular solve, pairwise Euclidean distance, erfc) serve as single steps.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import cholesky, solve_triangular
from scipy.spatial.distance import cdist
from scipy.special import erfc

__all__ = [
    "valid_list", "candidate_coords", "matern", "standardize", "GPFit", "gp_fit",
    "gp_posterior", "predict", "phi_pdf", "Phi_cdf", "expected_improvement",
    "probability_of_improvement", "negative_lcb", "acquisition",
    "contextual_variance_lambda", "masked_argmax", "masked_topk", "AF_NAMES",
]

AF_NAMES = ("ei", "poi", "lcb")


# --- Sec. III-D (general structure): the discrete, normalized, constrained space

def valid_list(sizes, invalid_mask=None):
    """Valid configurations of the Cartesian product of the parameter lists.

    Sec. III-D: the search space is discrete and normalized; restricted
    configurations are removed before optimization.  The product is
    enumerated row-major, last parameter fastest.  Returns (flat indices,
    codes) where codes[i, p] is the value index of parameter p.
    """
    total = int(np.prod(sizes, dtype=np.int64))
    flat = np.arange(total, dtype=np.int64)
    if invalid_mask is not None:
        flat = flat[np.asarray(invalid_mask).reshape(-1) == 0]
    codes = np.stack(np.unravel_index(flat, tuple(int(s) for s in sizes)), axis=1)
    return flat, codes


def candidate_coords(grids, codes):
    """Normalized coordinates x[i, p] = grids[p][codes[i, p]] (Sec. III-D)."""
    codes = np.asarray(codes)
    return np.stack([np.asarray(grids[p], dtype=np.float64)[codes[:, p]]
                     for p in range(codes.shape[1])], axis=1)


# --- Sec. III-B: Matern covariance with fixed lengthscale

def matern(r, nu, lengthscale):
    """Matern covariance k(r) for nu = 3/2 or 5/2 (Sec. III-B).

    The half-integer forms are a polynomial times an exponential in
    t = sqrt(2 nu) r / l with r the Euclidean distance:
        nu = 3/2:  (1 + t) exp(-t)
        nu = 5/2:  (1 + t + t^2 / 3) exp(-t)
    (t^2/3 = 5 r^2 / (3 l^2) for nu = 5/2.)  Unit signal variance: k(0) = 1.
    """
    r = np.asarray(r, dtype=np.float64)
    t = math.sqrt(2.0 * nu) * r / lengthscale
    if nu == 1.5:
        return (1.0 + t) * np.exp(-t)
    if nu == 2.5:
        return (1.0 + t + t * t / 3.0) * np.exp(-t)
    raise ValueError("nu must be 1.5 or 2.5")


# --- Sec. III-B / III-G: zero-mean GP regression on the observations

def standardize(y):
    """Zero mean, unit (population) standard deviation; std 0 is treated as 1."""
    y = np.asarray(y, dtype=np.float64)
    mean = float(np.mean(y))
    std = float(np.std(y))
    if std == 0.0:
        std = 1.0
    return (y - mean) / std, mean, std


class GPFit:
    """Cholesky factor L of K(X, X) + jitter I and alpha = K^-1 y~."""

    def __init__(self, X, ytilde, nu, lengthscale, jitter, L, alpha, y_mean, y_std):
        self.X, self.ytilde = X, ytilde
        self.nu, self.lengthscale, self.jitter = nu, lengthscale, jitter
        self.L, self.alpha = L, alpha
        self.y_mean, self.y_std = y_mean, y_std


def gp_fit(X, y, nu, lengthscale, jitter=1e-10, normalize_y=True):
    """Fit the zero-mean GP with a fixed-lengthscale Matern kernel (Sec. III-B).

    Only valid observations are passed in (Sec. III-D: runtime-invalid
    configurations are not fitted).  K = k(||x_i - x_j||) + jitter on the
    diagonal; L = chol(K); alpha = K^-1 y~ by two triangular solves.
    """
    X = np.asarray(X, dtype=np.float64)
    if normalize_y:
        yt, mean, std = standardize(y)
    else:
        yt, mean, std = np.asarray(y, dtype=np.float64), 0.0, 1.0
    K = matern(cdist(X, X), nu, lengthscale) + jitter * np.eye(len(X))
    L = cholesky(K, lower=True)
    alpha = solve_triangular(L.T, solve_triangular(L, yt, lower=True), lower=False)
    return GPFit(X, yt, nu, lengthscale, jitter, L, alpha, mean, std)


def gp_posterior(fit: GPFit, Xc):
    """Posterior mean and variance at the candidates, in standardized units.

        mu(c)     = k*(c) . alpha
        var(c)    = k(0) - || L^-1 k*(c) ||^2, clamped at 0
    with k*(c)_j = k(||x_c - x_j||).  Exhaustive over the given candidates
    (Sec. III-G: every discrete point is predicted).
    """
    Ks = matern(cdist(np.asarray(Xc, dtype=np.float64), fit.X), fit.nu, fit.lengthscale)
    mu = Ks @ fit.alpha
    v = solve_triangular(fit.L, Ks.T, lower=True)
    var = np.maximum(0.0, 1.0 - np.sum(v * v, axis=0))
    return mu, var


def predict(X, y, Xc, nu=1.5, lengthscale=1.5, jitter=1e-10, normalize_y=True):
    """gp_fit then gp_posterior; returns (mu, var, fit)."""
    fit = gp_fit(X, y, nu, lengthscale, jitter, normalize_y)
    mu, var = gp_posterior(fit, Xc)
    return mu, var, fit


# --- Sec. III-C: acquisition functions, minimization variants

def phi_pdf(z):
    return np.exp(-0.5 * np.asarray(z, dtype=np.float64) ** 2) / math.sqrt(2.0 * math.pi)


def Phi_cdf(z):
    return 0.5 * erfc(-np.asarray(z, dtype=np.float64) / math.sqrt(2.0))


def expected_improvement(mu, sigma, fplus, lam):
    """EI for minimization with exploration offset lam (Sec. III-C, III-F).

    Improvement over the best observation f+ by at least lam:
    E[max(f+ - lam - g, 0)] with g ~ N(mu, sigma^2), i.e.
    delta Phi(delta / sigma) + sigma phi(delta / sigma), delta = f+ - mu - lam;
    at sigma = 0 it is max(delta, 0).  Larger is better.
    """
    mu = np.asarray(mu, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    delta = fplus - mu - lam
    with np.errstate(divide="ignore", invalid="ignore"):
        z = delta / sigma
        ei = delta * Phi_cdf(z) + sigma * phi_pdf(z)
    return np.where(sigma > 0, ei, np.maximum(delta, 0.0))


def probability_of_improvement(mu, sigma, fplus, lam):
    """PI for minimization: P(g <= f+ - lam) = Phi((f+ - mu - lam) / sigma)."""
    mu = np.asarray(mu, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    delta = fplus - mu - lam
    with np.errstate(divide="ignore", invalid="ignore"):
        pi = Phi_cdf(delta / sigma)
    return np.where(sigma > 0, pi, (delta > 0).astype(np.float64))


def negative_lcb(mu, sigma, lam):
    """Lower confidence bound mu - lam sigma, negated so larger is better."""
    return -(np.asarray(mu, dtype=np.float64) - lam * np.asarray(sigma, dtype=np.float64))


def acquisition(name, mu, sigma, fplus, lam):
    if name == "ei":
        return expected_improvement(mu, sigma, fplus, lam)
    if name == "poi":
        return probability_of_improvement(mu, sigma, fplus, lam)
    if name == "lcb":
        return negative_lcb(mu, sigma, lam)
    raise ValueError(name)


# --- Sec. III-F: contextual variance exploration factor

def contextual_variance_lambda(mean_var, fplus, mu_s, mean_var_s):
    """lambda = (mean_var / (mu_s / f+)) / mean_var_s   (Sec. III-F).

    mean_var    mean posterior variance now
    fplus       best (lowest) observation so far, raw units, > 0
    mu_s        mean of the initial sample's observations, raw units, > 0
    mean_var_s  mean posterior variance right after the initial sample
    """
    if not (fplus > 0 and mu_s > 0):
        raise ValueError("contextual variance needs f+ > 0 and mu_s > 0")
    return (mean_var / (mu_s / fplus)) / mean_var_s


# --- argmax over the non-evaluated valid configurations (Sec. III-D)

def masked_argmax(scores, mask):
    """Index of the largest score among mask == True; ties -> lowest index."""
    scores = np.asarray(scores, dtype=np.float64)
    idx = np.flatnonzero(mask)
    if idx.size == 0:
        return -1
    best = idx[np.argmax(scores[idx])]     # np.argmax returns the first maximum
    return int(best)


def masked_topk(scores, mask, k):
    """The k best (index, score) among mask == True, best first; ties -> lower index."""
    scores = np.asarray(scores, dtype=np.float64)
    idx = np.flatnonzero(mask)
    order = np.lexsort((idx, -scores[idx]))[:k]
    return [(int(idx[o]), float(scores[idx[o]])) for o in order]
