"""Per-candidate amplification of FP32 rounding in the GP posterior (test analysis).

A reduced-precision pass evaluates K* in FP32, so each k*_j carries a relative
rounding error of a few u = 2^-24 whatever the contraction's operand split.
To first order that error reaches

    mu      = k* . alpha             as  sum_j alpha_j k*_j eps_j   <= u_K sum_j |alpha_j k*_j|
    sigma^2 = 1 - k*^T K^-1 k*       as  2 sum_j w_j k*_j eps_j     <= u_K 2 sum_j |w_j k*_j|

with w = K^-1 k*.  These sums are the condition numbers of mu and sigma^2
with respect to K*; they are computed here in FP64 from the oracle's fit.
"""
import numpy as np
from scipy.linalg import solve_triangular
from scipy.spatial.distance import cdist

import oracle as O

U32 = 2.0 ** -24


def amplification(fit, Xc):
    """(sum_j |alpha_j k*_j|, 2 sum_j |w_j k*_j|) for every candidate row of Xc."""
    Ks = O.matern(cdist(np.asarray(Xc, dtype=np.float64), fit.X), fit.nu, fit.lengthscale)
    a_mu = np.abs(Ks) @ np.abs(fit.alpha)
    V = solve_triangular(fit.L, Ks.T, lower=True)
    W = solve_triangular(fit.L.T, V, lower=False)
    a_var = 2.0 * np.sum(np.abs(W.T * Ks), axis=1)
    return a_mu, a_var


def rounding_ratios(fit, Xc, mu, rmu, var, rvar):
    """Largest observed error in units of u times the amplification, for mu and
    sigma^2: a pass whose only error is the FP32 rounding of K* (and of the
    sums) stays at a small multiple of 1 everywhere."""
    a_mu, a_var = amplification(fit, Xc)
    rm = np.abs(np.asarray(mu, np.float64) - rmu) / (U32 * a_mu)
    rv = np.abs(np.asarray(var, np.float64) - rvar) / (U32 * np.maximum(a_var, 1.0))
    return float(rm.max()), float(rv.max())
