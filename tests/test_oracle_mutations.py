"""Planted mistakes in the oracle (on the CPU) must fail at least one pin.

Each case swaps one oracle function for a plausible wrong variant -- a dropped
term, a wrong sign, a transposed operand, a wrong index -- and checks that
the pin tests written against the paper catch it.
"""
import math

import numpy as np
import pytest
from scipy.linalg import solve_triangular

import oracle.bo_oracle as ob
import oracle.selection as osel
import test_oracle_acq as T_acq
import test_oracle_gp as T_gp
import test_oracle_matern as T_mat
import test_oracle_selection as T_sel


def _fails(fn, *a):
    with pytest.raises(AssertionError):
        fn(*a)


def test_dropped_quadratic_term_in_matern52(monkeypatch):
    def bad(r, nu, l):
        t = math.sqrt(2 * nu) * np.asarray(r, dtype=np.float64) / l
        return (1 + t) * np.exp(-t)
    monkeypatch.setattr(T_mat, "matern", bad)
    _fails(T_mat.test_equals_bessel_form, 2.5, 1.5)


def test_sqrt_of_r_instead_of_r(monkeypatch):
    def bad(r, nu, l):       # the garbled printed form sqrt(3 r)/l
        t = np.sqrt(2 * nu * np.asarray(r, dtype=np.float64)) / l
        return (1 + t) * np.exp(-t)
    monkeypatch.setattr(T_mat, "matern", bad)
    _fails(T_mat.test_equals_bessel_form, 1.5, 1.5)


def test_transposed_triangular_solve(monkeypatch):
    def bad_post(fit, Xc):
        Ks = ob.matern(ob.cdist(np.asarray(Xc), fit.X), fit.nu, fit.lengthscale)
        v = solve_triangular(fit.L.T, Ks.T, lower=False)       # L^-T k* instead of L^-1 k*
        return Ks @ fit.alpha, np.maximum(0.0, 1.0 - np.sum(v * v, axis=0))
    monkeypatch.setattr(ob, "gp_posterior", bad_post)
    _fails(T_gp.test_matches_exact_rational_inverse, 3, 7, 2.5, 0.8, 1)


def test_jitter_on_every_entry(monkeypatch):
    orig = ob.matern

    def bad(r, nu, l):
        return orig(r, nu, l) + 1e-3
    monkeypatch.setattr(ob, "matern", bad)
    _fails(T_gp.test_single_observation_posterior)


def test_ei_sign_flip(monkeypatch):
    def bad(mu, sigma, fplus, lam):
        delta = np.asarray(mu) - fplus - lam          # maximization form
        z = delta / sigma
        return delta * ob.Phi_cdf(z) + sigma * ob.phi_pdf(z)
    monkeypatch.setattr(T_acq, "expected_improvement", bad)
    _fails(T_acq.test_definitions_by_integration, 0.3, 0.7, 0.1, 0.05)


def test_pi_offset_sign(monkeypatch):
    def bad(mu, sigma, fplus, lam):
        return ob.Phi_cdf((fplus + lam - np.asarray(mu)) / sigma)
    monkeypatch.setattr(T_acq, "probability_of_improvement", bad)
    _fails(T_acq.test_definitions_by_integration, 0.3, 0.7, 0.1, 0.05)


def test_cv_inverted_ratio(monkeypatch):
    def bad(mean_var, fplus, mu_s, mean_var_s):
        return (mean_var / (fplus / mu_s)) / mean_var_s
    monkeypatch.setattr(T_acq, "contextual_variance_lambda", bad)
    _fails(T_acq.test_contextual_variance)


def test_argmax_last_of_ties(monkeypatch):
    def bad(scores, mask):
        idx = np.flatnonzero(mask)
        s = np.asarray(scores)[idx]
        return int(idx[len(s) - 1 - np.argmax(s[::-1])])
    monkeypatch.setattr(T_acq, "masked_argmax", bad)
    _fails(T_acq.test_masked_argmax_and_topk_brute_force)


def test_dos_without_discount(monkeypatch):
    def bad(self, afs, value):
        for a in afs:
            self.dos[a] = self.dos[a] + value
    monkeypatch.setattr(osel.MultiSelector, "credit", bad)
    _fails(T_sel.test_dos_definition)
