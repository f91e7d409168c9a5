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


# ---- initial sample (Sec. III-E) ---------------------------------------------
import oracle.sampling as osamp  # noqa: E402
import test_oracle_sampling as T_samp  # noqa: E402


def test_maximin_keeping_the_worst_design(monkeypatch):
    orig = osamp.min_pair_sq_distance
    monkeypatch.setattr(osamp, "min_pair_sq_distance", lambda pts: -orig(pts))
    _fails(T_samp.test_maximin_improves_with_more_designs)


def test_strata_ignored_plain_random_values(monkeypatch):
    def bad(sizes, n, draw):
        out = np.zeros((n, len(sizes)), dtype=np.int64)
        for p in range(len(sizes)):
            for i in range(n):
                out[i, p] = draw() % sizes[p]
        return out
    monkeypatch.setattr(osamp, "latin_hypercube", bad)
    monkeypatch.setattr(T_samp, "latin_hypercube", bad)
    _fails(T_samp.test_latin_property_one_value_per_stratum, 0)


def test_stratum_mapping_off_by_one(monkeypatch):
    orig = osamp.latin_hypercube

    def bad(sizes, n, draw):
        v = orig(sizes, n, draw)
        return np.minimum(v + 1, np.array(sizes) - 1)
    monkeypatch.setattr(T_samp, "latin_hypercube", bad)
    _fails(T_samp.test_each_stratum_holds_one_sample, 1)


def test_restricted_samples_not_replaced(monkeypatch):
    orig = osamp.initial_design

    def bad(grids, mask, count, mode="maximin", designs=100, seed=0, draw=None):
        return orig(grids, None, count, mode, designs, seed, draw)    # mask ignored
    monkeypatch.setattr(T_samp, "initial_design", bad)
    _fails(T_samp.test_restricted_samples_are_replaced_and_valid_ones_kept, "lhs")


def test_column_major_enumeration(monkeypatch):
    import test_oracle_space as T_sp

    def bad(sizes, invalid_mask=None):          # first parameter fastest
        total = int(np.prod(sizes, dtype=np.int64))
        flat = np.arange(total, dtype=np.int64)
        if invalid_mask is not None:
            flat = flat[np.asarray(invalid_mask).reshape(-1) == 0]
        codes = np.stack(np.unravel_index(flat, tuple(int(s) for s in sizes), order="F"), axis=1)
        return flat, codes
    monkeypatch.setattr(T_sp.O, "valid_list", bad)
    _fails(T_sp.test_valid_list_hand_enumerated)
