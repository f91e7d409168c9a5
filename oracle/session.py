"""Oracle BO session: observe / suggest on a discrete constrained space.

Test infrastructure only (see the package docstring).  One suggest follows
the loop of Sec. III-A: fit the surrogate on the valid observations, predict
every non-evaluated valid configuration (Sec. III-D, III-G), compute the
exploration factor (Sec. III-F), score with the acquisition functions
(Sec. III-C), take the masked argmax, and let the AF selection of Sec. III-G
decide which picks a round hands out.

Readings (the paper is silent on these):
  * Observations are standardized (mean, population std; std 0 -> 1) before
    fitting; mu, sigma, f+ enter the acquisition functions in those units.
  * The contextual-variance baseline is fixed at the first prediction pass:
    mu_s = mean of the valid raw observations made before it, and
    mean_var_s = that pass's mean variance, so lambda = f+/mu_s there.  The
    mean variance is over the valid, non-evaluated configurations scored.
  * Initial sampling handled by the session (n_init > 0) lasts until n_init
    valid (finite) observations exist (Sec. III-E: invalid initial samples
    are replaced until all are valid).  With init "lhs" / "maximin" the
    session first hands out the design of oracle.sampling.initial_design
    (skipping configurations already evaluated); otherwise, and after the
    design, suggests draw uniformly among the non-evaluated valid
    configurations with splitmix64: r = next() mod (#non-evaluated), and the
    r-th non-evaluated configuration in valid-list order is taken.
"""
from __future__ import annotations

import math

import numpy as np

from .bo_oracle import (AF_NAMES, acquisition, candidate_coords, contextual_variance_lambda,
                        gp_fit, gp_posterior, masked_topk, valid_list)
from .sampling import initial_design
from .selection import make_selector

__all__ = ["OracleSession", "SplitMix64", "SuggestInfo"]

_M64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 (Steele, Lea and Flood, 2014), written from its definition."""

    def __init__(self, seed):
        self.state = seed & _M64

    def next(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)


class SuggestInfo(dict):
    """idx, af, mu, sigma, score, lam, mean_var, predicted (bool)."""


class OracleSession:
    def __init__(self, grids, invalid_mask=None, nu=1.5, lengthscale=1.5, jitter=1e-10,
                 af="ei", explore="cv", lambda_const=0.01, skip_threshold=5, rif=0.1,
                 discount=None, normalize_y=True, n_init=0, seed=0, init="maximin", init_designs=100):
        self.grids = [np.asarray(g, dtype=np.float64) for g in grids]
        sizes = [len(g) for g in self.grids]
        self.invalid_mask = invalid_mask
        self.flat, self.codes = valid_list(sizes, invalid_mask)
        self.coords = candidate_coords(self.grids, self.codes)
        self.N = len(self.flat)
        self.visited = np.zeros(self.N, dtype=bool)
        self.obs_idx, self.obs_y = [], []
        self.nu, self.lengthscale, self.jitter = nu, lengthscale, jitter
        self.af, self.explore, self.lambda_const = af, explore, lambda_const
        self.normalize_y = normalize_y
        self.n_init = n_init
        self.rng = SplitMix64(seed)
        self.init, self.init_designs, self.seed = init, init_designs, seed
        self.init_queue = None
        self.selector = make_selector(af, skip_threshold, discount, rif)
        self.mu_s = None
        self.mean_var_s = None
        self.queue = []           # [(idx, [afs])] still to hand out this round
        self.outstanding = {}     # idx -> [afs] handed out, not yet observed
        self.last_pass = None     # dict of the last prediction pass (for tests)

    # -- bookkeeping ---------------------------------------------------------
    def finite_y(self):
        return [y for y in self.obs_y if math.isfinite(y)]

    def observe(self, idx, y):
        if not (0 <= idx < self.N):
            raise IndexError(idx)
        if self.visited[idx]:
            raise KeyError("duplicate observation")
        self.visited[idx] = True
        self.obs_idx.append(int(idx))
        self.obs_y.append(float(y))
        afs = self.outstanding.pop(int(idx), None)
        if afs is not None:
            val = float(y)
            if not math.isfinite(val):
                fy = self.finite_y()
                val = float(np.median(fy)) if fy else None
            if val is not None:
                self.selector.credit(afs, val)

    def _design(self, count):
        """The initial design, drawn from the session's splitmix64 stream."""
        return initial_design(self.grids, self.invalid_mask, count, self.init, self.init_designs,
                              draw=self.rng.next)

    def _random_pick(self):
        free = np.flatnonzero(~self.visited)
        r = self.rng.next() % len(free)
        return int(free[r])

    # -- the prediction pass ---------------------------------------------------
    def prediction_pass(self, active):
        fin = [(i, y) for i, y in zip(self.obs_idx, self.obs_y) if math.isfinite(y)]
        X = self.coords[[i for i, _ in fin]]
        y = np.array([y for _, y in fin])
        fit = gp_fit(X, y, self.nu, self.lengthscale, self.jitter, self.normalize_y)
        mask = ~self.visited
        mu, var = gp_posterior(fit, self.coords)
        sigma = np.sqrt(var)
        mean_var = float(np.mean(var[mask]))
        fplus_raw = float(np.min(y))
        if self.explore == "cv":
            if self.mu_s is None:
                self.mu_s = float(np.mean(y))
                self.mean_var_s = mean_var
            lam = contextual_variance_lambda(mean_var, fplus_raw, self.mu_s, self.mean_var_s)
        else:
            lam = self.lambda_const
        fplus = (fplus_raw - fit.y_mean) / fit.y_std
        scores = {a: acquisition(a, mu, sigma, fplus, lam) for a in active}
        k = len(active)
        topk = {a: masked_topk(scores[a], mask, k) for a in active}
        self.last_pass = dict(mu=mu, var=var, sigma=sigma, mean_var=mean_var, lam=lam,
                              fplus=fplus, scores=scores, topk=topk, mask=mask, fit=fit)
        return self.last_pass

    def suggest(self):
        free = int(np.count_nonzero(~self.visited))
        if free == 0:
            raise StopIteration("search space exhausted")
        if len(self.finite_y()) < self.n_init or not self.finite_y():
            if self.init != "random" and self.n_init > 0:
                if self.init_queue is None:
                    count = min(self.n_init, len(self.visited))
                    self.init_queue = list(self._design(count))
                while self.init_queue and self.visited[self.init_queue[0]]:
                    self.init_queue.pop(0)
                if self.init_queue:
                    return SuggestInfo(idx=int(self.init_queue.pop(0)), af=None, predicted=False)
            return SuggestInfo(idx=self._random_pick(), af=None, predicted=False)
        while self.queue:
            idx, afs = self.queue.pop(0)
            if not self.visited[idx]:
                self.outstanding[idx] = afs
                return self._info(idx, afs)
        self.selector.begin_round()
        self.outstanding = {}
        p = self.prediction_pass(self.selector.active)
        self.queue = list(self.selector.assign(p["topk"]))
        idx, afs = self.queue.pop(0)
        self.outstanding[idx] = afs
        return self._info(idx, afs)

    def _info(self, idx, afs):
        p = self.last_pass
        return SuggestInfo(idx=int(idx), af=afs[0], predicted=True, mu=float(p["mu"][idx]),
                           sigma=float(p["sigma"][idx]),
                           score=float(p["scores"][afs[0]][idx]),
                           lam=float(p["lam"]), mean_var=float(p["mean_var"]))


assert AF_NAMES == ("ei", "poi", "lcb")
