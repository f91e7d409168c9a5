"""A complete tuning run on top of the suggest library, and the paper's
quality measures of a run.

`minimize` is the loop of Sec. III-A as a user runs it: the session hands out
the initial sample (Sec. III-E), then one suggestion per evaluation; every
result, including failed (NaN) ones, is observed.  `random_search` is the
baseline strategy.  `mae` and `mdf` are the measures of Sec. IV: the mean
absolute error of the best configuration found after 40, 60, ..., 220
evaluations against the global optimum, and the mean deviation factor of a
strategy's mean MAE across kernels.

Readings: the best configuration found is the one with the lowest observed
(noisy) value; its error is measured with the noise-free objective (`truth`),
as the paper's averaged measurements are.  The MDF divides a strategy's mean
MAE on a kernel by the mean over all compared strategies of their mean MAE on
that kernel, then averages over kernels.
"""
from __future__ import annotations

import numpy as np

from .bo import BOError, Space

BO_ERR_EXHAUSTED = 4          # include/bo_suggest.h

__all__ = ["minimize", "random_search", "best_found", "mae", "mdf"]

CHECKPOINTS = tuple(range(40, 221, 20))   # 20 i for i = 2..11


def minimize(objective, grids, invalid_mask=None, *, budget=220, n_init=20, space=None, **params):
    """Tune: `objective(idx) -> float` (NaN for a failed configuration) over
    valid-list indices.  Returns (indices, values) in evaluation order."""
    own = space is None
    s = Space(grids, invalid_mask, n_init=n_init, **params) if own else space
    idx, val = [], []
    try:
        for _ in range(budget):
            try:
                i = int(s.suggest()["idx"])
            except BOError as e:
                if e.code == BO_ERR_EXHAUSTED:
                    break
                raise
            v = float(objective(i))
            s.observe(i, v)
            idx.append(i)
            val.append(v)
    finally:
        if own:
            s.close()
    return np.array(idx, dtype=np.int64), np.array(val, dtype=np.float64)


def random_search(objective, n_valid, *, budget=220, seed=0):
    """Uniform random distinct configurations (the baseline strategy)."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(n_valid, size=min(budget, n_valid), replace=False).astype(np.int64)
    return idx, np.array([float(objective(int(i))) for i in idx], dtype=np.float64)


def best_found(idx, values, count):
    """Valid-list index of the lowest observed value among the first `count`
    evaluations (failed ones never count), or -1."""
    v = np.where(np.isfinite(values[:count]), values[:count], np.inf)
    return int(idx[int(np.argmin(v))]) if count and np.isfinite(v).any() else -1


def mae(idx, values, truth, f_opt, checkpoints=CHECKPOINTS):
    """Mean over the checkpoints of |truth(best found) - f_opt| (Sec. IV)."""
    errs = []
    for k in checkpoints:
        b = best_found(idx, values, min(k, len(idx)))
        errs.append(abs(truth(b) - f_opt) if b >= 0 else np.inf)
    return float(np.mean(errs))


def mdf(mean_mae):
    """mean_mae[strategy][kernel] -> {strategy: (MDF, std of the factors)}."""
    strategies = list(mean_mae)
    kernels = list(next(iter(mean_mae.values())))
    out = {}
    for s in strategies:
        f = [mean_mae[s][k] / np.mean([mean_mae[t][k] for t in strategies]) for k in kernels]
        out[s] = (float(np.mean(f)), float(np.std(f)))
    return out
