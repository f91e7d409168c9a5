"""Behaviour of the oracle's BO session (Sec. III-A, III-D, III-F)."""
import math

import numpy as np
import pytest

from oracle import OracleSession, SplitMix64
from paper_2111_14991_gb300 import workloads as W
from golden_values import load

G = load("closed_forms.txt")


def test_splitmix64_reference_values():
    r = SplitMix64(0)
    assert [r.next() for _ in range(3)] == [int(G[f"splitmix64_seed0_{i}"], 16) for i in range(3)]


def small_space():
    return W.config1_space()


def test_init_phase_and_no_revisit():
    sp = small_space()
    s = OracleSession(sp.grids, sp.invalid, n_init=10, seed=3)
    land = W.Landscape(sp, 0)
    seen = set()
    for t in range(30):
        info = s.suggest()
        assert info["predicted"] == (t >= 10)
        assert 0 <= info["idx"] < s.N and info["idx"] not in seen
        seen.add(info["idx"])
        s.observe(info["idx"], land(info["idx"]))
    with pytest.raises(KeyError):
        s.observe(next(iter(seen)), 1.0)
    with pytest.raises(IndexError):
        s.observe(s.N, 1.0)


def test_first_pass_lambda_is_ratio():
    sp = small_space()
    land = W.Landscape(sp, 1)
    s = OracleSession(sp.grids, sp.invalid)
    ys = []
    for i in W.random_initial_sample(sp.n_valid, 20, 1):
        ys.append(land(i))
        s.observe(int(i), ys[-1])
    info = s.suggest()
    assert info["lam"] == pytest.approx(min(ys) / np.mean(ys), rel=1e-13)


def test_invalid_observations_not_fitted():
    sp = small_space()
    s = OracleSession(sp.grids, sp.invalid)
    s.observe(0, 2.0)
    s.observe(5, float("nan"))
    s.observe(9, 3.0)
    s.suggest()
    assert len(s.last_pass["fit"].X) == 2
    assert s.visited[5] and not s.last_pass["mask"][5]


def test_exhaustion():
    grids = [np.array([0.0, 1.0]), np.array([0.0, 1.0])]
    s = OracleSession(grids, None)
    for i in range(4):
        info = s.suggest()
        s.observe(info["idx"], 1.0 + i)
    with pytest.raises(StopIteration):
        s.suggest()


@pytest.mark.parametrize("af", ["ei", "poi", "lcb", "multi", "advanced_multi"])
def test_bo_beats_random_search(af):
    """Behavioural pin of the signs: minimization BO finds lower values than random."""
    sp = small_space()
    wins = 0
    for seed in range(3):
        land = W.Landscape(sp, seed)
        s = OracleSession(sp.grids, sp.invalid, af=af)
        init = W.random_initial_sample(sp.n_valid, 20, seed)
        for i in init:
            s.observe(int(i), land(i))
        for _ in range(40):
            i = s.suggest()["idx"]
            s.observe(i, land(i))
        best_bo = np.min(land.clean(s.obs_idx))
        rng = np.random.default_rng(seed + 77)
        rand = [np.min(land.clean(rng.choice(sp.n_valid, 60, replace=False))) for _ in range(20)]
        wins += best_bo <= np.median(rand)
    assert wins == 3

