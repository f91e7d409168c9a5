"""Pins of the oracle's initial sample (Sec. III-E, Table I): the Latin
hypercube property, the maximin choice, and the replacement of restricted
samples, checked against what the construction must guarantee rather than
against its own formulas."""
import itertools

import numpy as np
import pytest

from oracle import SplitMix64, valid_list
from oracle.sampling import _splitmix64, initial_design, latin_hypercube, min_pair_sq_distance
from paper_2111_14991_gb300 import workloads as W


def grids_of(sizes):
    return [np.linspace(0.0, 1.0, m) if m > 1 else np.zeros(1) for m in sizes]


def sample_values(grids, idx, mask=None):
    _, codes = valid_list([len(g) for g in grids], mask)
    return codes[np.asarray(idx)]


def test_stream_is_splitmix64():
    a, b = _splitmix64(12345), SplitMix64(12345)
    assert [a() for _ in range(5)] == [b.next() for _ in range(5)]


@pytest.mark.parametrize("seed", range(6))
def test_latin_property_one_value_per_stratum(seed):
    # m = n values per parameter: every value is taken exactly once per parameter
    n = 12
    v = latin_hypercube([n, n, n], n, _splitmix64(seed))
    for p in range(3):
        assert sorted(v[:, p]) == list(range(n))


@pytest.mark.parametrize("seed", range(6))
def test_each_stratum_holds_one_sample(seed):
    # m = 3n: the value index // 3 is the stratum, which must be a permutation
    n = 10
    v = latin_hypercube([3 * n, 3 * n], n, _splitmix64(seed))
    for p in range(2):
        assert sorted(v[:, p] // 3) == list(range(n))


def test_mapping_matches_floating_point_definition():
    # floor(u m) with u = (stratum + U) / n, evaluated in floating point where
    # the product is not within rounding of an integer
    draw = _splitmix64(7)
    n, m = 20, 7
    v = latin_hypercube([m], n, draw)
    draw2 = _splitmix64(7)
    strata = list(range(n))
    for i in range(n - 1, 0, -1):
        j = draw2() % (i + 1)
        strata[i], strata[j] = strata[j], strata[i]
    for i in range(n):
        u = (strata[i] + (draw2() >> 11) / 2.0 ** 53) / n
        x = u * m
        if abs(x - round(x)) > 1e-9:
            assert v[i, 0] == int(np.floor(x))


def test_few_values_are_balanced():
    # m < n: value v of parameter p is taken by the strata inside [v/m, (v+1)/m)
    n, m = 20, 6
    for seed in range(10):
        v = latin_hypercube([m], n, _splitmix64(seed))
        counts = np.bincount(v[:, 0], minlength=m)
        assert np.all(np.abs(counts - n / m) < 2)


def test_two_by_two_brute_force():
    # sizes (2, 2), two samples: a Latin design is one of the two diagonals
    diagonals = [{(0, 0), (1, 1)}, {(0, 1), (1, 0)}]
    for seed in range(20):
        idx = initial_design(grids_of([2, 2]), None, 2, "lhs", seed=seed)
        assert {tuple(r) for r in sample_values(grids_of([2, 2]), idx)} in diagonals


def pair_score(grids, idx, mask=None):
    codes = sample_values(grids, idx, mask)
    pts = np.array([[grids[p][c[p]] for p in range(len(grids))] for c in codes])
    best = np.inf
    for a, b in itertools.combinations(range(len(pts)), 2):
        best = min(best, float(np.sum((pts[a] - pts[b]) ** 2)))
    return best


@pytest.mark.parametrize("seed", range(5))
def test_maximin_spreads_at_least_as_well_as_its_first_design(seed):
    g = grids_of([8, 6, 5, 4])
    lhs = initial_design(g, None, 12, "lhs", seed=seed)           # the first design of the stream
    mm = initial_design(g, None, 12, "maximin", designs=30, seed=seed)
    assert pair_score(g, mm) >= pair_score(g, lhs)


def test_maximin_improves_with_more_designs():
    g = grids_of([8, 6, 5, 4])
    for seed in range(5):
        few = initial_design(g, None, 12, "maximin", designs=3, seed=seed)
        many = initial_design(g, None, 12, "maximin", designs=40, seed=seed)
        assert pair_score(g, many) >= pair_score(g, few)


def test_maximin_beats_random_on_average():
    g = grids_of([10, 10, 10])
    mm = [pair_score(g, initial_design(g, None, 15, "maximin", designs=50, seed=s)) for s in range(10)]
    rnd = [pair_score(g, initial_design(g, None, 15, "random", seed=s)) for s in range(10)]
    assert np.mean(mm) > 2.0 * np.mean(rnd)


def test_min_pair_distance_brute_force():
    rng = np.random.default_rng(0)
    pts = rng.random((9, 3))
    ref = min(float(np.sum((a - b) ** 2)) for a, b in itertools.combinations(pts, 2))
    assert min_pair_sq_distance(pts) == pytest.approx(ref, rel=1e-15)


@pytest.mark.parametrize("mode", ["lhs", "maximin"])
def test_restricted_samples_are_replaced_and_valid_ones_kept(mode):
    sp = W.paper_shaped_space("conv")                        # restricted configurations present
    sizes = [len(g) for g in sp.grids]
    assert sp.invalid is not None and sp.invalid.any()
    free = initial_design(sp.grids, None, 20, mode, designs=10, seed=4)
    masked = initial_design(sp.grids, sp.invalid, 20, mode, designs=10, seed=4)
    flat_free, _ = valid_list(sizes, None)
    flat_masked, _ = valid_list(sizes, sp.invalid)
    assert len(set(masked.tolist())) == 20 and masked.min() >= 0 and masked.max() < len(flat_masked)
    # the design does not depend on the mask: samples that are valid under it stay where they are
    kept = 0
    for a, b in zip(free, masked):
        f = int(flat_free[a])
        if not sp.invalid.reshape(-1)[f]:
            assert int(flat_masked[b]) == f
            kept += 1
    assert 0 < kept < 20


def test_random_mode_distinct_and_in_range():
    sp = W.config1_space()
    idx = initial_design(sp.grids, sp.invalid, 50, "random", seed=1)
    assert len(set(idx.tolist())) == 50 and idx.min() >= 0 and idx.max() < sp.n_valid


def test_count_out_of_range():
    with pytest.raises(ValueError):
        initial_design(grids_of([2, 2]), None, 5, "lhs")
