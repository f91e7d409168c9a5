"""Batched form: every space's result is the same alone and inside a batch.

A batch runs the update of all its spaces in five launches and the prediction
passes of all of them in one persistent tensor-core launch plus one
acquisition launch (from a captured graph once a shape repeats).  Each space
here has a twin driven alone through bo_observe / bo_suggest with the same
inputs; posteriors, factors and picks must agree.
"""
import math

import numpy as np
import pytest

from paper_2111_14991_gb300 import workloads as W
from tolerances import pick_ok

pytestmark = pytest.mark.gpu

SPECS = [  # (seed, d, N valid, n initial observations, af, n_init)
    (11, 3, 1500, 20, "ei", 0), (12, 9, 40000, 90, "ei", 0), (13, 5, 7000, 33, "lcb", 0),
    (14, 7, 21000, 64, "multi", 0), (15, 4, 3000, 1, "poi", 0), (16, 8, 12000, 0, "ei", 3),
]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2111_14991_gb300 import build
    build.build()


def twins(precision):
    from paper_2111_14991_gb300 import Space
    alone, member, lands = [], [], []
    for seed, d, n_valid, n0, af, n_init in SPECS:
        sp = W.generic_space(seed, d, n_valid)
        land = W.Landscape(sp, seed)
        pair = [Space(sp.grids, sp.invalid, precision=precision, af=af, n_init=n_init, seed=seed, n_max=160)
                for _ in range(2)]
        if n0:
            for i in W.clustered_observations(land, n0, seed):
                v = float(land.clean([i])[0])
                for s in pair:
                    s.observe(int(i), v)
        alone.append(pair[0])
        member.append(pair[1])
        lands.append(land)
    return alone, member, lands


@pytest.mark.parametrize("precision", ["fp16x3", "tf32x3", "tf32", "fp64"])
def test_batch_equals_alone(precision):
    from paper_2111_14991_gb300 import Batch
    alone, member, lands = twins(precision)
    batch = Batch(member)
    for step in range(6):
        if step == 3 and precision != "fp64":
            r = batch.autotune(reps=1)              # shapes of the batched launch; results unchanged
            assert r["tried"] > 1
        bidx, bstatus, binfo = batch.suggest()
        assert not bstatus.any(), bstatus
        picks = []
        for i, a in enumerate(alone):
            ai = a.suggest()
            if ai["predicted"] and binfo[i]["predicted"] and binfo[i]["n_scored"]:
                ma, va = a.last_posterior()
                mb, vb = member[i].last_posterior()
                np.testing.assert_allclose(mb, ma, rtol=1e-6, atol=1e-7)
                np.testing.assert_allclose(vb, va, rtol=1e-6, atol=1e-7)
                assert binfo[i]["lam"] == pytest.approx(ai["lam"], rel=1e-9)
                sc_a = ai["score"]
                assert bidx[i] == ai["idx"] or abs(binfo[i]["score"] - sc_a) <= 1e-6 * max(abs(sc_a), 1.0)
            else:
                assert bidx[i] == ai["idx"]      # random (init) or queued picks
            picks.append(ai["idx"])
        ys = []
        for i, land in enumerate(lands):
            v = float(land.clean([picks[i]])[0])
            if step == 2 and i == 0:
                v = float("nan")                    # a runtime-invalid configuration
            ys.append(v)
            alone[i].observe(picks[i], v)
        st = batch.observe(picks, ys)
        assert not st.any(), st
        for i in range(len(alone)):
            la, ba = alone[i].factor()
            lb, bb = member[i].factor()
            assert la.shape == lb.shape
            if la.size:
                np.testing.assert_allclose(lb, la, rtol=1e-12, atol=1e-12 * np.abs(la).max())
                np.testing.assert_allclose(bb, ba, rtol=1e-12, atol=1e-12 * np.abs(ba).max())
    assert batch.launch_count() > 0
    batch.close()
    for s in alone + member:
        s.close()


def test_batch_rejects_mixed_precision():
    from paper_2111_14991_gb300 import Batch, BOError, Space
    grids = [np.linspace(0, 1, 5), np.linspace(0, 1, 4)]
    a = Space(grids, None, precision="fp16x3")
    b = Space(grids, None, precision="fp64")
    with pytest.raises(BOError):
        Batch([a, b])
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3"])
def test_batch_with_wide_spaces_equals_alone(precision):
    """A batch holding a space with n > 256 runs two MMA issuers (one per
    256-column accumulator region) for every space in it; each space's
    posterior must still equal its single-space pass, where spaces with
    n <= 256 take the one-issuer path."""
    from paper_2111_14991_gb300 import Batch, Space
    specs = [(21, 9, 30000, 300), (22, 5, 8000, 100), (23, 7, 20000, 260), (24, 4, 2000, 40)]
    alone, member = [], []
    for seed, d, n_valid, n0 in specs:
        sp = W.generic_space(seed, d, n_valid)
        land = W.Landscape(sp, seed)
        pair = [Space(sp.grids, sp.invalid, precision=precision, n_max=320) for _ in range(2)]
        for i in W.clustered_observations(land, n0, seed):
            v = float(land.clean([i])[0])
            for s in pair:
                s.observe(int(i), v)
        alone.append(pair[0])
        member.append(pair[1])
    batch = Batch(member)
    bidx, bstatus, binfo = batch.suggest()
    assert not bstatus.any(), bstatus
    for i, a in enumerate(alone):
        ai = a.suggest()
        ma, va = a.last_posterior()
        mb, vb = member[i].last_posterior()
        np.testing.assert_array_equal(mb, ma)
        np.testing.assert_array_equal(vb, va)
        assert bidx[i] == ai["idx"]
    for s in alone + member:
        s.close()
