"""Scripted scenarios for the AF selection of Sec. III-G (readings in oracle/selection.py)."""
import pytest

from oracle import AdvancedMultiSelector, MultiSelector, SingleSelector
from golden_values import load

G = load("closed_forms.txt")


def tk(*idx):
    return [(i, 1.0 - 0.1 * r) for r, i in enumerate(idx)]


def test_dos_definition():
    s = MultiSelector(discount=0.9)
    for o in (1.0, 2.0, 3.0):
        s.credit(["ei"], o)
    assert s.dos["ei"] == pytest.approx(float(G["dos_123_g0.9"]), rel=1e-15)
    assert s.dos["poi"] == 0.0


def test_single_selector():
    s = SingleSelector("poi")
    s.begin_round()
    assert s.assign({"poi": tk(7, 3)}) == [(7, ["poi"])]


def run_multi_round(s, picks, obs):
    s.begin_round()
    out = s.assign({a: tk(picks[a], 1000 + i) for i, a in enumerate(("ei", "poi", "lcb"))})
    for idx, afs in out:
        s.credit(afs, obs[idx])
    return out


def test_multi_duplicates_and_skip():
    s = MultiSelector(skip_threshold=5, discount=0.65)
    out = run_multi_round(s, {"ei": 1, "poi": 2, "lcb": 3}, {1: 1.0, 2: 5.0, 3: 2.0})
    assert out == [(1, ["ei"]), (2, ["poi"]), (3, ["lcb"])]
    for r in range(6):   # ei and poi agree six times: counts 1..6
        a, c = 10 + r, 20 + r
        out = run_multi_round(s, {"ei": a, "poi": a, "lcb": c}, {a: 1.0, c: 2.0})
        assert out == [(a, ["ei", "poi"]), (c, ["lcb"])]
        if r < 5:
            assert s.dup["ei"] == r + 1
    assert s.dup == {"ei": 6, "poi": 6, "lcb": 0}
    assert s.active == ["ei", "poi", "lcb"]
    s.begin_round()     # 6 > 5: ei and poi pitted; poi's dos is higher (its solo 5.0)
    assert s.dos["poi"] > s.dos["ei"]
    assert s.active == ["ei", "lcb"]
    assert s.dup == {"ei": 0, "poi": 0, "lcb": 0}


def test_multi_threshold_not_exceeded():
    s = MultiSelector(skip_threshold=5)
    for r in range(6):   # five duplicates after the first round -> count 5, not > 5
        a = 10 + r
        picks = {"ei": a, "poi": a if r > 0 else 99, "lcb": 50 + r}
        run_multi_round(s, picks, {a: 1.0, 99: 1.0, 50 + r: 1.0})
    s.begin_round()
    assert s.active == ["ei", "poi", "lcb"]


def test_multi_triple_duplicate_counts():
    s = MultiSelector()
    s.begin_round()
    out = s.assign({"ei": tk(4), "poi": tk(4), "lcb": tk(4)})
    assert out == [(4, ["ei", "poi", "lcb"])]
    assert s.dup == {"ei": 2, "poi": 2, "lcb": 2}


def adv_round(s, values):
    s.begin_round()
    for a in list(s.active):
        s.credit([a], values[a])


def test_adv_multi_assign_avoids_duplicates():
    s = AdvancedMultiSelector()
    s.begin_round()
    out = s.assign({"ei": tk(5, 6, 7), "poi": tk(5, 6, 8), "lcb": tk(6, 5, 9)})
    assert out == [(5, ["ei"]), (6, ["poi"]), (9, ["lcb"])]


def test_adv_multi_skip():
    s = AdvancedMultiSelector(skip_threshold=5, rif=0.1)
    vals = {"ei": 1.6, "poi": 2.0, "lcb": 1.6}
    adv_round(s, vals)                # round 1: no judging yet
    for r in range(4):
        adv_round(s, vals)
        assert s.over["poi"] == r + 1 and s.under["ei"] == 0
    assert s.active == ["ei", "poi", "lcb"]
    adv_round(s, vals)                # fifth over count: poi skipped, others reset
    assert s.active == ["ei", "lcb"]
    assert s.over["ei"] == s.under["ei"] == s.over["lcb"] == s.under["lcb"] == 0


def test_adv_multi_promote():
    s = AdvancedMultiSelector(skip_threshold=5, rif=0.1)
    vals = {"ei": 1.0, "poi": 1.5, "lcb": 1.5}   # ei well below the mean
    adv_round(s, vals)
    for _ in range(4):
        adv_round(s, vals)
    assert s.active == ["ei", "poi", "lcb"] and s.under["ei"] == 4
    adv_round(s, vals)
    assert s.active == ["ei"]
    s.begin_round()                   # a single AF is never judged
    assert s.active == ["ei"]
