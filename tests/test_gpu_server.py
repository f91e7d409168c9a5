"""Serving form: continuous batching, admission by device memory, and every
result the same alone and in the mix."""
import time

import numpy as np
import pytest

from paper_2111_14991_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SPECS = [(21, 3, 2000, 30), (22, 9, 30000, 70), (23, 5, 9000, 40), (24, 7, 15000, 55), (25, 4, 4000, 25)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2111_14991_gb300 import build
    build.build()


def sessions():
    out = []
    for seed, d, n_valid, n_obs in SPECS:
        sp = W.generic_space(seed, d, n_valid)
        land = W.Landscape(sp, seed)
        idx = W.clustered_observations(land, n_obs, seed)
        out.append((sp, idx, land.clean(idx)))
    return out


def drain(server, expected, timeout=120.0):
    got, t0 = [], time.time()
    while len(got) < expected and time.time() - t0 < timeout:
        got += server.poll(wait_ms=50)
    assert len(got) == expected, (len(got), expected)
    return got


def test_served_results_equal_alone():
    """Requests of all sessions are submitted at once, interleaved, so the
    server batches them across sessions; each session's twin replays the same
    request sequence alone (bo_observe + bo_suggest)."""
    from paper_2111_14991_gb300 import Server, Space
    data = sessions()
    srv = Server(budget_bytes=8 << 30)
    sids = [srv.open(sp.grids, sp.invalid, precision="fp16x3", n_max=96) for sp, _, _ in data]
    total = 0
    for r in range(max(len(idx) for _, idx, _ in data)):
        for k, (sp, idx, y) in enumerate(data):
            if r < len(idx):
                srv.submit(sids[k], int(idx[r]), float(y[r]), tag=k * 1000 + r)
                total += 1
    got = {c["tag"]: c for c in drain(srv, total)}
    st = srv.stats()
    assert st["iterations"] < st["completed"]          # requests were batched together
    srv.close()
    for k, (sp, idx, y) in enumerate(data):
        a = Space(sp.grids, sp.invalid, precision="fp16x3", n_max=96)
        for r in range(len(idx)):
            a.observe(int(idx[r]), float(y[r]))
            ref = a.suggest()
            c = got[k * 1000 + r]
            assert c["status"] == 0 and c["observed"], c
            assert c["idx"] == ref["idx"] or \
                abs(c["info"]["score"] - ref["score"]) <= 1e-6 * max(abs(ref["score"]), 1), (k, r)
            assert c["info"]["lam"] == pytest.approx(ref["lam"], rel=1e-9)
            assert c["info"]["mu"] == pytest.approx(ref["mu"], rel=1e-5, abs=1e-6)
        a.close()


def test_admission_by_memory_budget():
    from paper_2111_14991_gb300 import Server
    data = sessions()[:4]
    srv = Server(budget_bytes=1 << 40)
    probe = srv.open(data[1][0].grids, data[1][0].invalid, precision="fp16x3", n_max=64)
    srv.close_session(probe)
    srv.close()
    # a budget that holds the two smallest sessions only
    srv = Server(budget_bytes=6 << 20, max_sessions=8)
    sids = []
    for sp, idx, y in data:
        try:
            sids.append(srv.open(sp.grids, sp.invalid, precision="fp16x3", n_max=64))
        except Exception as e:      # larger than the whole budget
            assert "budget" in str(e)
            sids.append(None)
    live = [s for s in sids if s is not None]
    assert len(live) >= 2
    for k, s in enumerate(sids):
        if s is not None:
            sp, idx, y = data[k]
            srv.submit(s, int(idx[0]), float(y[0]), tag=k)
    got = drain(srv, len(live))
    assert all(c["status"] == 0 for c in got)
    st = srv.stats()
    assert st["bytes_in_use"] <= 6 << 20
    for s in live:
        srv.close_session(s)
    srv.close()


def test_rejects_session_above_budget():
    from paper_2111_14991_gb300 import BOError, Server
    sp = W.generic_space(31, 6, 50000)
    srv = Server(budget_bytes=1 << 20)
    with pytest.raises(BOError) as e:
        srv.open(sp.grids, sp.invalid, precision="fp16x3", n_max=128)
    assert e.value.code == 6
    srv.close()


def test_queued_session_admitted_when_memory_frees():
    """Admission as memory frees up: under a budget that holds either of two
    sessions but not both, the second waits (its requests stay pending) while
    the first is served; closing the first admits the second, whose results
    equal its alone twin's and the FP64 oracle's (Sec. III-A loop per request:
    observe, then suggest)."""
    import oracle as O
    from paper_2111_14991_gb300 import Server, Space
    from tolerances import REDUCED, pick_ok
    a_sp = W.generic_space(41, 6, 24000)
    b_sp = W.generic_space(42, 5, 20000)
    data = []
    for seed, sp in ((41, a_sp), (42, b_sp)):
        land = W.Landscape(sp, seed)
        idx = W.clustered_observations(land, 30, seed)
        data.append((sp, idx, land.clean(idx)))
    # each session's device bytes, measured alone
    sizes = []
    for sp, idx, y in data:
        srv = Server(budget_bytes=1 << 40)
        s = srv.open(sp.grids, sp.invalid, precision="fp16x3", n_max=64)
        srv.submit(s, int(idx[0]), float(y[0]), tag=0)
        drain(srv, 1)
        sizes.append(srv.stats()["bytes_in_use"])
        srv.close()
    budget = int(max(sizes) * 1.25) + (256 << 10)     # the estimate adds at most 48 KB of tables
    assert sum(sizes) > budget
    srv = Server(budget_bytes=budget, max_sessions=8)
    sa = srv.open(a_sp.grids, a_sp.invalid, precision="fp16x3", n_max=64)
    sb = srv.open(b_sp.grids, b_sp.invalid, precision="fp16x3", n_max=64)
    (_, ia, ya), (_, ib, yb) = data
    for r in range(len(ia)):
        srv.submit(sa, int(ia[r]), float(ya[r]), tag=r)
    for r in range(len(ib)):
        srv.submit(sb, int(ib[r]), float(yb[r]), tag=1000 + r)
    got = drain(srv, len(ia))
    assert sorted(c["tag"] for c in got) == list(range(len(ia)))
    time.sleep(0.2)
    assert srv.poll(wait_ms=50) == []                # B still waits for memory
    st = srv.stats()
    assert st["admitted"] == 1 and st["bytes_in_use"] <= budget
    srv.close_session(sa)                            # A retires, B is admitted
    got_b = {c["tag"] - 1000: c for c in drain(srv, len(ib))}
    st = srv.stats()
    assert st["admitted"] == 2 and st["closed"] >= 1 and st["bytes_in_use"] <= budget
    srv.close()
    twin = Space(b_sp.grids, b_sp.invalid, precision="fp16x3", n_max=64)
    o = O.OracleSession(b_sp.grids, b_sp.invalid)
    for r in range(len(ib)):
        twin.observe(int(ib[r]), float(yb[r]))
        o.observe(int(ib[r]), float(yb[r]))
        ref = twin.suggest()
        orc = o.suggest()
        c = got_b[r]
        assert c["status"] == 0 and c["observed"], c
        assert c["idx"] == ref["idx"] or \
            abs(c["info"]["score"] - ref["score"]) <= 1e-6 * max(abs(ref["score"]), 1), r
        p = o.last_pass
        assert pick_ok(p["scores"]["ei"], c["idx"], orc["idx"], **REDUCED), (r, c["idx"], orc["idx"])
        assert abs(c["info"]["mu"] - p["mu"][c["idx"]]) <= 1e-3 * max(abs(p["mu"][c["idx"]]), 1.0)
        assert abs(c["info"]["sigma"] - p["sigma"][c["idx"]]) <= 1e-3
    twin.close()
