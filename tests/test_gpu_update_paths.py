"""The two forms of the single-space observation update agree.

By default a space's FP64 update (k, l = L^-1 k, w, then the pivot row with
beta and alpha) runs as one cooperative launch; with BO_NO_COOP set at
creation it runs as four phase launches.  Both must give the same factor and posterior: the only
difference is the block width of the pivot's reduction, whose last-bit
difference the conditioning of K (about 1e7 here) can amplify; so the results
must agree to 1e-9 of their scale (the FP64 parity bar is 1e-6) in FP64 mode,
and to 1e-5 in FP16x3 mode (bar 1e-3), on a space fed the same observations.
"""
import os

import numpy as np
import pytest

from paper_2111_14991_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2111_14991_gb300 import build
    build.build()


def fitted(sp, idx, y, precision, coop):
    from paper_2111_14991_gb300 import Space
    old = os.environ.pop("BO_NO_COOP", None)
    if not coop:
        os.environ["BO_NO_COOP"] = "1"
    try:
        s = Space(sp.grids, sp.invalid, precision=precision, n_max=128)
    finally:
        os.environ.pop("BO_NO_COOP", None)
        if old is not None:
            os.environ["BO_NO_COOP"] = old
    for i, v in zip(idx, y):
        s.observe(int(i), float(v))
    s.sync()
    linv, beta = s.factor()
    mu, var = s.predict()
    launches = s.launch_count()
    s.close()
    return linv, beta, np.asarray(mu, dtype=np.float64), np.asarray(var, dtype=np.float64), launches


@pytest.mark.parametrize("precision", ["fp64", "fp16x3"])
def test_cooperative_and_phase_updates_agree(precision):
    sp = W.config1_space()
    land = W.Landscape(sp, 4)
    idx = W.clustered_observations(land, 100, 4)
    y = [float(land.clean([i])[0]) for i in idx]
    a = fitted(sp, idx, y, precision, coop=True)
    b = fitted(sp, idx, y, precision, coop=False)
    for x, z in zip(a[:2], b[:2]):                 # L^-1 and beta, FP64 in both modes
        assert np.max(np.abs(x - z)) <= 1e-9 * max(1.0, float(np.max(np.abs(z)))), precision
    tol = 1e-9 if precision == "fp64" else 1e-5
    assert np.max(np.abs(a[2] - b[2])) <= tol and np.max(np.abs(a[3] - b[3])) <= tol, precision
    assert a[4] < b[4]                              # one launch per update instead of several


def suggest_run(sp, land, precision, fused, steps=25, seed=3):
    """EI suggestions with the given observations fed in order; with fused
    (BO_FUSED_ACQ) the tensor-core pass carries the acquisition as its tail
    (one cooperative launch), without it the acquisition is its own launch."""
    from paper_2111_14991_gb300 import Space
    old = os.environ.pop("BO_FUSED_ACQ", None)
    if fused:
        os.environ["BO_FUSED_ACQ"] = "1"
    try:
        s = Space(sp.grids, sp.invalid, precision=precision, n_max=128)
    finally:
        os.environ.pop("BO_FUSED_ACQ", None)
        if old is not None:
            os.environ["BO_FUSED_ACQ"] = old
    for i in W.random_initial_sample(sp.n_valid, 20, seed):
        s.observe(int(i), float(land.clean([i])[0]))
    out = []
    for _ in range(steps):
        r = s.suggest()
        out.append(r)
        s.observe(r["idx"], float(land.clean([r["idx"]])[0]))
    launches = s.launch_count()
    s.close()
    return out, launches


@pytest.mark.parametrize("precision", ["fp16x3", "tf32x3"])
def test_fused_and_separate_acquisition_agree(precision):
    """The acquisition tail of the prediction pass and the separate acquisition
    kernel score with the same FP32 arithmetic and keep the same (score, index)
    order: the same suggestions, scores, lambda and mean variance."""
    sp = W.paper_shaped_space("pnpoly")
    land = W.Landscape(sp, 9)
    a, la = suggest_run(sp, land, precision, fused=True)
    b, lb = suggest_run(sp, land, precision, fused=False)
    for t, (x, z) in enumerate(zip(a, b)):
        assert x["idx"] == z["idx"], (t, x, z)
        assert x["score"] == z["score"] and x["mu"] == z["mu"] and x["sigma"] == z["sigma"], (t, x, z)
        assert x["lam"] == pytest.approx(z["lam"], rel=1e-12)
        assert x["mean_var"] == pytest.approx(z["mean_var"], rel=1e-12)
    assert la < lb                                  # one launch per pass instead of two


PDL_CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, ".")
from paper_2111_14991_gb300 import Space, build
from paper_2111_14991_gb300 import workloads as W
build.build()
sp = W.paper_shaped_space("pnpoly")
land = W.Landscape(sp, 11)
out = {}
for precision in ("fp16x3", "fp64"):
    s = Space(sp.grids, sp.invalid, precision=precision, n_max=64)
    for i in W.random_initial_sample(sp.n_valid, 20, 11):
        s.observe(int(i), float(land.clean([i])[0]))
    picks = []
    for _ in range(10):
        r = s.suggest()
        picks.append([int(r["idx"]), float(r["score"]), float(r["lam"])])
        s.observe(r["idx"], float(land.clean([r["idx"]])[0]))
    mu, var = s.predict()
    s.close()
    out[precision] = dict(picks=picks, mu=float(np.sum(np.abs(mu))), var=float(np.sum(var)))
print(json.dumps(out))
"""


def test_dependent_launches_change_nothing():
    """Programmatic dependent launches (the default) and plain launches
    (BO_NO_PDL, read once per process: each setting runs in its own process)
    give the same suggestions, scores and posteriors, bit for bit."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = []
    for pdl in (True, False):
        env = dict(os.environ)
        env.pop("BO_NO_PDL", None)
        if not pdl:
            env["BO_NO_PDL"] = "1"
        r = subprocess.run([sys.executable, "-c", PDL_CHILD], cwd=root, env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        res.append(json.loads(r.stdout.strip().splitlines()[-1]))
    assert res[0] == res[1]
