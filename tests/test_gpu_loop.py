"""Whole tuning runs through the library (Sec. III-A loop, Sec. IV protocol:
20 initial samples + 200 suggestions) on the paper-shaped synthetic kernels:
the fast suggest keeps the method's behaviour -- it beats random search on
every kernel, in FP64 and in the FP16x3 form."""
import numpy as np
import pytest

from paper_2111_14991_gb300 import workloads as W
from paper_2111_14991_gb300.loop import mae, mdf, minimize, random_search

pytestmark = pytest.mark.gpu

KERNELS = ["gemm", "conv", "pnpoly", "expdist", "adding"]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2111_14991_gb300 import build
    build.build()


def problem(name, rep):
    sp = W.paper_shaped_space(name)
    land = W.Landscape(sp, 100 + rep)
    ok = np.ones(sp.n_valid, bool) if sp.runtime_invalid is None else ~sp.runtime_invalid
    f_opt = float(np.min(land.clean(np.flatnonzero(ok))))
    return sp, land, (lambda i: float(land.clean([i])[0])), f_opt


def test_bo_beats_random_search_on_every_kernel():
    reps_bo, reps_rnd = 2, 6
    mean_mae = {"fp64": {}, "fp16x3": {}, "random": {}}
    for name in KERNELS:
        for prec in ("fp64", "fp16x3"):
            errs = []
            for r in range(reps_bo):
                sp, land, truth, f_opt = problem(name, r)
                idx, val = minimize(land, sp.grids, sp.invalid, budget=220, n_init=20, seed=r, precision=prec)
                assert len(idx) == 220 and len(set(idx.tolist())) == 220
                errs.append(mae(idx, val, truth, f_opt))
            mean_mae[prec][name] = float(np.mean(errs))
        errs = []
        for r in range(reps_rnd):
            sp, land, truth, f_opt = problem(name, r)
            idx, val = random_search(land, sp.n_valid, budget=220, seed=r)
            errs.append(mae(idx, val, truth, f_opt))
        mean_mae["random"][name] = float(np.mean(errs))
    for name in KERNELS:
        assert mean_mae["fp64"][name] < mean_mae["random"][name], (name, mean_mae)
        assert mean_mae["fp16x3"][name] < mean_mae["random"][name], (name, mean_mae)
    f = mdf(mean_mae)
    assert f["fp64"][0] < f["random"][0] and f["fp16x3"][0] < f["random"][0], f
