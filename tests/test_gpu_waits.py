"""Bounded device waits: failure detection without a GPU fault.

Every wait in the library's kernels (mbarrier phases of the prediction
kernel's roles, grid barriers of the fused observation update) gives up after
its limit, records BO_ERR_TIMEOUT and lets the kernel return.  bo_selftest_waits
makes one wait of each kind run out on purpose (a phase nothing completes; a
grid barrier one of two blocks never reaches); the test checks the recorded
status, that it took the limit (not a fault), and that the context still runs a
normal prediction pass afterwards.
"""
import time

import numpy as np
import pytest

from paper_2111_14991_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BO_ERR_TIMEOUT = 8


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2111_14991_gb300 import build
    build.build()


def test_bounded_waits_report_timeout_and_context_survives():
    import torch
    from paper_2111_14991_gb300 import Space, bo
    t0 = time.time()
    mbar, grid = bo.selftest_waits()
    took = time.time() - t0
    assert mbar == BO_ERR_TIMEOUT and grid == BO_ERR_TIMEOUT, (mbar, grid)
    assert 3.5 < took < 30.0, took                 # two waits of 2 s each ran out
    sp = W.config1_space()
    land = W.Landscape(sp, 1)
    idx = W.clustered_observations(land, 24, 1)
    s = Space(sp.grids, sp.invalid, precision="fp16x3", n_max=32)
    for i in idx:
        s.observe(int(i), float(land.clean([i])[0]))
    mu, var = s.predict()
    s.close()
    torch.cuda.synchronize()
    assert np.all(np.isfinite(mu)) and np.all(np.isfinite(var))
