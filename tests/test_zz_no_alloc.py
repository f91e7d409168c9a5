"""The allocation-free acquisition entry point (bo_acquire_noalloc).

Callers that cannot allocate device memory at the call site (a fixed memory
arena, device memory reserved up front by another framework, a loop where an
allocation is not allowed) score a posterior they already hold with this entry
point; its scratch is a fixed array inside the library.  Here it must give the
same pass result as the session's own acquisition (bo_replay_*) on the same
posterior, on two calls in a row (the second reuses the array the first left).
This file is collected last so that a run stopping at the first failure has run
every other test already.
"""
import ctypes as C
import math

import numpy as np
import pytest

from paper_2111_14991_gb300 import workloads as W
from tolerances import FP64, REDUCED

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2111_14991_gb300 import build
    build.build()


def sequential_stats(y):
    """Mean, population std and minimum summed in observation order."""
    m = 0.0
    for v in y:
        m += v
    m /= len(y)
    s = 0.0
    for v in y:
        s += (v - m) * (v - m)
    s = math.sqrt(s / len(y))
    return m, (s if s != 0.0 else 1.0), min(y)


@pytest.mark.parametrize("precision", ["fp16x3", "fp64"])
def test_noalloc_matches_session_pass_twice(precision):
    """FP32 posteriors (packed score/index keys in the scratch) and FP64
    posteriors (separate scores and indices): both partial layouts."""
    import torch
    from paper_2111_14991_gb300 import Space
    from paper_2111_14991_gb300 import bo
    f64 = precision == "fp64"
    tol = FP64 if f64 else REDUCED
    sp = W.config2_space()
    land = W.Landscape(sp, 3)
    idx = W.clustered_observations(land, 60, 3)
    y = [float(land.clean([i])[0]) for i in idx]
    s = Space(sp.grids, sp.invalid, precision=precision, n_max=64)
    for i, v in zip(idx[:59], y[:59]):
        s.observe(int(i), v)
    s.replay_enqueue(idx[59:], y[59:])
    ref = s.replay_fetch(1)[0]
    mu, var = s.predict()                     # the same posterior (same state, same kernel)
    s.close()

    N = sp.n_valid
    words = np.zeros((N + 31) // 32, dtype=np.uint32)
    for i in idx:
        words[i >> 5] |= np.uint32(1) << np.uint32(i & 31)
    dev = torch.device("cuda")
    ftype = torch.float64 if f64 else torch.float32
    t_mu = torch.tensor(mu, dtype=ftype, device=dev)
    t_var = torch.tensor(var, dtype=ftype, device=dev)
    t_vis = torch.tensor(words.view(np.int32), device=dev)
    t_res = torch.zeros(C.sizeof(bo.PassResult), dtype=torch.uint8, device=dev)
    mean, sd, ymin = sequential_stats(y)
    p = bo.AcqParams()
    p.n_cand, p.n_unvisited, p.sum_var = N, N - len(idx), ref["sum_var"]
    p.n_af = 3
    p.af[0], p.af[1], p.af[2] = 0, 1, 2
    p.explore, p.n_fit, p.lambda_const = 0, len(idx), 0.01
    p.fplus, p.fplus_raw, p.mu_s_raw = (ymin - mean) / sd, ymin, mean
    p.mean_var_s = ref["mean_var_s"]
    stream = torch.cuda.current_stream()
    for call in range(2):
        t_res.zero_()
        bo.acquire_noalloc(t_mu.data_ptr(), t_var.data_ptr(), t_vis.data_ptr(), int(f64), p,
                           t_res.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got = bo.pass_result_dict(bo.PassResult.from_buffer_copy(t_res.cpu().numpy().tobytes()))
        assert got["status"] == 0 and got["n_scored"] == N - len(idx), (call, got)
        assert got["mean_var"] == pytest.approx(ref["mean_var"], rel=1e-12)
        assert got["lam"] == pytest.approx(ref["lam"], rel=1e-9)
        for q in range(3):
            for k in range(3):
                a, b = got["top_score"][q][k], ref["top_score"][q][k]
                assert abs(a - b) <= tol["rel"] * max(abs(b), tol["floor"]), (call, q, k)
            assert got["top_idx"][q][0] == ref["top_idx"][q][0] or \
                abs(got["top_score"][q][0] - ref["top_score"][q][0]) <= 1e-6, (call, q)


def test_noalloc_rejects_too_many_candidates():
    from paper_2111_14991_gb300 import bo
    p = bo.AcqParams()
    p.n_cand = 4194304 + 1
    p.n_unvisited = 10
    p.n_af = 1
    with pytest.raises(bo.BOError) as e:
        bo.acquire_noalloc(16, 16, 16, 0, p, 16, 0)    # rejected before any device access
    assert e.value.code == 11 and "fixed scratch" in str(e.value)


def test_noalloc_rejects_unknown_explore_mode():
    from paper_2111_14991_gb300 import bo
    p = bo.AcqParams()
    p.n_cand, p.n_unvisited, p.n_af = 100, 10, 1
    p.explore = 7
    with pytest.raises(bo.BOError) as e:
        bo.acquire_noalloc(16, 16, 16, 0, p, 16, 0)    # rejected before any device access
    assert e.value.code == 1 and "explore" in str(e.value)
