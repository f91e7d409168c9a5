"""Selection order of the acquisition pass on the GPU (both posterior types).

The masked top-3 per acquisition function is defined as: higher score first,
equal scores to the lower valid-list index (ties go to the lower index, reading
c14), evaluated candidates never selected, a NaN score never wins.  The FP32
pass keeps (score, index) as one packed 64-bit key; these cases pin that its
order is exactly this one, on inputs whose scores are exact (sigma = 0 gives
EI = max(delta, 0), PI = [delta > 0], LCB = -mu with no rounding) or exactly
tied, so the expected lists follow from the definition without any tolerance.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EI, PI, LCB = 0, 1, 2


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2111_14991_gb300 import build
    build.build()


def expected_top3(scores, visited):
    order = sorted((i for i in range(len(scores)) if not visited[i] and not np.isnan(scores[i])),
                   key=lambda i: (-scores[i], i))
    return order[:3]


def run_pass(mu, var, visited, f64, fplus=0.0, lam=0.0):
    import torch
    from paper_2111_14991_gb300 import bo
    n = len(mu)
    dt = torch.float64 if f64 else torch.float32
    words = np.zeros((n + 31) // 32, dtype=np.uint32)
    for i in np.flatnonzero(visited):
        words[i >> 5] |= np.uint32(1) << np.uint32(i & 31)
    dev = torch.device("cuda")
    t_mu = torch.tensor(mu, dtype=dt, device=dev)
    t_var = torch.tensor(var, dtype=dt, device=dev)
    t_vis = torch.tensor(words.view(np.int32), device=dev)
    t_res = torch.zeros(C.sizeof(bo.PassResult), dtype=torch.uint8, device=dev)
    p = bo.AcqParams()
    p.n_cand, p.n_unvisited = n, int(n - visited.sum())
    p.sum_var = float(np.nansum(np.where(visited, 0.0, var)))
    p.n_af = 3
    p.af[0], p.af[1], p.af[2] = EI, PI, LCB
    p.explore, p.n_fit, p.lambda_const = 1, 10, lam          # constant exploration factor
    p.fplus, p.fplus_raw, p.mu_s_raw, p.mean_var_s = fplus, 1.0, 1.0, 1.0
    bo.acquire_noalloc(t_mu.data_ptr(), t_var.data_ptr(), t_vis.data_ptr(), 1 if f64 else 0, p,
                       t_res.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return bo.pass_result_dict(bo.PassResult.from_buffer_copy(t_res.cpu().numpy().tobytes()))


@pytest.mark.parametrize("f64", [0, 1])
def test_exact_ties_go_to_the_lowest_unvisited_index(f64):
    n = 70_000                                  # several blocks of the pass, a ragged tail
    mu = np.full(n, 0.25)
    var = np.full(n, 0.5)
    visited = np.zeros(n, dtype=bool)
    visited[[0, 2, 5]] = True
    got = run_pass(mu, var, visited, f64, fplus=0.1, lam=0.01)
    for q in range(3):
        assert list(got["top_idx"][q]) == [1, 3, 4], (f64, q, got["top_idx"][q])


@pytest.mark.parametrize("f64", [0, 1])
def test_signed_scores_order_and_zero_ties(f64):
    """sigma = 0: LCB = -mu over mixed signs; EI = max(-mu, 0); PI = [mu < 0]."""
    rng = np.random.default_rng(7)
    n = 50_003
    mu = rng.permutation(np.arange(n, dtype=np.float64) - 20_000.0) / 64.0   # exact in FP32
    var = np.zeros(n)
    visited = np.zeros(n, dtype=bool)
    best = np.argsort(mu)[:5]                   # the five most negative means
    visited[best[[0, 2]]] = True                # the best and the third are evaluated
    got = run_pass(mu, var, visited, f64, fplus=0.0, lam=0.0)
    lcb = -mu
    ei = np.maximum(-mu, 0.0)
    pi = (mu < 0).astype(np.float64)
    assert list(got["top_idx"][EI]) == expected_top3(ei, visited)
    assert list(got["top_idx"][LCB]) == expected_top3(lcb, visited)
    assert list(got["top_idx"][PI]) == expected_top3(pi, visited)      # ties at 1: lowest indices
    assert list(got["top_idx"][LCB]) == [int(best[1]), int(best[3]), int(best[4])]
    assert got["top_score"][LCB][0] == pytest.approx(-mu[best[1]], rel=0, abs=0)


@pytest.mark.parametrize("f64", [0, 1])
def test_nan_posterior_never_wins(f64):
    n = 5_000
    mu = np.linspace(1.0, 2.0, n)               # sigma = 0: EI = PI = 0 (ties), LCB = -mu
    var = np.zeros(n)
    mu[10], var[10] = np.nan, 0.5               # z = NaN: every score of candidate 10 is NaN
    visited = np.zeros(n, dtype=bool)
    got = run_pass(mu, var, visited, f64, fplus=0.0, lam=0.0)
    for q in range(3):
        assert 10 not in list(got["top_idx"][q]), (f64, q)
    assert list(got["top_idx"][LCB]) == [0, 1, 2]
