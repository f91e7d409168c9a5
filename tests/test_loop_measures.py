"""The tuning-quality measures of Sec. IV (host code, no device)."""
import numpy as np
import pytest


def test_loop_measures_follow_the_protocol():
    """Sec. IV: MAE averages |f(best after 20 i) - f_opt| for i = 2..11; the
    MDF divides each kernel's mean MAE by its mean over strategies."""
    from paper_2111_14991_gb300.loop import best_found, mae, mdf
    idx = np.arange(220)
    vals = np.linspace(10.0, 1.0, 220)              # strictly improving: best = last seen
    vals[5] = np.nan                                # failed evaluations never count
    truth = lambda i: float(i)                      # true value = index
    assert best_found(idx, vals, 40) == 39
    assert mae(idx, vals, truth, 0.0) == pytest.approx(np.mean([20 * i - 1 for i in range(2, 12)]))
    f = mdf({"a": {"k1": 1.0, "k2": 4.0}, "b": {"k1": 3.0, "k2": 4.0}})
    assert f["a"][0] == pytest.approx((0.5 + 1.0) / 2) and f["b"][0] == pytest.approx((1.5 + 1.0) / 2)
