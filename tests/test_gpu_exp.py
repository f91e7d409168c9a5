"""The exponential of the FP64 prediction pass against CUDA's exp and numpy.

The FP64 pass evaluates e^-t of the Matern covariance (paper Sec. III-B) with
its own table-driven reduction (Tang, ACM TOMS 1989) instead of a general exp.
Its error bound: 1.3 ulp with a correctly rounded table (host check of the
same steps), plus the table's own rounding (CUDA's exp2, at most 1 ulp), so
3 ulp of either reference.  Covers small t (no reduction), the range the
covariance meets (t <= 10), the whole accepted range (t <= 700), the exact
table points t = k ln2/64, and the cut-off above 700 (0) and NaN (kept).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2111_14991_gb300 import build
    build.build()


def test_exp_neg_within_three_ulp():
    from paper_2111_14991_gb300 import bo
    rng = np.random.default_rng(7)
    t = np.concatenate([
        np.linspace(0.0, 1e-3, 5001),
        rng.uniform(0.0, 10.0, 400_000),
        rng.uniform(0.0, 700.0, 200_000),
        np.arange(0, 4000) * (np.log(2.0) / 64.0),
    ])
    out, ref = bo.selftest_exp(t)
    want = np.exp(-t)
    ulp = np.spacing(want)
    err_np = np.abs(out - want) / ulp
    err_cuda = np.abs(out - ref) / np.spacing(ref)
    print(f"PARITY exp_neg: max {err_np.max():.2f} ulp vs numpy, {err_cuda.max():.2f} ulp vs CUDA exp")
    assert err_np.max() <= 3.0, t[np.argmax(err_np)]
    assert err_cuda.max() <= 3.0, t[np.argmax(err_cuda)]
    assert out[0] == 1.0


def test_exp_neg_cutoff_and_nan():
    from paper_2111_14991_gb300 import bo
    t = np.array([700.0, 700.5, 745.0, 1e6, np.inf, np.nan])
    out, _ = bo.selftest_exp(t)
    assert out[0] > 0.0 and abs(out[0] - np.exp(-700.0)) <= 3 * np.spacing(np.exp(-700.0))
    assert np.all(out[1:5] == 0.0)
    assert np.isnan(out[5])
