"""Parity tolerances of the GPU path against the FP64 oracle.

Errors are relative to max(|ref|, 1): 1 is the prior standard deviation in
standardized units (k(0) = 1, std(y~) = 1).  The posterior mean crosses zero
and the standard deviation vanishes at observations, so a relative error needs
a scale there, and below it FP64 itself is not exact: with cond(K) ~ 3e8
(nu = 5/2, l = 0.8, 80 clustered points) two FP64 algorithms -- the oracle's
triangular solves and the incremental inverse -- already differ by ~5e-9.
FP64 mode: 1e-6.  Reduced-precision modes (FP32 accumulation): 1e-3.
"""
import numpy as np

FP64 = dict(rel=1e-6, floor=1.0)
REDUCED = dict(rel=1e-3, floor=1.0)


def tol_for(precision):
    return FP64 if precision == "fp64" else REDUCED


def scaled_err(got, ref, floor):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(got - ref) / np.maximum(np.abs(ref), floor)


def assert_close(got, ref, rel, floor, what=""):
    err = scaled_err(got, ref, floor)
    worst = int(np.argmax(err)) if err.size else 0
    assert err.size == 0 or err[worst] <= rel, (
        f"{what}: max scaled error {err[worst]:.3e} > {rel:.1e} at {worst} "
        f"(got {np.ravel(got)[worst]!r}, ref {np.ravel(ref)[worst]!r})")
    return float(err.max()) if err.size else 0.0


def pick_ok(scores_ref, got_idx, ref_idx, rel, floor):
    """The GPU pick is correct if it is the oracle's, or if the oracle scores it
    within tolerance of the oracle's own best (the top values are that close)."""
    if got_idx == ref_idx:
        return True
    a, b = float(scores_ref[got_idx]), float(scores_ref[ref_idx])
    return abs(a - b) <= rel * max(abs(b), floor)
