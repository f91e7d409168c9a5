"""Parity tolerances of the GPU path against the FP64 oracle.

Two error measures are computed for mu and sigma:

* scaled: |got - ref| / max(|ref|, 1).  1 is the prior standard deviation in
  standardized units (k(0) = 1, std(y~) = 1), so below it the error is
  absolute.  The posterior mean crosses zero and sigma vanishes at
  observations, so a relative error needs a scale there.
* strict: |got - ref| / max(|ref|, 1e-3), relative down to a thousandth of
  the prior standard deviation.

FP64 mode must meet 1e-6 in both measures.  The reduced-precision modes
(FP32 K*, FP32 accumulation) must meet 1e-3 scaled; their strict error is
reported beside it, together with the bound the FP32 arithmetic puts on it
(see strict_bound_mu / strict_bound_var): K* carries a relative rounding of
a few 2^-24 per element, which reaches mu amplified by sum_j |alpha_j k*_j|
and sigma^2 by 2 sum_j |w_j k*_j| (w = K^-1 k*), at any operand split.
"""
import numpy as np

FP64 = dict(rel=1e-6, floor=1.0)
REDUCED = dict(rel=1e-3, floor=1.0)
STRICT_FLOOR = 1e-3
FP64_STRICT = dict(rel=1e-6, floor=STRICT_FLOOR)
U32 = 2.0 ** -24


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


def parity_report(tag, mu, rmu, var, rvar, rel):
    """Scaled and strict errors of mu and sigma, and the share of candidates
    whose strict error exceeds rel; printed as one PARITY line."""
    sd, rsd = np.sqrt(np.maximum(var, 0.0)), np.sqrt(np.maximum(rvar, 0.0))
    r = {}
    for name, g, o in (("mu", mu, rmu), ("sigma", sd, rsd)):
        sc = scaled_err(g, o, 1.0)
        st = scaled_err(g, o, STRICT_FLOOR)
        r[name] = dict(scaled=float(sc.max()), strict=float(st.max()), strict_over=float(np.mean(st > rel)))
    print(f"PARITY {tag}: mu scaled {r['mu']['scaled']:.2e} strict {r['mu']['strict']:.2e} "
          f"(over {r['mu']['strict_over']:.1%}) | sigma scaled {r['sigma']['scaled']:.2e} strict "
          f"{r['sigma']['strict']:.2e} (over {r['sigma']['strict_over']:.1%})")
    return r


def pick_ok(scores_ref, got_idx, ref_idx, rel, floor):
    """The GPU pick is correct if it is the oracle's, or if the oracle scores it
    within tolerance of the oracle's own best (the top values are that close)."""
    if got_idx == ref_idx:
        return True
    a, b = float(scores_ref[got_idx]), float(scores_ref[ref_idx])
    return abs(a - b) <= rel * max(abs(b), floor)
