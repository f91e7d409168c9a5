"""Seeded synthetic inputs: search spaces, tuning landscapes, observation lists.

This module only *generates inputs*. It holds none of the method's arithmetic
(no kernel function, no GP, no acquisition function), so both the CPU oracle
and the CUDA path can be fed from it.

Search spaces follow the paper's representation (Sec. III-C): every numeric
parameter has a discrete list of values, each list is mapped linearly to
[0, 1] by its position (so powers of two become equally spaced), and the
space is the Cartesian product minus the configurations a restriction marks
invalid.  Products are enumerated row-major with the last parameter fastest.

The objective stands in for running a tuned GPU kernel: a smooth bowl plus a
sinusoidal roughness term, times 5 % log-normal noise, in milliseconds.
Runtime-invalid configurations (those that compile-or-run fail, Sec. III-C.2)
return NaN.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Space", "Landscape", "config1_space", "config2_space", "config3_space",
    "batched_spaces", "batched_specs", "batched_space", "paper_shaped_space", "PAPER_SHAPED", "generic_space",
    "random_initial_sample", "clustered_observations",
]


@dataclass
class Space:
    """A discrete, normalized, constrained search space.

    values[p]  raw parameter values of parameter p
    grids[p]   normalized values in [0, 1] (index-linear), float64
    invalid    uint8 mask over the Cartesian product (1 = restricted)
    """
    name: str
    names: list
    values: list
    grids: list
    invalid: np.ndarray
    runtime_invalid: np.ndarray | None = None   # bool over the valid list
    meta: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        return len(self.grids)

    @property
    def sizes(self) -> list:
        return [len(g) for g in self.grids]

    @property
    def total(self) -> int:
        return int(np.prod(self.sizes, dtype=np.int64))

    def valid_flat(self) -> np.ndarray:
        """Flat product indices of the valid configurations, ascending."""
        return np.flatnonzero(self.invalid == 0).astype(np.int64)

    def valid_codes(self) -> np.ndarray:
        """Per-parameter value indices of the valid configurations, N x d."""
        flat = self.valid_flat()
        return np.stack(np.unravel_index(flat, self.sizes), axis=1).astype(np.int32)

    def valid_coords(self) -> np.ndarray:
        codes = self.valid_codes()
        return np.stack([self.grids[p][codes[:, p]] for p in range(self.d)], axis=1)

    @property
    def n_valid(self) -> int:
        return int(np.count_nonzero(self.invalid == 0))


def _index_linear(m: int) -> np.ndarray:
    if m == 1:
        return np.zeros(1)
    return np.arange(m, dtype=np.float64) / (m - 1)


def _product(values):
    return np.meshgrid(*[np.asarray(v, dtype=np.float64) for v in values], indexing="ij")


def _make(name, names, values, invalid_fn, **meta) -> Space:
    mesh = _product(values)
    invalid = invalid_fn(*mesh).reshape(-1).astype(np.uint8)
    grids = [_index_linear(len(v)) for v in values]
    return Space(name, list(names), [np.asarray(v, dtype=np.float64) for v in values],
                 grids, invalid, meta=dict(meta))


def config1_space() -> Space:
    """4 integer params: 5,120 configurations, 2,560 valid."""
    values = [np.arange(16, 513, 16), [1, 2, 4, 8, 16], np.arange(1, 9), [0, 1, 2, 4]]
    return _make("blocks-4p", ["block_x", "block_y", "tile", "unroll"], values,
                 lambda bx, by, t, u: (bx * by > 1024) | (bx * t > 2048))


def _gemm_like_invalid(bx, by, tx, ty, vec, unroll, cache):
    smem = (bx * tx + by * ty) * vec * 16 * (1 + cache)
    regs = tx * ty * vec / 2 + 2 * unroll + 24
    return (bx * by > 1024) | (smem > 96 * 1024) | (regs > 128)


_GEMM7 = [np.arange(16, 321, 16), [1, 2, 4, 8, 16, 32], np.arange(1, 9), np.arange(1, 9),
          [1, 2, 4, 8], [0, 1, 2, 4], [0, 1]]
_GEMM7_NAMES = ["block_x", "block_y", "tile_x", "tile_y", "vec", "unroll", "cache"]


def config2_space() -> Space:
    """7-param GEMM-tiling-like grid: 245,760 configurations, 113,247 valid."""
    return _make("gemm-7p", _GEMM7_NAMES, _GEMM7, _gemm_like_invalid)


def config3_space() -> Space:
    """9 params (the 7 above + k-split, stages): 3,932,160 configurations, 1,032,469 valid."""
    values = _GEMM7 + [[1, 2, 4, 8], [1, 2, 3, 4]]

    def invalid(bx, by, tx, ty, vec, unroll, cache, ksplit, stages):
        smem = (bx * tx + by * ty) * vec * 16 * (1 + cache)
        regs = tx * ty * vec / 2 + 2 * unroll + 24
        threads = bx * by
        return (threads < 64) | (threads > 1024) | (smem * stages > 64 * 1024) | \
               (regs + 4 * ksplit > 128)
    return _make("gemm-9p", _GEMM7_NAMES + ["ksplit", "stages"], values, invalid)


# ---------------------------------------------------------------------------
# generic spaces: batched sessions and the paper-shaped set

def _grid_sizes(rng, d, target_total):
    """Per-parameter list lengths (>= 2) whose product is close to target_total."""
    base = target_total ** (1.0 / d)
    sizes = [max(2, int(round(base * math.exp(rng.uniform(-0.35, 0.35))))) for _ in range(d)]
    for _ in range(200):
        prod = float(np.prod(sizes))
        if abs(math.log(prod / target_total)) < 0.08:
            break
        p = int(rng.integers(d))
        if prod > target_total and sizes[p] > 2:
            sizes[p] -= 1
        elif prod < target_total:
            sizes[p] += 1
    return sizes


def generic_space(seed: int, d: int, n_valid: int, name: str = "generic",
                  oversample: float = 2.5) -> Space:
    """d params with list sizes whose product is ~oversample * n_valid.

    A seeded weighted-sum restriction on the normalized coordinates keeps
    exactly the n_valid configurations with the smallest weighted sum (ties
    broken by product order), so the valid count is hit exactly.
    """
    rng = np.random.default_rng(seed)
    total_target = max(int(oversample * n_valid), n_valid + 1)
    sizes = _grid_sizes(rng, d, total_target)
    while int(np.prod(sizes)) < n_valid:
        sizes[int(rng.integers(d))] += 1
    grids = [_index_linear(m) for m in sizes]
    w = rng.uniform(0.5, 1.5, size=d)
    total = int(np.prod(sizes))
    s = np.zeros(total)
    idx = np.arange(total, dtype=np.int64)
    stride = 1
    for p in range(d - 1, -1, -1):
        s += w[p] * grids[p][(idx // stride) % sizes[p]]
        stride *= sizes[p]
    order = np.argsort(s, kind="stable")
    invalid = np.ones(total, dtype=np.uint8)
    invalid[order[:n_valid]] = 0
    values = [np.arange(m, dtype=np.float64) for m in sizes]
    return Space(name, [f"p{p}" for p in range(d)], values, grids, invalid,
                 meta={"seed": seed})


# Sizes (valid count, runtime-invalid count, d) of the paper's search spaces
# on the GTX Titan X and the A100 (Table 2, Table 3, Sec. IV-E).
PAPER_SHAPED = {
    "gemm":    dict(d=15, n=17956, runtime_invalid=0),
    "conv":    dict(d=8, n=9400, runtime_invalid=3624),
    "pnpoly":  dict(d=5, n=8184, runtime_invalid=323),
    "expdist": dict(d=7, n=14400, runtime_invalid=7320),
    "adding":  dict(d=4, n=4654, runtime_invalid=0),
}


def paper_shaped_space(kind: str, seed: int = 0) -> Space:
    """A generic space with the paper's size, dimensionality and invalid share.

    Runtime-invalid configurations are clustered: the ones nearest to a few
    seeded centres in normalized coordinates.
    """
    spec = PAPER_SHAPED[kind]
    sp = generic_space(seed * 7919 + 17 + len(kind), spec["d"], spec["n"],
                       name=f"paper-{kind}", oversample=1.6)
    k = spec["runtime_invalid"]
    ri = np.zeros(sp.n_valid, dtype=bool)
    if k:
        rng = np.random.default_rng(seed + 31)
        coords = sp.valid_coords()
        centres = rng.uniform(0, 1, size=(3, sp.d))
        dist = np.min(np.stack([np.sum((coords - c) ** 2, axis=1) for c in centres]), axis=0)
        ri[np.argsort(dist, kind="stable")[:k]] = True
    sp.runtime_invalid = ri
    return sp


def batched_specs(count: int = 256, seed: int = 0, n_min: int = 1000, n_max: int = 500_000):
    """(d, n_valid, n_obs) of each uneven session: d ~ U{3..9},
    N ~ log-uniform[n_min, n_max], n_obs ~ U{20..400}."""
    rng = np.random.default_rng(seed + 4242)
    out = []
    for _ in range(count):
        d = int(rng.integers(3, 10))
        n_valid = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        n_obs = int(rng.integers(20, 401))
        out.append((d, n_valid, n_obs))
    return out


def batched_space(seed: int, s: int, spec) -> Space:
    """Session s of the batched configuration with spec (d, n_valid, n_obs)."""
    d, n_valid, n_obs = spec
    sp = generic_space(seed * 100003 + s, d, n_valid, name=f"batched-{s}")
    sp.meta.update(n_obs=n_obs, session=s)
    return sp


def batched_spaces(count: int = 256, seed: int = 0, n_min: int = 1000, n_max: int = 500_000):
    """Uneven sessions: d ~ U{3..9}, N ~ log-uniform[n_min, n_max], n_obs ~ U{20..400}."""
    return [batched_space(seed, s, spec) for s, spec in enumerate(batched_specs(count, seed, n_min, n_max))]


# ---------------------------------------------------------------------------
# landscapes and observation lists

class Landscape:
    """t(x) = t0 [1 + 4 sum w_k (x_k - c_k)^2 + 0.3 sum (1 + sin(2 pi om_k x_k + ph_k)) / 2]
    times exp(0.05 eps), eps ~ N(0, 1) per evaluation; x in normalized coordinates."""

    def __init__(self, space: Space, seed: int, t0: float = 1.0, noise: float = 0.05):
        rng = np.random.default_rng(seed)
        d = space.d
        self.space = space
        self.c = rng.uniform(0.15, 0.85, size=d)
        self.w = rng.uniform(0.5, 2.0, size=d)
        self.om = rng.integers(1, 5, size=d).astype(np.float64)
        self.ph = rng.uniform(0.0, 2 * math.pi, size=d)
        self.t0 = t0
        self.noise = noise
        self.noise_rng = np.random.default_rng(seed + 2000)
        self._coords = None

    def coords(self) -> np.ndarray:
        if self._coords is None:
            self._coords = self.space.valid_coords()
        return self._coords

    def clean(self, idx) -> np.ndarray:
        """Noise-free objective at valid-list indices."""
        x = self.coords()[np.asarray(idx, dtype=np.int64)]
        bowl = 4.0 * np.sum(self.w * (x - self.c) ** 2, axis=-1)
        rough = 0.3 * np.sum(0.5 * (1 + np.sin(2 * math.pi * self.om * x + self.ph)), axis=-1)
        return self.t0 * (1.0 + bowl + rough)

    def __call__(self, idx) -> float:
        """One noisy evaluation at a valid-list index (NaN if runtime-invalid)."""
        idx = int(idx)
        ri = self.space.runtime_invalid
        eps = self.noise_rng.standard_normal()
        if ri is not None and ri[idx]:
            return float("nan")
        return float(self.clean([idx])[0] * math.exp(self.noise * eps))


def random_initial_sample(n_valid: int, count: int, seed: int) -> np.ndarray:
    """count distinct valid-list indices drawn uniformly (seeded)."""
    rng = np.random.default_rng(seed + 1000)
    return rng.choice(n_valid, size=min(count, n_valid), replace=False).astype(np.int64)


def clustered_observations(land: Landscape, count: int, seed: int, n_random: int = 20,
                           temperature: float = 0.15, pool: int = 200_000) -> np.ndarray:
    """Distinct valid-list indices shaped like a BO trace: n_random uniform
    picks, then picks drawn without replacement with probability proportional
    to exp(-(t(x) - t_min) / (temperature * t_min)), so they crowd the good
    region the way acquisition-driven picks do."""
    n_valid = land.space.n_valid
    rng = np.random.default_rng(seed + 5000)
    first = random_initial_sample(n_valid, min(n_random, count), seed)
    if count <= len(first):
        return first[:count]
    cand = np.arange(n_valid) if n_valid <= pool else rng.choice(n_valid, pool, replace=False)
    cand = np.setdiff1d(cand, first)
    t = land.clean(cand)
    logits = -(t - t.min()) / (temperature * t.min())
    p = np.exp(logits - logits.max())
    p /= p.sum()
    rest = rng.choice(cand, size=min(count - len(first), int(np.count_nonzero(p))),
                      replace=False, p=p)
    return np.concatenate([first, rest]).astype(np.int64)
