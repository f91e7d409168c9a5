"""Oracle initial sample of a search space (paper Sec. III-E, Table I).

Test infrastructure only (see the package docstring).  The paper first takes
a Latin hypercube sample of the search space, then replaces every invalid
sample by a random one until all initial samples are valid; Table I selects
the "maximin" variant.  The steps below follow that order.

Readings (the paper gives no formulas for these; the draw order is fixed so
that an independent implementation can be compared index for index):
  * The hypercube is over the parameters' value lists: with n samples, each
    parameter's unit interval is cut into n strata, a random permutation
    assigns strata to samples, a uniform jitter places each sample inside its
    stratum at u, and the parameter takes value index floor(u * m) of its m
    values (exactly, in integers).
  * "maximin" keeps, of `designs` such hypercubes, the first one whose
    smallest pairwise squared Euclidean distance between the samples'
    normalized parameter values is largest (the paper does not say how many
    are compared; 100 by default).
  * Invalid means restricted (not in the valid list); a sample repeating an
    earlier one is replaced too.  Replacements are uniform over the valid
    list, drawn in sample order, redrawn while already taken.
  * Random numbers: one splitmix64 stream (Steele, Lea and Flood 2014) seeded
    with `seed`; Fisher-Yates (Durstenfeld) shuffles j = next() mod (i + 1)
    for i from n-1 down to 1; jitters U = (next() >> 11) / 2**53; random valid
    picks next() mod N_valid.
"""
from __future__ import annotations

import numpy as np

from .bo_oracle import valid_list

__all__ = ["latin_hypercube", "min_pair_sq_distance", "initial_design"]


def _splitmix64(seed):
    """A function returning successive splitmix64 outputs, from its published
    definition."""
    m64 = (1 << 64) - 1
    state = [seed & m64]

    def draw():
        state[0] = (state[0] + 0x9E3779B97F4A7C15) & m64
        z = state[0]
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m64
        return z ^ (z >> 31)
    return draw


def latin_hypercube(sizes, n, draw):
    """One Latin hypercube of n samples over parameters with `sizes` values:
    an (n, d) array of value indices (Sec. III-E)."""
    d = len(sizes)
    out = np.zeros((n, d), dtype=np.int64)
    for p in range(d):
        strata = list(range(n))
        for i in range(n - 1, 0, -1):
            j = draw() % (i + 1)
            strata[i], strata[j] = strata[j], strata[i]
        for i in range(n):
            jitter = draw() >> 11                # U = jitter / 2**53
            # floor(u * m) with u = (stratum + U) / n, in exact integers
            out[i, p] = ((strata[i] << 53) + jitter) * sizes[p] // (n << 53)
    return out


def min_pair_sq_distance(points):
    """Smallest squared Euclidean distance between two rows of `points`
    (the maximin criterion); the per-parameter terms are added in order."""
    n, d = points.shape
    best = np.inf
    for i in range(n):
        for j in range(i + 1, n):
            s = 0.0
            for p in range(d):
                df = float(points[i, p]) - float(points[j, p])
                s = s + df * df
            best = min(best, s)
    return best


def initial_design(grids, invalid_mask, count, mode="maximin", designs=100, seed=0, draw=None):
    """Valid-list indices of the initial sample (Sec. III-E): 'random',
    'lhs' or 'maximin'.  Random numbers come from `draw()` when given (a
    session's own stream, which the sample advances), else from a fresh
    splitmix64 stream seeded with `seed`."""
    grids = [np.asarray(g, dtype=np.float64) for g in grids]
    sizes = [len(g) for g in grids]
    flat, _ = valid_list(sizes, invalid_mask)
    position = {int(f): i for i, f in enumerate(flat)}
    n_valid = len(flat)
    if not 1 <= count <= n_valid:
        raise ValueError("count out of range")
    if draw is None:
        draw = _splitmix64(seed)
    taken = set()

    def random_valid():
        while True:
            r = draw() % n_valid
            if r not in taken:
                taken.add(r)
                return r

    if mode == "random":
        return np.array([random_valid() for _ in range(count)], dtype=np.int64)

    # 1. Latin hypercube(s); maximin keeps the best spread of `designs`
    rounds = max(designs, 1) if mode == "maximin" else 1
    best, best_score = None, None
    for t in range(rounds):
        v = latin_hypercube(sizes, count, draw)
        score = 0.0
        if rounds > 1 and count > 1:
            pts = np.array([[grids[p][v[i, p]] for p in range(len(sizes))] for i in range(count)])
            score = min_pair_sq_distance(pts)
        if best is None or score > best_score:
            best, best_score = v, score
    # 2. configurations; restricted or repeated samples are replaced at random
    chosen = []
    for i in range(count):
        f = 0
        for p in range(len(sizes)):
            f = f * sizes[p] + int(best[i, p])
        idx = position.get(f, -1)
        if idx >= 0 and idx not in taken:
            taken.add(idx)
            chosen.append(idx)
        else:
            chosen.append(-1)
    return np.array([c if c >= 0 else random_valid() for c in chosen], dtype=np.int64)
