"""Plain FP64 CPU oracle of the Bayesian-optimization suggest step.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
link anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is written from the paper (Willemsen, van Nieuwpoort, van Werkhoven,
"Bayesian Optimization for auto-tuning GPU kernels"), shares no code with the
CUDA library, and computes everything in IEEE double precision with numpy /
scipy primitives (Cholesky, triangular solve, Euclidean distance, erfc) as
single steps.  Each function cites the passage it follows.

Parity status of each part (what pins it, see tests/test_oracle_*.py):
  matern            pinned: closed forms, scipy Bessel form of the Matern family
  gp_posterior      pinned: brute-force rational inverse, sklearn GPR, invariants
  acquisition       pinned: closed-form EI / PI values, limits, Monte Carlo
  contextual λ      pinned: exact ratio at the first pass, linearity
  argmax / top-k    pinned: brute force
  dos               pinned: hand sums
  initial sample    pinned: Latin property (one value / stratum per parameter),
                    brute-force 2x2 designs, maximin monotone in the number of
                    designs and above its first design, restricted samples
                    replaced with the valid ones kept in place
  multi / adv-multi selection
                    parity unpinned against the paper (it prints no trace);
                    pinned only to the readings of Sec. III-G listed in the
                    docstrings, by scripted scenarios.
"""
from .bo_oracle import *  # noqa: F401,F403
from .selection import *  # noqa: F401,F403
from .sampling import *  # noqa: F401,F403
from .session import *  # noqa: F401,F403
