"""GB300-native suggest step of Bayesian optimization for GPU-kernel tuning.

    from paper_2111_14991_gb300 import Space
    s = Space(grids, invalid_mask, af="advanced_multi", precision="fp16x3")
    s.observe(idx, runtime); nxt = s.suggest()["idx"]

`Space` wraps the C ABI of include/bo_suggest.h (libbo_suggest.so, built by
paper_2111_14991_gb300.build).  `workloads` holds the seeded synthetic inputs.
"""
from .bo import Batch, BOError, Server, Space, lib  # noqa: F401

__all__ = ["Space", "Batch", "Server", "BOError", "lib"]
