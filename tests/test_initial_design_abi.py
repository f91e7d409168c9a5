"""bo_initial_design (host code of the library, no device) against the oracle:
the same valid-list indices, index for index (integer work: bit-exact)."""
import numpy as np
import pytest

import oracle.sampling as S
from paper_2111_14991_gb300 import workloads as W


@pytest.fixture(scope="module")
def bo():
    from paper_2111_14991_gb300 import build
    build.build()
    from paper_2111_14991_gb300 import bo as B
    return B


SPACES = {
    "config1": W.config1_space,
    "conv": lambda: W.paper_shaped_space("conv"),
    "gemm15": lambda: W.paper_shaped_space("gemm"),
    "tiny": lambda: W.generic_space(5, 3, 7),
}


@pytest.mark.parametrize("name", list(SPACES))
@pytest.mark.parametrize("mode", ["random", "lhs", "maximin"])
@pytest.mark.parametrize("seed", [0, 99])
def test_library_equals_oracle(bo, name, mode, seed):
    sp = SPACES[name]()
    count = min(20, sp.n_valid)
    designs = 25
    lib = bo.initial_design(sp.grids, sp.invalid, count, init=mode, init_designs=designs, seed=seed)
    ref = S.initial_design(sp.grids, sp.invalid, count, mode, designs, seed)
    np.testing.assert_array_equal(lib, ref)


def test_whole_space_and_errors(bo):
    sp = W.generic_space(5, 3, 7)
    all_idx = bo.initial_design(sp.grids, sp.invalid, sp.n_valid, init="maximin", seed=3)
    assert sorted(all_idx.tolist()) == list(range(sp.n_valid))
    from paper_2111_14991_gb300 import BOError
    with pytest.raises(BOError):
        bo.initial_design(sp.grids, sp.invalid, sp.n_valid + 1, init="lhs")
    with pytest.raises(BOError):
        bo.initial_design(sp.grids, sp.invalid, 0, init="lhs")
