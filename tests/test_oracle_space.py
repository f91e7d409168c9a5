"""The oracle's candidate set (Sec. III-D) against a hand-enumerated space.

A 2 x 3 product with two restricted configurations, written out by hand:
row-major order with the last parameter fastest, restricted entries removed,
coordinates read from each parameter's normalized grid.  A column-major
enumeration, a mask applied in the other order, or swapped grids fail here.
"""
import numpy as np

import oracle as O

GRIDS = [np.array([0.0, 1.0]), np.array([0.0, 0.25, 1.0])]
# product order (p0, p1): (0,0) (0,1) (0,2) (1,0) (1,1) (1,2); flat 1 and 3 restricted
MASK = np.array([0, 1, 0, 1, 0, 0], dtype=np.uint8)
FLAT = [0, 2, 4, 5]
CODES = [[0, 0], [0, 2], [1, 1], [1, 2]]
COORDS = [[0.0, 0.0], [0.0, 1.0], [1.0, 0.25], [1.0, 1.0]]


def test_valid_list_hand_enumerated():
    flat, codes = O.valid_list([2, 3], MASK)
    assert flat.tolist() == FLAT
    assert codes.tolist() == CODES


def test_valid_list_without_mask_is_the_whole_product():
    flat, codes = O.valid_list([2, 3], None)
    assert flat.tolist() == list(range(6))
    assert codes.tolist() == [[0, 0], [0, 1], [0, 2], [1, 0], [1, 1], [1, 2]]


def test_candidate_coords_hand_enumerated():
    _, codes = O.valid_list([2, 3], MASK)
    assert O.candidate_coords(GRIDS, codes).tolist() == COORDS


def test_mask_as_a_product_shaped_array():
    flat, _ = O.valid_list([2, 3], MASK.reshape(2, 3))
    assert flat.tolist() == FLAT
