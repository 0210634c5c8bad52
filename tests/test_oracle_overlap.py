"""Pins of the oracle's enclosing-sphere overlap test (App. I-C assumes that the enclosing
spheres of the scatterers do not intersect): hand-made configurations with known answers."""
import numpy as np

from oracle import geometry


def test_touching_spheres_do_not_overlap():
    pos = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [1.0, 0.0, 0.0]])
    assert geometry.first_overlap(pos, [0.25, 0.25, 0.25]) is None  # 0.5^2 == (0.25 + 0.25)^2


def test_nearly_touching_spheres_overlap():
    pos = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    assert geometry.first_overlap(pos, [0.25, 0.25 + 2 ** -40]) == (0, 1)


def test_three_dimensional_separation_counts():
    # (0.3, 0.4, 1.2): distance 1.3; radii summing to 1.29 / 1.31
    pos = np.array([[0.0, 0.0, 0.0], [0.3, 0.4, 1.2]])
    assert geometry.first_overlap(pos, [0.6, 0.69]) is None
    assert geometry.first_overlap(pos, [0.6, 0.71]) == (0, 1)


def test_first_pair_is_the_smallest_i_then_j():
    pos = np.array([[0.0, 0.0, 0.0], [5.0, 0.0, 0.0], [5.1, 0.0, 0.0], [0.05, 0.0, 0.0], [0.1, 0.0, 0.0]])
    r = [0.01, 0.1, 0.1, 0.01, 0.01]
    # overlaps: (1, 2) and (3, 4): d = 0.05 > 0.02, so only (1, 2)
    assert geometry.first_overlap(pos, r) == (1, 2)
    r[0] = 0.2  # now (0, 3) and (0, 4) overlap too; (0, 3) comes first
    assert geometry.first_overlap(pos, r) == (0, 3)
