"""Pins of the smoothing-length oracle (oracle/knn.py): a cubic lattice,
whose neighbour shells are known in closed form; brute force and the k-d tree
agree on clustered sets; duplicates; the scaling of distances."""
import numpy as np
import pytest

import lensgen
from oracle import knn


def lattice(n):
    g = np.arange(n, dtype=np.float64)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def test_cubic_lattice_shells():
    # neighbours of an interior site: 6 at a, 12 at a sqrt2, 8 at a sqrt3, 6 at 2a, 24 at a sqrt5
    a = 0.25
    p = lattice(9) * a
    centre = (np.abs(p / a - 4) <= 2).all(axis=1)  # sites at least 2 from every face
    for k, d in [(1, a), (6, a), (7, a * np.sqrt(2)), (18, a * np.sqrt(2)), (19, a * np.sqrt(3)),
                 (26, a * np.sqrt(3)), (27, 2 * a), (32, 2 * a), (33, a * np.sqrt(5))]:
        got = knn.kth_neighbour_distance_brute(p, k)
        np.testing.assert_allclose(got[centre], d, rtol=1e-12)


def test_brute_force_and_tree_agree_on_clustered_points():
    xyz = lensgen.nfw_positions_3d(3000, 11)
    for k in (1, 8, 32):
        np.testing.assert_allclose(knn.kth_neighbour_distance_brute(xyz, k),
                                   knn.kth_neighbour_distance_tree(xyz, k), rtol=1e-12)


def test_duplicates_and_scaling():
    g = np.random.default_rng(3)
    p = g.normal(size=(400, 3))
    q = np.concatenate([p, p[:50]])  # 50 points appear twice
    d = knn.kth_neighbour_distance_brute(q, 1)
    assert (d[:50] == 0).all() and (d[400:] == 0).all() and (d[50:400] > 0).all()
    np.testing.assert_allclose(knn.kth_neighbour_distance_brute(3.5 * p, 9),
                               3.5 * knn.kth_neighbour_distance_brute(p, 9), rtol=1e-12)
    with pytest.raises(ValueError):
        knn.kth_neighbour_distance_brute(p[:5], 5)
