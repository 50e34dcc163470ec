"""FP64 oracle of the smoothing lengths of Sec. 3.1: for every particle the
distance to its k-th nearest other particle in 3D (the paper prefers the 3D
neighbour distance; the workloads use k = 32).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Distances are taken in FP64 on the given (float32-rounded) positions, the
values the GPU receives.  Small sets are searched by brute force (every
pair); larger ones with scipy's cKDTree (a library neighbour search).
"""
from __future__ import annotations

import numpy as np


def kth_neighbour_distance_brute(xyz, k):
    """All pairs: sort each particle's distances to the others."""
    p = np.asarray(xyz, np.float64)
    n = p.shape[0]
    if n <= k:
        raise ValueError("need more than k particles")
    out = np.empty(n)
    for s in range(0, n, 512):
        d2 = ((p[s:s + 512, None, :] - p[None, :, :]) ** 2).sum(axis=2)
        idx = np.arange(s, min(s + 512, n))
        d2[idx - s, idx] = np.inf  # the particle itself
        out[s:s + 512] = np.sqrt(np.partition(d2, k - 1, axis=1)[:, k - 1])
    return out


def kth_neighbour_distance_tree(xyz, k, workers=-1):
    """The same through scipy's cKDTree (query k + 1 including the point itself)."""
    from scipy.spatial import cKDTree
    p = np.asarray(xyz, np.float64)
    if p.shape[0] <= k:
        raise ValueError("need more than k particles")
    d, i = cKDTree(p).query(p, k=k + 1, workers=workers)
    # duplicates: the point itself may come after an identical neighbour;
    # either way the k + 1 smallest distances include the zero of the self-pair
    return d[:, k]


def kth_neighbour_distance(xyz, k, brute_max=4000):
    n = np.asarray(xyz).shape[0]
    return kth_neighbour_distance_brute(xyz, k) if n <= brute_max else kth_neighbour_distance_tree(xyz, k)
