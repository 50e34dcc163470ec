"""FP64 oracle of the cell-refinement step (Sec. 3.4 interpolation, App. A).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): used by the tests and by
nothing in the product library.

Rays sit on a uniform grid: ray (i, j) at (x0 + i h, y0 + j h), flat index
i + nx j.  Each ray is the centre of a cell of side h; its neighbours are the
four edge-adjacent rays E (i+1, j), N (i, j+1), W (i-1, j), S (i, j-1).  A
cell is refined into k x k sub-cells (k odd) whose centres are
x_c + (d_a, d_b), d_a = (a - (k-1)/2) h / k.

Uniformity test and magnification matrix (two modes):

* KAPPA_GAMMA: the cell is uniform if kappa, gamma1 and gamma2 at every
  neighbour are within tol of the centre's; A is Eq. magmatrix at the centre,
  [[1 - kappa - gamma1, -gamma2], [-gamma2, 1 - kappa + gamma1]].
* DEFLECTION (App. A): source positions y = x - alpha (lens equation); for
  every pair of neighbours not colinear with the centre (E-N, N-W, W-S, S-E)
  the three points give A by the App. A solve of dy = A dx; the cell is
  uniform if no element of A differs by more than tol between pairs, and A is
  the average over the pairs.

Sub-cell source positions follow Eq. linear_lens_equation,
y = y_c + A (x - x_c), for uniform cells; non-uniform cells get NaN (the
caller shoots those rays with the full solver).

A is reported as (a11, a21, a12, a22) with A = [[a11, a21], [a12, a22]]:
dy1 = a11 dx1 + a21 dx2, dy2 = a12 dx1 + a22 dx2 (the App. A layout).
"""
from __future__ import annotations

import numpy as np

KAPPA_GAMMA, DEFLECTION = 0, 1

# neighbour offsets (di, dj) and the four pairs not colinear with the centre
NEIGHBOURS = ((1, 0), (0, 1), (-1, 0), (0, -1))  # E, N, W, S
PAIRS = ((0, 1), (1, 2), (2, 3), (3, 0))          # E-N, N-W, W-S, S-E


def app_a_solve(dx1, dy1, dx2, dy2):
    """App. A: A from two displacement pairs dy^(n) = A dx^(n).  dx*, dy* are
    (..., 2) arrays; returns (a11, a21, a12, a22) and det."""
    det = dx1[..., 0] * dx2[..., 1] - dx1[..., 1] * dx2[..., 0]
    a11 = (dx2[..., 1] * dy1[..., 0] - dx1[..., 1] * dy2[..., 0]) / det
    a22 = (dx1[..., 0] * dy2[..., 1] - dx2[..., 0] * dy1[..., 1]) / det
    a12 = (dx2[..., 1] * dy1[..., 1] - dx1[..., 1] * dy2[..., 1]) / det
    a21 = (dx1[..., 0] * dy2[..., 0] - dx2[..., 0] * dy1[..., 0]) / det
    return np.stack([a11, a21, a12, a22], axis=-1), det


def refine_cells(x0, y0, h, nx, ny, alpha1, alpha2, kappa, gamma1, gamma2, cells, k, tol, mode):
    """Returns (uniform (n,) bool, A (n, 4), y_sub (n, k, k, 2) [b, a, xy],
    stat (n,)): stat is the largest neighbour difference (KAPPA_GAMMA) or
    element spread between pairs (DEFLECTION) that was compared with tol."""
    cells = np.asarray(cells, np.int64)
    i, j = cells % nx, cells // nx
    if np.any((i < 1) | (i > nx - 2) | (j < 1) | (j > ny - 2)):
        raise ValueError("cells must be interior")
    a1 = np.asarray(alpha1, np.float64)
    a2 = np.asarray(alpha2, np.float64)
    xc = np.stack([x0 + i * h, y0 + j * h], axis=-1)
    yc = xc - np.stack([a1[cells], a2[cells]], axis=-1)
    if mode == KAPPA_GAMMA:
        q = [np.asarray(v, np.float64) for v in (kappa, gamma1, gamma2)]
        stat = np.zeros(cells.size)
        for di, dj in NEIGHBOURS:
            nb = (i + di) + nx * (j + dj)
            for v in q:
                stat = np.maximum(stat, np.abs(v[nb] - v[cells]))
        ka, g1, g2 = (v[cells] for v in q)
        A = np.stack([1.0 - ka - g1, -g2, -g2, 1.0 - ka + g1], axis=-1)
    elif mode == DEFLECTION:
        dxs, dys = [], []
        for di, dj in NEIGHBOURS:
            nb = (i + di) + nx * (j + dj)
            dx = np.broadcast_to(np.array([di * h, dj * h]), (cells.size, 2))
            dy = dx - np.stack([a1[nb] - a1[cells], a2[nb] - a2[cells]], axis=-1)
            dxs.append(dx)
            dys.append(dy)
        As = np.stack([app_a_solve(dxs[p], dys[p], dxs[q], dys[q])[0] for p, q in PAIRS], axis=1)
        stat = (As.max(axis=1) - As.min(axis=1)).max(axis=1)
        A = As.mean(axis=1)
    else:
        raise ValueError("mode")
    uniform = stat <= tol
    d = (np.arange(k) - (k - 1) / 2) * h / k
    db, da = np.meshgrid(d, d, indexing="ij")  # [b, a]
    ys = np.empty((cells.size, k, k, 2))
    ys[..., 0] = yc[:, None, None, 0] + A[:, None, None, 0] * da + A[:, None, None, 1] * db
    ys[..., 1] = yc[:, None, None, 1] + A[:, None, None, 2] * da + A[:, None, None, 3] * db
    ys[~uniform] = np.nan
    return uniform, A, ys, stat


def interior_cells(nx, ny):
    """Flat indices of every interior ray of an nx x ny grid."""
    i, j = np.meshgrid(np.arange(1, nx - 1), np.arange(1, ny - 1), indexing="xy")
    return (i + nx * j).ravel().astype(np.int64)
