"""Oracle for image finding by adaptive grid refinement (Sec. 4) and the SIS
finite-source magnification it is tested against (Sec. 5.2, App. B).

TEST INFRASTRUCTURE ONLY (see the package docstring): plain Python and numpy,
FP64, slow, written from the paper's description step by step.

sis_finite_source_mu(b, R, r_e)
    App. B: magnification of a uniform circular source of radius R whose
    centre is at distance b from an SIS of Einstein radius r_e, by the 1D
    integrals of the point magnifications mu_+- = 1 +- r_e/|y| over the disk.

find_images(alpha, sources, prm)
    Sec. 4 for uniform circular sources: telescoping source sizes on a grid of
    cells refined by thirds, images as connected sets of cells whose source
    points fall in the source (neighbours of neighbours), inner and outer
    borders, a uniform refinement to n_min cells per image, then refinement of
    the largest border cells until each image's largest border cell is a
    fraction f_area of its area (and the outer border is as fine as the inner
    one), with a level cap as the minimum grid size.

The readings (where the paper leaves a choice):
  I1 a cell (L, i, j) has side h_L = S / (N 3^L) and centre
     (x0 + (i + 1/2) h_L, y0 + (j + 1/2) h_L); refining makes its 9 children
     (L+1, 3i+a, 3j+b); the middle child keeps the parent's ray (same centre).
  I2 the "source size" of a circle is its radius: telescoping starts at
     r_0 = h_0 / sqrt(mu_min) (an image of magnification mu_min then has the
     radius of a coarse cell and always holds a grid point) and divides by 3
     while above R, then uses R; at each size r, cells with a source point
     inside (|y - y_c| < r) and h_L > r sqrt(mu_min) / 3 are refined,
     repeatedly, until none remain.
  I3 neighbours share an edge; an image is a connected set of image cells.
  I4 inner border: image cells with a non-image neighbour; outer border:
     non-image cells with an image neighbour (of each image they touch).
  I5 uniform step: while an image has fewer than n_min cells, refine all its
     cells and its outer border.
  I6 border step: an image is done when its largest border cell (inner or
     outer) has area below f_area times the image's area and its outer
     border's largest cell is no larger than its inner border's largest;
     otherwise its border cells (inner and outer) of the largest size are
     refined.  Cells at level L_max are never refined.
  I7 the image area is the sum of its cells' areas (per-level cell counts
     times h_L^2, summed from level 0 up); mu = area / (pi R^2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.integrate import quad


# ------------------------------------------------------------ App. B (SIS)

def _half_angle(s, b, R):
    """Half the angle of the circle |y| = s (about the lens) inside the disk
    |y - y_c| <= R, |y_c| = b."""
    if s <= R - b:
        return math.pi
    if s <= abs(b - R) or s >= b + R:
        return 0.0
    c = (s * s + b * b - R * R) / (2.0 * s * b)
    return math.acos(min(1.0, max(-1.0, c)))


def sis_finite_source_mu(b: float, R: float, r_e: float = 1.0):
    """(mu_plus, |mu_minus|, ring) for a uniform disk source (App. B).

    mu_+ = 1 + r_e <1/|y|>,  |mu_-| = <(r_e/|y| - 1) [|y| < r_e]>, averages
    over the disk; in polar coordinates about the lens the disk meets the
    circle |y| = s in an arc of half-angle phi(s), so
    int 1/|y| d^2y = 2 int phi(s) ds and int d^2y = 2 int s phi(s) ds.
    ring: the source covers the lens centre (b < R): the two images join
    into one (Sec. 5.2 counts it as one image of magnification mu_+ + |mu_-|).
    """
    area = math.pi * R * R
    lo, hi = max(0.0, b - R), b + R
    pts = [p for p in (R - b, abs(b - R)) if lo < p < hi]
    f1 = lambda s: 2.0 * _half_angle(s, b, R)
    fa = lambda s: 2.0 * s * _half_angle(s, b, R)
    i1, _ = quad(f1, lo, hi, points=pts or None, epsabs=0, epsrel=1e-12, limit=400)
    mu_p = 1.0 + r_e * i1 / area
    if lo >= r_e:
        mu_m = 0.0
    else:
        top = min(hi, r_e)
        pts_m = [p for p in pts if p < top]
        j1, _ = quad(f1, lo, top, points=pts_m or None, epsabs=0, epsrel=1e-12, limit=400)
        ja, _ = quad(fa, lo, top, points=pts_m or None, epsabs=0, epsrel=1e-12, limit=400)
        mu_m = (r_e * j1 - ja) / area
    return mu_p, mu_m, b < R


# ------------------------------------------------------------ image finding

@dataclass
class AmrParams:
    x0: float           # lower-left corner of the initial grid
    y0: float
    side: float         # S: the initial grid covers [x0, x0+S] x [y0, y0+S]
    n: int              # N x N initial cells
    l_max: int = 12     # minimum grid size h_0 / 3^l_max
    mu_min: float = 0.01
    f_area: float = 5e-4
    n_min: int = 50


def cell_size(prm: AmrParams, L: int) -> float:
    return prm.side / float(prm.n * 3 ** L)


def cell_centre(prm: AmrParams, L: int, i: int, j: int):
    h = cell_size(prm, L)
    return prm.x0 + (i + 0.5) * h, prm.y0 + (j + 0.5) * h


def code(prm: AmrParams, L: int, i: int, j: int) -> int:
    """Order of cells for canonical image labels: the level-0 cell index,
    then one base-9 digit 3 a + b per level (a, b the child's column, row),
    padded to level l_max (the smallest code a cell covers)."""
    s = 3 ** L
    c = (i // s) * prm.n + (j // s)
    for lv in range(1, L + 1):
        d = 3 ** (L - lv)
        c = c * 9 + 3 * ((i // d) % 3) + ((j // d) % 3)
    return c * 9 ** (prm.l_max - L)


class _Grid:
    """Leaf cells of one source's grid: (L, i, j) -> source point (yx, yy)."""

    def __init__(self, prm, alpha):
        self.prm, self.alpha = prm, alpha
        self.leaves = {}
        self.rays = 0
        cells = [(0, i, j) for i in range(prm.n) for j in range(prm.n)]
        self._shoot(cells)

    def _shoot(self, cells):
        if not cells:
            return
        xy = np.array([cell_centre(self.prm, *c) for c in cells], dtype=np.float64)
        a1, a2 = self.alpha(xy[:, 0], xy[:, 1])
        for c, (x, y), b1, b2 in zip(cells, xy, a1, a2):
            self.leaves[c] = (x - b1, y - b2)
        self.rays += len(cells)

    def refine(self, cells):
        new = []
        for (L, i, j) in cells:
            if L >= self.prm.l_max or (L, i, j) not in self.leaves:
                continue
            y = self.leaves.pop((L, i, j))
            for a in range(3):
                for b in range(3):
                    ch = (L + 1, 3 * i + a, 3 * j + b)
                    if a == 1 and b == 1:
                        self.leaves[ch] = y          # I1: the middle child keeps the ray
                    else:
                        new.append(ch)
        self._shoot(new)
        return len(new)

    def inside(self, yc, r):
        r2 = r * r
        return {c for c, y in self.leaves.items()
                if (y[0] - yc[0]) * (y[0] - yc[0]) + (y[1] - yc[1]) * (y[1] - yc[1]) < r2}

    def _container(self, L, i, j):
        """The leaf at level <= L containing cell (L, i, j), or None."""
        for lv in range(L, -1, -1):
            d = 3 ** (L - lv)
            c = (lv, i // d, j // d)
            if c in self.leaves:
                return c
        return None

    def adjacent_pairs(self):
        """Every pair of leaves sharing an edge, once (I3)."""
        top = self.prm.n
        pairs = set()
        for (L, i, j) in self.leaves:
            lim = top * 3 ** L
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                ni, nj = i + di, j + dj
                if not (0 <= ni < lim and 0 <= nj < lim):
                    continue
                nb = self._container(L, ni, nj)
                if nb is not None:    # a finer neighbour finds this leaf itself
                    pairs.add(tuple(sorted([(L, i, j), nb])))
        return pairs


def _images(grid, yc, r):
    """Images (neighbours of neighbours), their inner and outer borders (I3, I4)."""
    inside = grid.inside(yc, r)
    pairs = grid.adjacent_pairs()
    nbrs = {}
    for a, b in pairs:
        nbrs.setdefault(a, []).append(b)
        nbrs.setdefault(b, []).append(a)
    label = {}
    images = []
    for c in sorted(inside, key=lambda c: code(grid.prm, *c)):
        if c in label:
            continue
        comp, stack = [], [c]
        label[c] = len(images)
        while stack:
            u = stack.pop()
            comp.append(u)
            for v in nbrs.get(u, ()):
                if v in inside and v not in label:
                    label[v] = len(images)
                    stack.append(v)
        images.append(comp)
    inner = [set() for _ in images]
    outer = [set() for _ in images]
    for a, b in pairs:
        if (a in inside) != (b in inside):
            ci, co = (a, b) if a in inside else (b, a)
            inner[label[ci]].add(ci)
            outer[label[ci]].add(co)
    return images, inner, outer


def _area(prm, cells):
    counts = [0] * (prm.l_max + 1)
    for (L, _, _) in cells:
        counts[L] += 1
    a = 0.0
    for L in range(prm.l_max + 1):
        h = cell_size(prm, L)
        a += counts[L] * (h * h)
    return a


def find_images(alpha, sources, prm: AmrParams, with_cells=False):
    """Images of each uniform circular source (yc_x, yc_y, R) (Sec. 4).

    alpha(x, y) -> (alpha1, alpha2) FP64 arrays.  Returns per source a dict:
    images (list of dicts: n_cells, area, mu, first = the image's smallest
    code), rays (rays shot), leaves (final leaf count) and, with with_cells,
    the final leaf set and the image cells.
    """
    out = []
    h0 = cell_size(prm, 0)
    smu = math.sqrt(prm.mu_min)
    for (ycx, ycy, R) in sources:
        yc = (ycx, ycy)
        g = _Grid(prm, alpha)
        # telescoping (I2)
        r = h0 / smu
        if r < R:
            r = R
        while True:
            thr = r * smu / 3.0
            while True:
                sel = [c for c in g.inside(yc, r)
                       if cell_size(prm, c[0]) > thr and c[0] < prm.l_max]
                if not sel or g.refine(sel) == 0:
                    break
            if r <= R:
                break
            r = r / 3.0
            if r < R:
                r = R
        # uniform step (I5)
        while True:
            imgs, inner, outer = _images(g, yc, R)
            sel = set()
            for k, comp in enumerate(imgs):
                if len(comp) < prm.n_min:
                    sel.update(comp)
                    sel.update(outer[k])
            sel = [c for c in sel if c[0] < prm.l_max]
            if not sel or g.refine(sel) == 0:
                break
        # border step (I6)
        while True:
            imgs, inner, outer = _images(g, yc, R)
            sel = []
            for k, comp in enumerate(imgs):
                area = _area(prm, comp)
                lin = min((c[0] for c in inner[k]), default=prm.l_max)
                lout = min((c[0] for c in outer[k]), default=prm.l_max)
                lb = min(lin, lout)
                hb = cell_size(prm, lb)
                done = (hb * hb < prm.f_area * area and lout >= lin) or lb >= prm.l_max
                if not done:
                    sel += [c for c in inner[k] | outer[k] if c[0] == lb]
            if not sel or g.refine(sel) == 0:
                break
        imgs, inner, outer = _images(g, yc, R)
        res = []
        for comp in imgs:
            area = _area(prm, comp)
            res.append({"n_cells": len(comp), "area": area, "mu": area / (math.pi * R * R),
                        "first": min(code(prm, *c) for c in comp)})
        rec = {"images": res, "rays": g.rays, "leaves": len(g.leaves)}
        if with_cells:
            rec["leaf_set"] = set(g.leaves)
            rec["image_cells"] = [sorted(c) for c in imgs]
        out.append(rec)
    return out
