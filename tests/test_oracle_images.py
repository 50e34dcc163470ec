"""Pins of the image-finding oracle (Sec. 4) and of the App. B finite-source
SIS magnification it is tested against (Sec. 5.2).

* App. B integrals: the centred source's closed form (mu = 4 r_e / R for the
  ring, 1 + 2 r_e / R for the outer part), the point-source limit
  mu = 1 +- r_e / b, and a Monte Carlo average of the point magnification over
  the disk;
* the grid: leaves tile the initial grid exactly, every leaf has its own ray,
  the edge-neighbour relation equals a brute-force geometric test;
* the images: each is a maximal connected set of cells whose source points
  are inside the source, the stopping rule holds at the end, image counts
  follow the SIS (two images inside r_e, one outside, one ring when the
  source covers the lens), and the magnifications are within the paper's
  0.7 % of App. B (Sec. 5.2).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import images as I

SIS = oracle.make_components(oracle.SIS, 0.0, 0.0, 0.0, 1.0)


def alpha_sis(x, y):
    o = oracle.direct_sum(SIS, x, y)
    return o[:, 0], o[:, 1]


def sis_params(**kw):
    return I.AmrParams(-10.0, -10.0, 20.0, 64, **kw)


# ------------------------------------------------------------ App. B

@pytest.mark.parametrize("R", [0.01, 0.1, 0.5, 0.9])
def test_centred_source_closed_form(R):
    mp, mm, ring = I.sis_finite_source_mu(0.0, R)
    # <1/|y|> over a centred disk = 2/R; inside r_e all of it
    assert ring
    assert mp == pytest.approx(1.0 + 2.0 / R, rel=1e-12)
    assert mm == pytest.approx(2.0 / R - 1.0, rel=1e-12)
    assert mp + mm == pytest.approx(4.0 / R, rel=1e-12)


@pytest.mark.parametrize("b", [0.3, 0.7, 1.6])
def test_point_source_limit(b):
    R = 1e-4 * b
    mp, mm, ring = I.sis_finite_source_mu(b, R)
    assert not ring
    assert mp == pytest.approx(1.0 + 1.0 / b, rel=1e-7)
    assert mm == pytest.approx(max(0.0, 1.0 / b - 1.0), rel=1e-7, abs=1e-12)


@pytest.mark.parametrize("b,R", [(0.5, 0.3), (0.95, 0.1), (1.2, 0.4), (0.1, 0.3)])
def test_monte_carlo_average(b, R):
    g = np.random.default_rng(11)
    n = 2_000_000
    r = R * np.sqrt(g.random(n))
    t = 2 * np.pi * g.random(n)
    s = np.hypot(b + r * np.cos(t), r * np.sin(t))
    mp, mm, _ = I.sis_finite_source_mu(b, R)
    fp = 1.0 + 1.0 / s
    fm = np.where(s < 1.0, 1.0 / s - 1.0, 0.0)
    assert abs(fp.mean() - mp) < 5 * fp.std() / math.sqrt(n)
    assert abs(fm.mean() - mm) < 5 * fm.std() / math.sqrt(n) + 1e-12


# ------------------------------------------------------------ the grid

def test_neighbours_match_geometry():
    """adjacent_pairs on an irregular grid equals the pairs of leaves whose
    closed squares share a segment of positive length."""
    prm = I.AmrParams(0.0, 0.0, 1.0, 3, l_max=4)
    g = I._Grid(prm, lambda x, y: (np.zeros_like(x), np.zeros_like(y)))
    rng = np.random.default_rng(3)
    for _ in range(6):
        leaves = sorted(g.leaves)
        pick = [leaves[k] for k in rng.choice(len(leaves), size=max(1, len(leaves) // 5), replace=False)]
        g.refine(pick)
    leaves = sorted(g.leaves)
    # exact integer geometry at the finest level
    box = {}
    for (L, i, j) in leaves:
        s = 3 ** (prm.l_max - L)
        box[(L, i, j)] = (i * s, (i + 1) * s, j * s, (j + 1) * s)
    brute = set()
    for a in range(len(leaves)):
        x0, x1, y0, y1 = box[leaves[a]]
        for b in range(a + 1, len(leaves)):
            u0, u1, v0, v1 = box[leaves[b]]
            share_x = (x1 == u0 or u1 == x0) and min(y1, v1) > max(y0, v0)
            share_y = (y1 == v0 or v1 == y0) and min(x1, u1) > max(x0, u0)
            if share_x or share_y:
                brute.add(tuple(sorted([leaves[a], leaves[b]])))
    assert g.adjacent_pairs() == brute
    # the leaves tile the grid
    area = sum((box[c][1] - box[c][0]) * (box[c][3] - box[c][2]) for c in leaves)
    assert area == (prm.n * 3 ** prm.l_max) ** 2


# ------------------------------------------------------------ the images

CASES = [(0.5, 0.1), (1.5, 0.1), (0.1, 0.9), (1.9, 0.05)]


@pytest.fixture(scope="module")
def found():
    prm = sis_params()
    res = I.find_images(alpha_sis, [(b, 0.0, R) for b, R in CASES], prm, with_cells=True)
    return prm, res


def test_images_against_appendix_b(found):
    prm, res = found
    for (b, R), r in zip(CASES, res):
        mp, mm, ring = I.sis_finite_source_mu(b, R)
        exp = [mp + mm] if ring else ([mp, mm] if mm > 0 else [mp])
        got = sorted((im["mu"] for im in r["images"]), reverse=True)
        assert len(got) == len(exp), (b, R, got)
        for a, e in zip(got, exp):
            assert abs(a / e - 1.0) < 7e-3, (b, R, a, e)


def test_images_are_maximal_components_and_criteria_hold(found):
    prm, res = found
    for (b, R), r in zip(CASES, res):
        g = I._Grid.__new__(I._Grid)
        g.prm = prm
        leaves = r["leaf_set"]
        # every leaf has its own ray: N^2 initial plus 8 per refinement
        assert (len(leaves) - prm.n ** 2) % 8 == 0
        assert r["rays"] == len(leaves)
        # the leaves tile the grid
        tot = sum(I.cell_size(prm, L) ** 2 for (L, _, _) in leaves)
        assert tot == pytest.approx(prm.side ** 2, rel=1e-12)
        # images: disjoint, connected, maximal, their cells inside the source
        g.leaves = {c: None for c in leaves}
        pairs = g.adjacent_pairs()
        where = {}
        for k, comp in enumerate(r["image_cells"]):
            for c in comp:
                assert c not in where
                where[c] = k
        for a, c in pairs:
            if a in where and c in where:
                assert where[a] == where[c]
        # stopping rule (I6) at the end
        for k, comp in enumerate(r["image_cells"]):
            inner = {a if a in where else c for a, c in pairs
                     if (a in where) != (c in where) and where.get(a, where.get(c)) == k}
            outer = {c if a in where else a for a, c in pairs
                     if (a in where) != (c in where) and where.get(a, where.get(c)) == k}
            area = sum(I.cell_size(prm, L) ** 2 for (L, _, _) in comp)
            lb = min(c[0] for c in inner | outer)
            assert (I.cell_size(prm, lb) ** 2 < prm.f_area * area
                    and min(c[0] for c in outer) >= min(c[0] for c in inner)) or lb >= prm.l_max
            assert len(comp) >= prm.n_min


def test_telescoping_finds_the_faint_image():
    """b = 0.95, R = 0.1: the negative image has mu = 0.058; with mu_min =
    0.01 the telescoping finds it (the coarse grid alone does not: no cell of
    the 64 x 64 grid maps into the source there)."""
    prm = sis_params(mu_min=0.01)
    r = I.find_images(alpha_sis, [(0.95, 0.0, 0.1)], prm)[0]
    mus = sorted(im["mu"] for im in r["images"])
    mp, mm, _ = I.sis_finite_source_mu(0.95, 0.1)
    assert len(mus) == 2 and abs(mus[0] / mm - 1) < 7e-3 and abs(mus[1] / mp - 1) < 7e-3
    g = I._Grid(prm, alpha_sis)
    assert not any(c for c in g.inside((0.95, 0.0), 0.1) if I.cell_centre(prm, *c)[0] < 0)


@pytest.mark.parametrize("n_min", [1000, 3000])
def test_uniform_step_brings_every_image_to_n_min(n_min):
    """I5 on its own: with a coarse telescoping (mu_min = 1) and a loose border
    rule (f_area = 0.5) the images keep a few hundred cells, so every image
    reaches n_min cells only through the uniform step; without it (n_min = 0)
    they stay below."""
    cases = [(0.5, 0.0, 0.1), (1.5, 0.0, 0.1)]
    loose = dict(f_area=0.5, l_max=10, mu_min=1.0)
    with_u = I.find_images(alpha_sis, cases, sis_params(n_min=n_min, **loose))
    without = I.find_images(alpha_sis, cases, sis_params(n_min=0, **loose))
    for a, b in zip(with_u, without):
        assert len(a["images"]) == len(b["images"]) > 0
        assert all(im["n_cells"] >= n_min for im in a["images"])
        assert max(im["n_cells"] for im in b["images"]) < n_min
