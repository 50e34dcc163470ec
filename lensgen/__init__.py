"""Seeded synthetic inputs for the ray-shooting workloads.

This module holds no lensing arithmetic: it draws particle positions, masses
and sizes and lays out ray positions.  Both the oracle side (tests, golden
scripts) and the CUDA side (tests, bench) take their inputs from here.  Every
generator uses numpy's PCG64 with an explicit seed and rounds particle data to
float32 (the values both sides then see exactly), except where FP64 is asked.

Workloads (sizes are parameters so tests can shrink them):
  point_disk      equal point masses uniform in the unit disk        (Sec. 5.1 tests)
  nfw_particles   3D NFW samples projected, smoothing = distance to the
                  k-th nearest neighbour in 3D                       (Sec. 3.1)
  nfw_halo_field  NFW halos with log-normal masses                   (Sec. 5.1 halo tests)
  salpeter_stars  stars with dN/dm ~ m^-2.35 on [0.1, 1]             (Sec. 3.5)
  grid_rays       cell-centred ray grids, row-major, x fastest
  refinement_batches  uneven jittered-grid batches from refinement levels (Sec. 4)
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def f32(a) -> np.ndarray:
    """Round to float32 and return as float32."""
    return np.asarray(a, dtype=np.float64).astype(np.float32)


# ---------------------------------------------------------------- particles

def uniform_disk(g: np.random.Generator, n: int, radius: float = 1.0,
                 center=(0.0, 0.0)):
    """n points uniform in a disk (r = R sqrt(U), phi = 2 pi U)."""
    r = radius * np.sqrt(g.random(n))
    phi = 2.0 * np.pi * g.random(n)
    return center[0] + r * np.cos(phi), center[1] + r * np.sin(phi)


def salpeter_masses(g: np.random.Generator, n: int, mmin=0.1, mmax=1.0, slope=2.35):
    """Inverse-CDF draw from dN/dm ~ m^-slope on [mmin, mmax]."""
    a = 1.0 - slope
    lo, hi = mmin ** a, mmax ** a
    return (lo + g.random(n) * (hi - lo)) ** (1.0 / a)


def _nfw_cdf(x):
    # enclosed 3D NFW mass shape, used only to draw radii
    return np.log1p(x) - x / (1.0 + x)


def nfw_radii(g: np.random.Generator, n: int, rs: float, rmax: float):
    """Radii drawn from a 3D NFW density rho ~ 1/[(r/rs)(1+r/rs)^2], r < rmax,
    by bisection on the inverse CDF (60 halvings, float64)."""
    X = rmax / rs
    target = g.random(n) * _nfw_cdf(X)
    lo = np.zeros(n)
    hi = np.full(n, X)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        below = _nfw_cdf(mid) < target
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi) * rs


def isotropic(g: np.random.Generator, r):
    """3D positions with radii r and isotropic directions."""
    n = r.shape[0]
    mu = 2.0 * g.random(n) - 1.0
    phi = 2.0 * np.pi * g.random(n)
    s = np.sqrt(1.0 - mu * mu)
    return r * s * np.cos(phi), r * s * np.sin(phi), r * mu


def knn_distance(x, y, z, k: int, workers: int = -1):
    """Distance from every point to its k-th nearest neighbour in 3D (itself
    excluded), via scipy's cKDTree (a library neighbour search)."""
    from scipy.spatial import cKDTree
    pts = np.stack([x, y, z], axis=1)
    tree = cKDTree(pts)
    d, _ = tree.query(pts, k=k + 1, workers=workers)
    return d[:, k]


def point_disk(n: int, seed: int, total_mass: float = 1.0):
    """n equal point masses uniform in the unit disk: float32 (n, 4) {x,y,m,0}."""
    g = rng(seed)
    x, y = uniform_disk(g, n)
    p = np.zeros((n, 4), dtype=np.float32)
    p[:, 0], p[:, 1], p[:, 2] = f32(x), f32(y), f32(np.full(n, total_mass / n))
    return p


def nfw_particles(n: int, seed: int, rs: float = 0.1, rmax: float = 1.0,
                  total_mass: float = 1.0, nsph: int | None = 32,
                  fixed_sigma: float | None = None):
    """Equal-mass particles of a 3D NFW halo, projected on (x, y).
    Smoothing r_sm = distance to the nsph-th 3D neighbour, or fixed_sigma.
    Returns float32 (n, 4) {x, y, m, r_sm}."""
    g = rng(seed)
    r = nfw_radii(g, n, rs, rmax)
    x, y, z = isotropic(g, r)
    if fixed_sigma is not None:
        sig = np.full(n, fixed_sigma)
    else:
        sig = knn_distance(x, y, z, nsph)
    p = np.zeros((n, 4), dtype=np.float32)
    p[:, 0], p[:, 1] = f32(x), f32(y)
    p[:, 2] = f32(np.full(n, total_mass / n))
    p[:, 3] = f32(sig)
    return p


def nfw_positions_3d(n: int, seed: int, rs: float = 0.1, rmax: float = 1.0):
    """The 3D positions nfw_particles(n, seed) projects (same draws), as
    float32 (n, 3) {x, y, z}: the input of the smoothing-length search."""
    g = rng(seed)
    r = nfw_radii(g, n, rs, rmax)
    x, y, z = isotropic(g, r)
    return np.stack([f32(x), f32(y), f32(z)], axis=1)


def nfw_halo_field(n: int, seed: int, log10_m_mean: float = -4.0, log10_m_sigma: float = 1.0,
                   rs_at_1e4: float = 0.02, box: float = 1.0, g=None):
    """NFW halos: log10 m ~ N(mean, sigma); positions uniform in [-box, box]^2;
    r_s = rs_at_1e4 (m / 1e-4)^(1/3).  float32 (n, 4) {x, y, m, r_s}."""
    g = rng(seed) if g is None else g
    m = 10.0 ** (log10_m_mean + log10_m_sigma * g.standard_normal(n))
    x = box * (2.0 * g.random(n) - 1.0)
    y = box * (2.0 * g.random(n) - 1.0)
    rs = rs_at_1e4 * (m / 1e-4) ** (1.0 / 3.0)
    p = np.zeros((n, 4), dtype=np.float32)
    p[:, 0], p[:, 1], p[:, 2], p[:, 3] = f32(x), f32(y), f32(m), f32(rs)
    return p


def nfw_test_halos(n: int, seed: int, size_max: float, conc: float = 3.0):
    """Halo test of Sec. 5.1: unit circle, sizes uniform up to size_max,
    dn/dm ~ m^-2 on [1e-3, 1], concentration conc.  Returns float32 (n, 4)
    {x, y, m, r_s} with R_max = conc * r_s = size."""
    g = rng(seed)
    x, y = uniform_disk(g, n)
    u = g.random(n)
    m = 1.0 / (1.0 / 1e-3 - u * (1.0 / 1e-3 - 1.0))   # inverse CDF of m^-2
    size = size_max * g.random(n)
    p = np.zeros((n, 4), dtype=np.float32)
    p[:, 0], p[:, 1], p[:, 2], p[:, 3] = f32(x), f32(y), f32(m), f32(size / conc)
    return p


def salpeter_stars_square(n: int, g, x0, x1, y0, y1, total_mass: float):
    m = salpeter_masses(g, n)
    m *= total_mass / m.sum()
    x = x0 + (x1 - x0) * g.random(n)
    y = y0 + (y1 - y0) * g.random(n)
    p = np.zeros((n, 4), dtype=np.float32)
    p[:, 0], p[:, 1], p[:, 2] = f32(x), f32(y), f32(m)
    return p


def salpeter_stars_disk(n: int, g, radius: float, total_mass: float):
    m = salpeter_masses(g, n)
    m *= total_mass / m.sum()
    x, y = uniform_disk(g, n, radius)
    p = np.zeros((n, 4), dtype=np.float32)
    p[:, 0], p[:, 1], p[:, 2] = f32(x), f32(y), f32(m)
    return p


# --------------------------------------------------------------------- rays

def grid_rays(n: int, lo: float, hi: float, dtype=np.float64):
    """n x n cell-centred grid over [lo, hi]^2, row-major with x fastest."""
    c = lo + (np.arange(n) + 0.5) * (hi - lo) / n
    X, Y = np.meshgrid(c, c)
    return X.reshape(-1).astype(dtype), Y.reshape(-1).astype(dtype)


def patch_offsets(n: int, width: float):
    """n x n cell-centred offsets over a square of the given width centred on
    0, as float32 (added in FP64 to an FP64 origin)."""
    c = (np.arange(n) + 0.5) * width / n - 0.5 * width
    X, Y = np.meshgrid(c, c)
    return f32(X.reshape(-1)), f32(Y.reshape(-1))


def refinement_batches(g, n_batches: int, nmin: float, nmax: float, center_box,
                       side0: float, levels: int = 9):
    """Ray batches as refinement emits them: sizes log-uniform in [nmin, nmax];
    batch centres uniform in center_box = (x0, x1, y0, y1); side side0 * 3^-l
    with l uniform in {0..levels-1} (each refinement divides a cell by 3,
    Sec. 4); ceil(sqrt(n_b))^2 jittered grid truncated to n_b.
    Returns (offsets int64 (B+1), origins float64 (B, 2), dx, dy float32)."""
    sizes = np.round(10.0 ** (math.log10(nmin) + g.random(n_batches) *
                              (math.log10(nmax) - math.log10(nmin)))).astype(np.int64)
    x0, x1, y0, y1 = center_box
    origins = np.stack([x0 + (x1 - x0) * g.random(n_batches),
                        y0 + (y1 - y0) * g.random(n_batches)], axis=1)
    lev = g.integers(0, levels, n_batches)
    offsets = np.zeros(n_batches + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    dx = np.empty(offsets[-1], dtype=np.float32)
    dy = np.empty(offsets[-1], dtype=np.float32)
    for b in range(n_batches):
        nb = int(sizes[b])
        k = int(math.ceil(math.sqrt(nb)))
        side = side0 * 3.0 ** (-int(lev[b]))
        h = side / k
        i = np.arange(nb)
        cx = (i % k + 0.5 + (g.random(nb) - 0.5)) * h - 0.5 * side
        cy = (i // k + 0.5 + (g.random(nb) - 0.5)) * h - 0.5 * side
        dx[offsets[b]:offsets[b + 1]] = f32(cx)
        dy[offsets[b]:offsets[b + 1]] = f32(cy)
    return offsets, origins, dx, dy


def sample_indices(g, n_total: int, k: int):
    return np.sort(g.choice(n_total, size=min(k, n_total), replace=False))


# ------------------------------------------------------------- the workloads

def workload_point_disk(n_part=2000, n_grid=64, seed=1):
    """Equal point masses (m = 1/n) in the unit disk; FP64 grid on [-1.2, 1.2]^2."""
    parts = point_disk(n_part, seed).astype(np.float64)
    rx, ry = grid_rays(n_grid, -1.2, 1.2)
    return dict(points=parts, rx=rx, ry=ry)


def workload_nfw_sph(n_part=1_000_000, n_grid=2048, seed=2, nsph=32, q=3.0):
    """Smoothed NFW particles (r_s = 0.1, r < 1, total mass 1), r_sm = 32nd
    3D neighbour distance, q = 3; rays on an n_grid^2 grid over [-1, 1]^2."""
    parts = nfw_particles(n_part, seed, nsph=nsph)
    rx, ry = grid_rays(n_grid, -1.0, 1.0, dtype=np.float32)
    return dict(gauss=parts, q=q, rx=rx, ry=ry)


def workload_refine(n_halos=1000, n_grid=2048, seed=3, conc=3.0, centre=(0.3, 0.2), width=0.03):
    """The batched workload's NFW halo field (same seed, so the same halos)
    and an n_grid^2 cell-centred grid of rays over a width-wide square at
    `centre` (an FP64 origin plus FP64 offsets, so ray (i, j) sits exactly at
    x0 + i h, y0 + j h): the input of the cell-refinement workload."""
    halos = nfw_halo_field(n_halos, seed, g=rng(seed))
    h = width / n_grid
    c = (np.arange(n_grid) + 0.5) * h - 0.5 * width
    X, Y = np.meshgrid(c, c)
    return dict(nfw=halos, conc=conc, origin=np.array(centre, np.float64), dx=X.reshape(-1), dy=Y.reshape(-1),
                n_grid=n_grid, h=h, x0=centre[0] + c[0], y0=centre[1] + c[0])


def workload_mixed_batches(n_halos=1000, n_stars=1_000_000, n_batches=256, nmin=1e3,
                           nmax=1e6, seed=3, kappa_star=0.5):
    """NFW halo field plus Salpeter stars in a 0.01-wide patch at (0.3, 0.2);
    uneven refinement batches centred in the star patch."""
    g = rng(seed)
    halos = nfw_halo_field(n_halos, seed, g=g)
    area = 0.01 * 0.01
    stars = salpeter_stars_square(n_stars, g, 0.295, 0.305, 0.195, 0.205,
                                  kappa_star * area / math.pi)
    offsets, origins, dx, dy = refinement_batches(
        g, n_batches, nmin, nmax, (0.295, 0.305, 0.195, 0.205), 0.01)
    return dict(nfw=halos, conc=3.0, points=stars, offsets=offsets, origins=origins,
                dx=dx, dy=dy)


def workload_fit(n_part=100_000, n_grid=1000, seed=4, sigma=0.01, q=3.0, noise=0.05):
    """Gaussian particles of fixed width from the NFW sampler (total mass 1);
    target masses m exp(noise N(0,1)); grid on [-1, 1]^2."""
    parts = nfw_particles(n_part, seed, fixed_sigma=sigma)
    g = rng(seed + 1000)
    target = parts.copy()
    target[:, 2] = f32(parts[:, 2].astype(np.float64) * np.exp(noise * g.standard_normal(n_part)))
    rx, ry = grid_rays(n_grid, -1.0, 1.0, dtype=np.float32)
    return dict(gauss=parts, target=target, q=q, rx=rx, ry=ry)


def workload_microlensing(n_stars=10_000_000, n_grid=4096, seed=5, r_e=0.5,
                          width=1e-6, center=(0.5, 0.0), kappa_star=0.5):
    """Salpeter stars uniform in the unit disk (kappa_* = 0.5, i.e. total
    m = 0.5) plus an SIS of Einstein radius 0.5 at the origin; rays on an
    n_grid^2 patch of the given width at `center` (FP64 origin, FP32 offsets)."""
    g = rng(seed)
    stars = salpeter_stars_disk(n_stars, g, 1.0, kappa_star * 1.0)
    dx, dy = patch_offsets(n_grid, width)
    return dict(points=stars, sis_re=r_e, origin=center, dx=dx, dy=dy)
