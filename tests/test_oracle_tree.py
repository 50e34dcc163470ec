"""Pins of the oracle's paper tree (Sec. 3.2 algorithm; Sec. 5.1 tests).

- theta_force = 0 reproduces the direct sum (Sec. 5.1).
- For halos, kappa is exact at any theta (Sec. 5.1 halo test): only halos
  whose support covers the ray carry surface density, and the big-particle
  lists make sure they are all evaluated in full.
- The error falls as theta falls, gamma converges at least as fast as alpha,
  and theta = 0.1 meets the 1e-4 median-alpha tolerance (Sec. 5.1 conclusion).
"""
import numpy as np
import pytest

import lensgen
import oracle
from oracle import GAUSS, NFW, POINT


def rel_err(a, ref, cols):
    d = np.linalg.norm(a[:, cols] - ref[:, cols], axis=1)
    r = np.linalg.norm(ref[:, cols], axis=1)
    return d / np.maximum(r, 1e-3 * np.median(r))


def point_set(n, seed):
    p = lensgen.point_disk(n, seed, total_mass=float(n)).astype(np.float64)
    return oracle.make_components(POINT, p[:, 0], p[:, 1], p[:, 2])


def halo_set(n, seed, size_max):
    h = lensgen.nfw_test_halos(n, seed, size_max).astype(np.float64)
    return oracle.make_components(NFW, h[:, 0], h[:, 1], h[:, 2], h[:, 3], 3.0 * h[:, 3])


def test_theta_zero_is_direct_sum():
    c = halo_set(300, 1, 0.3)
    g = np.random.default_rng(2)
    rx, ry = g.uniform(-1, 1, 64), g.uniform(-1, 1, 64)
    t = oracle.PaperTree(c, 5, 0.0)
    out, cnt = t.eval(rx, ry)
    ref = oracle.direct_sum(c, rx, ry)
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    assert np.all(cnt[:, 0] == 0)                          # no cell accepted
    assert np.all(cnt[:, 1] + cnt[:, 2] == len(c))         # every particle once


@pytest.mark.parametrize("theta", [0.1, 0.3, 0.55, 0.8, 1.0])
def test_halo_kappa_exact_at_any_theta(theta):
    c = halo_set(1000, 3, 0.3)
    g = np.random.default_rng(4)
    rx, ry = g.uniform(-1, 1, 200), g.uniform(-1, 1, 200)
    out, _ = oracle.PaperTree(c, 5, theta).eval(rx, ry)
    ref = oracle.direct_sum(c, rx, ry)
    np.testing.assert_allclose(out[:, 2], ref[:, 2], rtol=1e-12, atol=1e-13)


def test_gaussian_kappa_exact_and_listed_particles_counted_once():
    p = lensgen.nfw_particles(3000, 5, nsph=16)
    c = oracle.make_components(GAUSS, p[:, 0], p[:, 1], p[:, 2], p[:, 3], 3.0)
    g = np.random.default_rng(6)
    rx, ry = g.uniform(-0.6, 0.6, 200), g.uniform(-0.6, 0.6, 200)
    ref = oracle.direct_sum(c, rx, ry)
    out, cnt = oracle.PaperTree(c, 5, 0.3).eval(rx, ry)
    np.testing.assert_allclose(out[:, 2], ref[:, 2], rtol=1e-11, atol=1e-11 * np.abs(ref[:, 2]).max())
    assert cnt[:, 3].sum() > 0        # big-list corrections happened


def test_error_falls_with_theta_and_gamma_converges_faster():
    """Sec. 5.1 point-mass test: 1e4 unit masses in the unit circle, the ray
    through the centre, many realizations; median fractional errors."""
    thetas = [0.1, 0.3, 0.6, 1.0]
    ea, eg = [], []
    for seed in range(24):
        c = point_set(10000, 100 + seed)
        ref = oracle.direct_sum(c, [0.0], [0.0])
        ra, rg = [], []
        for th in thetas:
            out, _ = oracle.PaperTree(c, 5, th).eval([0.0], [0.0])
            ra.append(np.linalg.norm(out[0, :2] - ref[0, :2]) / np.linalg.norm(ref[0, :2]))
            rg.append(np.linalg.norm(out[0, 3:] - ref[0, 3:]) / np.linalg.norm(ref[0, 3:]))
        ea.append(ra)
        eg.append(rg)
    ma, mg = np.median(ea, axis=0), np.median(eg, axis=0)
    assert np.all(np.diff(ma) > 0) and np.all(np.diff(mg) > 0)
    assert ma[0] <= 1e-4                      # theta = 0.1 is sufficient
    assert np.all(mg <= ma)                   # gamma converges faster


def test_counts_account_for_every_particle_once_when_opening_everything():
    c = point_set(500, 30)
    out, cnt = oracle.PaperTree(c, 1, 0.0).eval([0.2], [0.1])
    assert cnt[0, 1] == 500 and cnt[0, 0] == 0
