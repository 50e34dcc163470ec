"""Pins of the oracle's single-component lensing quantities.

Each check ties the oracle to something other than its own formula:
quadrature of the paper's surface densities (Sec. 3.1 Eq. smoothing; the 3D
NFW density projected numerically), the SIS results of App. B (golden file),
the point-mass lens equation, and the definitions of kappa and gamma as
derivatives of alpha (Eqs. kappa, gamma_1, gamma_2) by finite differences.
"""
import json
import math
import os

import mpmath
import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import DISK, GAUSS, NFW, POINT, SIS

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def comp(t, x=0.0, y=0.0, m=1.0, p0=0.0, p1=0.0):
    return oracle.make_components(t, x, y, m, p0, p1)[0]


def enclosed_from_alpha(c, r, phi=0.3):
    a = oracle.eval_component(c, c["x"] + r * math.cos(phi), c["y"] + r * math.sin(phi))
    return math.hypot(a[0], a[1]) * r, a


# ------------------------------------------------------------------ Gaussian

@pytest.mark.parametrize("sig,q", [(0.05, 3.0), (1.3, 2.0), (0.01, 4.0)])
def test_gauss_enclosed_mass_matches_quadrature_of_surface_density(sig, q):
    """Sec. 3.1 Eq. smoothing gives Sigma; |alpha| r must equal int 2 pi r Sigma."""
    m = 0.7
    c = comp(GAUSS, 0.1, -0.2, m, sig, q)
    Nq = 1.0 - math.exp(-q * q / 2)

    def sigma_m(r):  # m-unit surface density, Eq. smoothing
        return m / (2 * math.pi * sig ** 2) * math.exp(-r * r / (2 * sig ** 2)) / Nq if r < q * sig else 0.0

    for frac in [1e-3, 0.2, 0.7, 1.0, 1.9, 2.9999, 3.5]:
        r = frac * sig
        M_quad, _ = integrate.quad(lambda s: 2 * math.pi * s * sigma_m(s), 0, min(r, q * sig),
                                   epsabs=0, epsrel=1e-13, limit=200)
        M_or, a = enclosed_from_alpha(c, r)
        assert M_or == pytest.approx(M_quad, rel=1e-10, abs=1e-300)
        # kappa = Sigma / Sigma_crit = pi * Sigma_m (m-units)
        assert a[2] == pytest.approx(math.pi * sigma_m(r), rel=1e-12, abs=1e-300)


def test_gauss_edge_is_outside_and_alpha_continuous():
    """C10 reading: at |x| = q r_sm exactly the particle counts as outside."""
    sig, q = 0.25, 3.0
    c = comp(GAUSS, 0.0, 0.0, 1.0, sig, q)
    a = oracle.eval_component(c, q * sig, 0.0)
    assert a[2] == 0.0
    ai = oracle.eval_component(c, q * sig * (1 - 1e-12), 0.0)
    assert ai[0] == pytest.approx(a[0], rel=1e-10)
    assert ai[2] > 0


def test_gauss_centre():
    sig, q, m = 0.2, 3.0, 2.0
    c = comp(GAUSS, 0.3, 0.4, m, sig, q)
    a = oracle.eval_component(c, 0.3, 0.4)
    assert a[0] == 0 and a[1] == 0 and a[3] == 0 and a[4] == 0
    assert a[2] == pytest.approx(math.pi * m / (2 * math.pi * sig ** 2) / (1 - math.exp(-q * q / 2)))


# ----------------------------------------------------------------------- NFW

def nfw_sigma_los(R, rs):
    """Projected 3D NFW density rho = 1/[(r/rs)(1+r/rs)^2] by quadrature along z."""
    f = lambda z: 1.0 / ((math.hypot(R, z) / rs) * (1 + math.hypot(R, z) / rs) ** 2)
    v1, _ = integrate.quad(f, 0, 10 * rs + 10 * R, epsabs=0, epsrel=1e-12, limit=400)
    v2, _ = integrate.quad(f, 10 * rs + 10 * R, np.inf, epsabs=0, epsrel=1e-12, limit=400)
    return 2 * (v1 + v2)


def nfw_mass2d(R, rs):
    v, _ = integrate.quad(lambda s: 2 * math.pi * s * nfw_sigma_los(s, rs), 0, R,
                          epsabs=0, epsrel=1e-10, limit=200, points=[rs] if rs < R else None)
    return v


@pytest.mark.parametrize("rs,Rmax", [(0.1, 0.3), (0.05, 0.5)])
def test_nfw_matches_projected_3d_density(rs, Rmax):
    """Sec. 3.2 analytic halo, read as the projected NFW truncated in 2D at
    R_max with total mass m: enclosed mass and kappa from LOS quadrature."""
    m = 0.37
    c = comp(NFW, 0.0, 0.0, m, rs, Rmax)
    Mtot = nfw_mass2d(Rmax, rs)
    for r in [0.003 * rs, 0.4 * rs, 0.999 * rs, rs * 1.0001, 2.2 * rs, 0.98 * Rmax]:
        M_or, a = enclosed_from_alpha(c, r)
        assert M_or == pytest.approx(m * nfw_mass2d(r, rs) / Mtot, rel=2e-8)
        kap = math.pi * m * nfw_sigma_los(r, rs) / Mtot
        assert a[2] == pytest.approx(kap, rel=2e-8)
    # outside R_max: a point mass of mass m
    M_or, a = enclosed_from_alpha(c, 1.5 * Rmax)
    assert M_or == pytest.approx(m, rel=1e-14) and a[2] == 0.0


def _g_mp(x):
    x = mpmath.mpf(x)
    if x < 1:
        return mpmath.log(x / 2) + mpmath.acosh(1 / x) / mpmath.sqrt(1 - x * x)
    if x > 1:
        return mpmath.log(x / 2) + mpmath.acos(1 / x) / mpmath.sqrt(x * x - 1)
    return mpmath.log(mpmath.mpf(1) / 2) + 1


@pytest.mark.parametrize("x", [1e-7, 1e-5, 3e-3, 0.0099, 0.0101, 0.5, 0.9999, 1.0, 1.00007, 1.3, 7.0])
def test_nfw_enclosed_mass_series_regions_vs_high_precision(x):
    """The small-x expansion and the near-1 series against 50-digit mpmath."""
    mpmath.mp.dps = 50
    rs, X, m = 1.0, 20.0, 1.0
    c = comp(NFW, 0.0, 0.0, m, rs, X * rs)
    M_or, _ = enclosed_from_alpha(c, x * rs, phi=0.0)
    ref = float(_g_mp(x) / _g_mp(X))
    assert M_or == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("x", [0.9, 0.95, 0.97, 0.999, 0.99963, 0.9999, 1.0, 1.0003, 1.001, 1.02, 1.05, 1.1])
def test_nfw_convergence_near_x1_vs_high_precision(x):
    """kappa = m f(x) / (2 r_s^2 g(X)), f = (1 - F)/(x^2 - 1), near x = 1,
    where the closed forms cancel (arccosh(1/x) is ill-conditioned there):
    against 50-digit mpmath at 1e-14."""
    mpmath.mp.dps = 50
    rs, X, m = 1.0, 20.0, 1.0
    c = comp(NFW, 0.0, 0.0, m, rs, X * rs)
    kap = oracle.eval_component(c, x * rs, 0.0)[2]
    xm = mpmath.mpf(x)
    if x < 1:
        F = mpmath.acosh(1 / xm) / mpmath.sqrt(1 - xm * xm)
    elif x > 1:
        F = mpmath.acos(1 / xm) / mpmath.sqrt(xm * xm - 1)
    else:
        F = mpmath.mpf(1)
    f = (1 - F) / (xm * xm - 1) if x != 1.0 else mpmath.mpf(1) / 3
    ref = float(m * f / (2 * rs * rs * _g_mp(X)))
    assert kap == pytest.approx(ref, rel=1e-14)


# ----------------------------------------------------------------------- SIS

def test_sis_appendix_b_images_and_magnifications():
    """App. B: both images map back to the source; mu from kappa, gamma."""
    with open(os.path.join(GOLDEN, "sis_appendix_b.json")) as f:
        cases = json.load(f)["cases"]
    for cs in cases:
        c = comp(SIS, 0.0, 0.0, 0.0, cs["r_e"])
        for key, mukey in [("x_plus", "mu_plus"), ("x_minus", "mu_minus")]:
            x = np.array(cs[key])
            a = oracle.eval_component(c, x[0], x[1])
            y = x - a[:2]                                     # Eq. lens_eq
            np.testing.assert_allclose(y, cs["y"], rtol=0, atol=1e-14)
            kap, g1, g2 = a[2], a[3], a[4]
            mu = 1.0 / ((1 - kap) ** 2 - (g1 * g1 + g2 * g2))  # Sec. 3.2 magnification
            assert mu == pytest.approx(cs[mukey], rel=1e-12)


# ----------------------------------------------------------------- point mass

def test_point_mass_lens_equation_images_and_einstein_ring():
    """Point lens: two images at r = (|y| +- sqrt(|y|^2 + 4 m))/2 along y;
    the ring r_E = sqrt(m) maps to the origin (Sec. 3.5 defines r_E)."""
    m = 0.3
    c = comp(POINT, 0.1, 0.2, m)
    ring = math.sqrt(m)
    a = oracle.eval_component(c, 0.1 + ring * 0.6, 0.2 + ring * 0.8)
    assert math.hypot(a[0], a[1]) == pytest.approx(ring, rel=1e-15)
    y = np.array([0.05, -0.12])
    b = np.linalg.norm(y)
    for sgn in (+1, -1):
        r = 0.5 * (b + sgn * math.sqrt(b * b + 4 * m))
        x = y / b * r
        a = oracle.eval_component(c, 0.1 + x[0], 0.2 + x[1])
        np.testing.assert_allclose(x - a[:2], y, atol=1e-14)
        assert a[2] == 0.0


def test_point_mass_on_top_is_skipped():
    c = comp(POINT, 0.5, 0.5, 1.0)
    assert np.all(oracle.eval_component(c, 0.5, 0.5) == 0)


# ---------------------------------------------------------------- uniform disk

def test_disk_gauss_law_and_negative_sheet():
    R, m = 0.4, -0.25
    c = comp(DISK, 0.2, 0.0, m, R)
    for r in [0.01, 0.2, 0.3999, 0.41, 2.0]:
        M_or, a = enclosed_from_alpha(c, r)
        a_vec = a[:2]
        M_expect = m * min(r, R) ** 2 / R ** 2   # uniform Sigma_m = m / (pi R^2)
        # signed enclosed mass: alpha points toward the centre for m < 0
        sgn = math.copysign(1.0, a_vec[0] * math.cos(0.3) + a_vec[1] * math.sin(0.3))
        assert sgn * M_or == pytest.approx(M_expect, rel=1e-13)


# --------------------------------------------- derivatives: kappa and gamma

def fd_jacobian(c, x, y, h):
    """4th-order central differences of alpha."""
    def a(px, py):
        return oracle.eval_component(c, px, py)[:2]
    d1 = (-a(x + 2 * h, y) + 8 * a(x + h, y) - 8 * a(x - h, y) + a(x - 2 * h, y)) / (12 * h)
    d2 = (-a(x, y + 2 * h) + 8 * a(x, y + h) - 8 * a(x, y - h) + a(x, y - 2 * h)) / (12 * h)
    return d1, d2  # d/dx1 (a1, a2), d/dx2 (a1, a2)


CASES = [
    (GAUSS, 0.5, 0.1, 3.0, [0.02, 0.13, 0.29, 0.5]),
    (NFW, 0.05, 0.4, 0.0, [0.001, 0.04, 0.051, 0.2, 0.39, 0.6]),
    (SIS, 0.3, 0.0, 0.0, [0.05, 0.3, 1.7]),
    (DISK, 0.3, 0.0, 0.0, [0.1, 0.29, 0.31, 0.9]),
    (POINT, 0.0, 0.0, 0.0, [0.05, 0.4]),
]


@pytest.mark.parametrize("t,p0,p1,_,radii", CASES)
def test_kappa_gamma_are_derivatives_of_alpha(t, p0, p1, _, radii):
    """Eqs. kappa, gamma_1, gamma_2: kappa = tr/2, gamma1 = (d1a1 - d2a2)/2,
    gamma2 = d1a2 = d2a1 (curl free), by finite differences of alpha."""
    if t == GAUSS:
        c = comp(t, 0.1, 0.2, 1.3, 0.1, 3.0)  # support 0.3
    else:
        c = comp(t, 0.1, 0.2, 1.3, p0, p1)
    for r in radii:
        for phi in [0.1, 1.3, 2.9, 4.4]:
            x, y = 0.1 + r * math.cos(phi), 0.2 + r * math.sin(phi)
            h = min(r, 0.01) * 1e-3
            d1, d2 = fd_jacobian(c, x, y, h)
            v = oracle.eval_component(c, x, y)
            scale = np.max(np.abs(np.r_[d1, d2])) + 1e-300
            tol = 1e-7 * scale
            assert v[2] == pytest.approx(0.5 * (d1[0] + d2[1]), abs=tol)
            assert v[3] == pytest.approx(0.5 * (d1[0] - d2[1]), abs=tol)
            assert v[4] == pytest.approx(d1[1], abs=tol)
            assert d1[1] == pytest.approx(d2[0], abs=tol)
