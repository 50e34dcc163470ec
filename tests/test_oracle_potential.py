"""Pins of the oracle's lensing potential (Eq. alpha: alpha = grad psi; the
Poisson equation: div grad psi = 2 kappa; Eq. timedelay) for every component
type, against the (separately pinned) deflection and convergence:

* 4th-order central differences of psi equal alpha;
* the 5-point Laplacian of psi equals 2 kappa inside the supports;
* psi(r_b) - psi(r_a) equals the quadrature of the radial alpha from r_a to r_b
  (checks the special functions Ein and the NFW shape H independently);
* closed forms (point m ln r, SIS r_E r, uniform disk), continuity at the
  support edge, and the direct sum is the sum of the components.
"""
import numpy as np
import pytest
from scipy.integrate import quad

import oracle

CASES = [
    ("point", oracle.make_components(oracle.POINT, 0.1, -0.2, 0.7)),
    ("gauss", oracle.make_components(oracle.GAUSS, 0.1, -0.2, 0.7, 0.05, 3.0)),
    ("gauss_q5", oracle.make_components(oracle.GAUSS, 0.1, -0.2, 0.7, 0.05, 5.0)),
    ("nfw", oracle.make_components(oracle.NFW, 0.1, -0.2, 0.7, 0.04, 0.2)),
    ("sis", oracle.make_components(oracle.SIS, 0.1, -0.2, 0.0, 0.3)),
    ("disk", oracle.make_components(oracle.DISK, 0.1, -0.2, -0.4, 0.12)),
]
# distances from the centre: inside the supports (0.15 sigma .. 2.8 sigma,
# small and large x of the NFW) and outside
RADII = [0.0075, 0.02, 0.06, 0.11, 0.14, 0.19, 0.35]


def psi_at(c, x, y):
    return oracle.potential_component(c, x, y)


@pytest.mark.parametrize("name,c", CASES)
def test_gradient_of_psi_is_alpha(name, c):
    h = 1e-5
    for r in RADII:
        for phi in (0.3, 2.1, 4.0):
            x, y = c["x"][0] + r * np.cos(phi), c["y"][0] + r * np.sin(phi)
            gx = (-psi_at(c, x + 2 * h, y) + 8 * psi_at(c, x + h, y) - 8 * psi_at(c, x - h, y)
                  + psi_at(c, x - 2 * h, y)) / (12 * h)
            gy = (-psi_at(c, x, y + 2 * h) + 8 * psi_at(c, x, y + h) - 8 * psi_at(c, x, y - h)
                  + psi_at(c, x, y - 2 * h)) / (12 * h)
            a = oracle.eval_component(c, x, y)
            scale = np.hypot(a[0], a[1])
            assert abs(gx - a[0]) <= 1e-7 * scale + 1e-12, (name, r, gx, a[0])
            assert abs(gy - a[1]) <= 1e-7 * scale + 1e-12, (name, r, gy, a[1])


@pytest.mark.parametrize("name,c", CASES)
def test_laplacian_of_psi_is_twice_kappa(name, c):
    for r in RADII:
        h = 0.005 * r  # the stencil's error scales as (h/r)^2
        x, y = c["x"][0] + r * np.cos(1.1), c["y"][0] + r * np.sin(1.1)
        edge = {"gauss": 0.15, "gauss_q5": 0.25, "nfw": 0.2, "disk": 0.12}.get(name)
        if edge is not None and abs(r - edge) < 5 * h:
            continue
        lap = (psi_at(c, x + h, y) + psi_at(c, x - h, y) + psi_at(c, x, y + h) + psi_at(c, x, y - h)
               - 4 * psi_at(c, x, y)) / (h * h)
        k = oracle.eval_component(c, x, y)[2]
        a = oracle.eval_component(c, x, y)
        scale = abs(2 * k) + np.hypot(a[0], a[1]) / r  # the Laplacian's size near r
        assert abs(lap - 2 * k) <= 5e-5 * scale, (name, r, lap, 2 * k)


@pytest.mark.parametrize("name,c", CASES)
def test_radial_difference_is_the_integral_of_alpha(name, c):
    cx, cy = c["x"][0], c["y"][0]

    def amag(r):
        # the radial component along +x (signed: a disk may carry negative mass)
        return oracle.eval_component(c, cx + r, cy)[0]

    for ra, rb in [(0.004, 0.03), (0.03, 0.13), (0.09, 0.3), (0.001, 0.5)]:
        pts = [p for p in (0.05 * 3.0, 0.05 * 5.0, 0.2, 0.12) if ra < p < rb]
        ref, _ = quad(amag, ra, rb, points=pts or None, epsabs=1e-14, epsrel=1e-12, limit=200)
        got = psi_at(c, cx + rb, cy) - psi_at(c, cx + ra, cy)
        assert got == pytest.approx(ref, rel=1e-9, abs=1e-13), (name, ra, rb)


def test_closed_forms_continuity_and_sum():
    p = oracle.make_components(oracle.POINT, 0.0, 0.0, 0.3)
    assert psi_at(p, 0.6, 0.8) == pytest.approx(0.3 * np.log(1.0), abs=1e-15)
    assert psi_at(p, 2.0, 0.0) == pytest.approx(0.3 * np.log(2.0), rel=1e-15)
    s = oracle.make_components(oracle.SIS, 0.0, 0.0, 0.0, 0.4)
    assert psi_at(s, 0.3, 0.4) == pytest.approx(0.4 * 0.5, rel=1e-15)
    d = oracle.make_components(oracle.DISK, 0.0, 0.0, 2.0, 0.5)
    assert psi_at(d, 0.0, 0.0) == pytest.approx(2.0 * (np.log(0.5) - 0.5), rel=1e-15)
    for name, c in CASES:
        edge = {"gauss": 0.15, "gauss_q5": 0.25, "nfw": 0.2, "disk": 0.12}.get(name)
        if edge is None:
            continue
        lo = psi_at(c, c["x"][0] + edge * (1 - 1e-9), c["y"][0])
        hi = psi_at(c, c["x"][0] + edge * (1 + 1e-9), c["y"][0])
        assert lo == pytest.approx(hi, rel=1e-7), name
    comps = oracle.concat(*(c for _, c in CASES))
    g = np.random.default_rng(5)
    rx, ry = g.uniform(-0.5, 0.5, 50), g.uniform(-0.5, 0.5, 50)
    tot, ab = oracle.direct_potential(comps, rx, ry, with_absum=True)
    each = np.array([[psi_at(comps[j], x, y) for j in range(comps.size)] for x, y in zip(rx, ry)])
    np.testing.assert_allclose(tot, each.sum(axis=1), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(ab, np.abs(each).sum(axis=1), rtol=1e-13)


def arrival_time(comps, x, y, src):
    """Eq. timedelay on one plane: tau(x) = |x - y_s|^2 / 2 - psi(x)."""
    psi = oracle.direct_potential(comps, np.array([x]), np.array([y]))[0]
    return 0.5 * ((x - src[0]) ** 2 + (y - src[1]) ** 2) - psi


@pytest.mark.parametrize("b", [0.1, 0.35, 0.8])
def test_sis_time_delay_between_images(b):
    """SIS of Einstein radius r_E: images at x+- = b +- r_E along the source
    direction (App. B); the arrival-time difference is 2 r_E b, and both
    images are stationary points of tau (the lens equation)."""
    rE = 0.7
    sis = oracle.make_components(oracle.SIS, 0.0, 0.0, 0.0, rE)
    src = (b * rE * np.cos(0.4), b * rE * np.sin(0.4))
    u = np.array([np.cos(0.4), np.sin(0.4)])
    yb = b * rE
    xp, xm = (yb + rE) * u, (yb - rE) * u
    dt = arrival_time(sis, *xm, src) - arrival_time(sis, *xp, src)
    assert dt == pytest.approx(2 * rE * yb, rel=1e-12)
    h = 1e-6
    for xi in (xp, xm):
        g = [(arrival_time(sis, *(xi + h * e), src) - arrival_time(sis, *(xi - h * e), src)) / (2 * h)
             for e in (np.array([1.0, 0.0]), np.array([0.0, 1.0]))]
        assert np.hypot(*g) < 1e-8


@pytest.mark.parametrize("y", [0.2, 1.0, 2.5])
def test_point_mass_time_delay_between_images(y):
    """Point mass m (r_E^2 = m in m-units): images at x+- = (y +- sqrt(y^2 + 4))
    / 2 in units of r_E; the arrival-time difference is r_E^2 [y sqrt(y^2 + 4)
    / 2 + ln((sqrt(y^2 + 4) + y) / (sqrt(y^2 + 4) - y))]."""
    m = 0.09
    rE = np.sqrt(m)
    pm = oracle.make_components(oracle.POINT, 0.0, 0.0, m)
    s = np.sqrt(y * y + 4)
    src = (y * rE, 0.0)
    xp, xm = 0.5 * (y + s) * rE, 0.5 * (y - s) * rE
    dt = arrival_time(pm, xm, 0.0, src) - arrival_time(pm, xp, 0.0, src)
    assert dt == pytest.approx(m * (0.5 * y * s + np.log((s + y) / (s - y))), rel=1e-12)
