"""Pins of the oracle's direct sum (Sec. 3.2 superposition; Sec. 5.1 theta = 0).

Invariants that any correct sum must satisfy: superposition and linearity in
the masses, rotation covariance (alpha spin 1, gamma spin 2, kappa scalar),
translation invariance, mirror parity, the far-field monopole limit, exact
cancellation by symmetry, and compensated summation of ill-conditioned sums.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import DISK, GAUSS, NFW, POINT, SIS


def mixed(seed, n=40):
    g = np.random.default_rng(seed)
    k = n // 4
    return oracle.concat(
        oracle.make_components(POINT, g.uniform(-1, 1, k), g.uniform(-1, 1, k), g.uniform(0.1, 1, k)),
        oracle.make_components(GAUSS, g.uniform(-1, 1, k), g.uniform(-1, 1, k), g.uniform(0.1, 1, k),
                               g.uniform(0.02, 0.2, k), 3.0),
        oracle.make_components(NFW, g.uniform(-1, 1, k), g.uniform(-1, 1, k), g.uniform(0.1, 1, k),
                               g.uniform(0.02, 0.1, k), g.uniform(0.2, 0.4, k)),
        oracle.make_components(DISK, 0.2, -0.1, -0.3, 0.5),
        oracle.make_components(SIS, -0.3, 0.25, 0.0, 0.4),
    )


def rays(seed, n=200, lo=-1.3, hi=1.3):
    g = np.random.default_rng(seed)
    return g.uniform(lo, hi, n), g.uniform(lo, hi, n)


def test_superposition_and_linearity():
    c = mixed(1)
    rx, ry = rays(2)
    full = oracle.direct_sum(c, rx, ry)
    a = oracle.direct_sum(c[:17], rx, ry)
    b = oracle.direct_sum(c[17:], rx, ry)
    np.testing.assert_allclose(full, a + b, rtol=1e-12, atol=1e-12 * np.abs(full).max())
    c2 = c.copy()
    lin = c2["type"] != SIS            # SIS strength is r_E, not m
    c2["m"][lin] *= 2.5
    c2["p0"][~lin] *= 2.5
    np.testing.assert_allclose(oracle.direct_sum(c2, rx, ry), 2.5 * full, rtol=1e-12,
                               atol=1e-12 * np.abs(full).max())


@pytest.mark.parametrize("ang", [0.37, math.pi / 2, 2.1])
def test_rotation_covariance(ang):
    c = mixed(3)
    rx, ry = rays(4)
    base = oracle.direct_sum(c, rx, ry)
    cs, sn = math.cos(ang), math.sin(ang)
    cr = c.copy()
    cr["x"], cr["y"] = cs * c["x"] - sn * c["y"], sn * c["x"] + cs * c["y"]
    rot = oracle.direct_sum(cr, cs * rx - sn * ry, sn * rx + cs * ry)
    a = base[:, 0] + 1j * base[:, 1]
    g = base[:, 3] + 1j * base[:, 4]
    tol = 1e-11 * np.abs(base).max()
    np.testing.assert_allclose(rot[:, 0] + 1j * rot[:, 1], a * np.exp(1j * ang), atol=tol)
    np.testing.assert_allclose(rot[:, 2], base[:, 2], atol=tol)
    np.testing.assert_allclose(rot[:, 3] + 1j * rot[:, 4], g * np.exp(2j * ang), atol=tol)


def test_translation_and_mirror():
    c = mixed(5)
    rx, ry = rays(6)
    base = oracle.direct_sum(c, rx, ry)
    ct = c.copy()
    ct["x"] += 0.75
    ct["y"] -= 0.5
    tr = oracle.direct_sum(ct, rx + 0.75, ry - 0.5)
    np.testing.assert_allclose(tr, base, atol=1e-10 * np.abs(base).max())
    cm = c.copy()
    cm["y"] = -c["y"]
    mi = oracle.direct_sum(cm, rx, -ry)
    sign = np.array([1, -1, 1, 1, -1])
    np.testing.assert_allclose(mi, base * sign, atol=1e-11 * np.abs(base).max())


def test_far_field_monopole():
    c = mixed(7)
    c = c[c["type"] != SIS]
    M = c["m"].sum()
    xc = (c["m"] * c["x"]).sum() / M
    yc = (c["m"] * c["y"]).sum() / M
    for R in [50.0, 500.0]:
        phi = np.linspace(0, 2 * np.pi, 9)[:-1]
        rx, ry = xc + R * np.cos(phi), yc + R * np.sin(phi)
        out = oracle.direct_sum(c, rx, ry)
        mono = M * np.stack([rx - xc, ry - yc]) / R ** 2
        # quadrupole remainder ~ M d^2 / R^3 with d ~ 1.5
        np.testing.assert_allclose(out[:, :2].T, mono, atol=abs(M) * 3.0 / R ** 3)
        assert np.all(out[:, 2] == 0.0)


def test_symmetric_configuration_cancels():
    # four equal masses at the corners of a square: alpha and gamma vanish at the centre
    c = oracle.make_components(GAUSS, [1, -1, 1, -1], [1, 1, -1, -1], 0.3, 0.2, 3.0)
    out = oracle.direct_sum(c, [0.0], [0.0])
    assert np.all(np.abs(out[0, [0, 1, 3, 4]]) < 1e-16)


def test_compensated_sum_on_cancelling_terms():
    """Many large opposite contributions: the sum must keep the small total."""
    n = 2000
    g = np.random.default_rng(9)
    x = g.uniform(1e-3, 1e-2, n)
    # pairs mirrored through the ray at the origin cancel exactly in alpha;
    # one extra point leaves a known small remainder
    c = oracle.concat(oracle.make_components(POINT, x, 0.0, 1.0),
                      oracle.make_components(POINT, -x, 0.0, 1.0),
                      oracle.make_components(POINT, 10.0, 0.0, 1e-3))
    out, ab = oracle.direct_sum(c, [0.0], [0.0], with_absum=True)
    # the lone mass at x = 10 pulls the ray towards +x: alpha1 = -1e-3 * 10 / 100
    assert out[0, 0] == pytest.approx(-1e-4, rel=1e-9)
    assert ab[0, 0] > 1e5 * abs(out[0, 0])


def test_absum_bounds_the_sum():
    c = mixed(11)
    rx, ry = rays(12)
    out, ab = oracle.direct_sum(c, rx, ry, with_absum=True)
    assert np.all(ab >= np.abs(out) * (1 - 1e-12))
