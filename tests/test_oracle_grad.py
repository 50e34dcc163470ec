"""Pins of the oracle gradient: the vector-Jacobian product of the direct sum
against central finite differences of the FP64 loss L = sum |alpha - alpha_t|^2
(the lens-fit loss; beta = theta - alpha, Eq. lens_eq, so source-plane
residuals equal deflection residuals).  L is quadratic in the masses, so the
mass differences are exact up to rounding.  The shape-parameter derivatives
(GAUSS r_sm and q, NFW r_s and R_max, SIS r_E, DISK R) are pinned per
component against central differences of the component's own alpha."""
import numpy as np
import pytest

import oracle
from oracle import DISK, GAUSS, NFW, POINT, SIS


def setup(seed=1):
    g = np.random.default_rng(seed)
    c = oracle.concat(
        oracle.make_components(GAUSS, g.uniform(-0.5, 0.5, 12), g.uniform(-0.5, 0.5, 12),
                               g.uniform(0.1, 1, 12), 0.15, 3.0),
        oracle.make_components(POINT, g.uniform(-0.5, 0.5, 4), g.uniform(-0.5, 0.5, 4),
                               g.uniform(0.1, 1, 4)),
        oracle.make_components(NFW, 0.1, 0.05, 0.5, 0.1, 0.4),
        oracle.make_components(SIS, -0.15, 0.1, 0.0, 0.3),
        oracle.make_components(DISK, 0.05, -0.2, -0.2, 0.5))
    rx, ry = g.uniform(-0.7, 0.7, 300), g.uniform(-0.7, 0.7, 300)
    target = oracle.direct_sum(c, rx, ry)[:, :2] * (1 + 0.05 * g.standard_normal((300, 2)))
    return c, rx, ry, target


def loss(c, rx, ry, target):
    a = oracle.direct_sum(c, rx, ry)[:, :2]
    return float(((a - target) ** 2).sum())


def fd4(f, h):
    return (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)


def test_vjp_matches_central_differences():
    c, rx, ry, target = setup()
    a = oracle.direct_sum(c, rx, ry)
    G = np.zeros_like(a)
    G[:, :2] = 2 * (a[:, :2] - target)
    grad = oracle.direct_vjp(c, rx, ry, G, params=True)
    np.testing.assert_array_equal(grad[:, :3], oracle.direct_vjp(c, rx, ry, G))
    for j in range(len(c)):
        fields = ["m", "x", "y"]
        if c[j]["type"] in (GAUSS, NFW):
            fields += ["p0", "p1"]
        elif c[j]["type"] in (SIS, DISK):
            fields += ["p0"]
        for field in fields:
            k = ["m", "x", "y", "p0", "p1"].index(field)
            if c[j]["type"] == SIS and field == "m":
                continue  # the SIS has no mass parameter (m is unused)
            # shape steps stay below 1e-5 relative: a ray 1.3e-5 from a
            # support edge (where d alpha / d r_sm jumps to 0) sits inside a
            # 1e-4 stencil
            h = {"m": 1e-4, "p0": 1e-6, "p1": 1e-6}.get(field, 0.0) * abs(c[j][field]) or 1e-6

            def shifted(d):
                cc = c.copy()
                cc[j][field] += d
                return loss(cc, rx, ry, target)
            # 4th-order central difference (point masses near rays are steep)
            assert grad[j, k] == pytest.approx(fd4(shifted, h), rel=2e-6, abs=1e-7 * np.abs(grad).max()), \
                (j, field)
        if c[j]["type"] == POINT:
            assert grad[j, 3] == 0.0 and grad[j, 4] == 0.0


@pytest.mark.parametrize("comp,radii", [
    (oracle.make_components(GAUSS, 0.0, 0.0, 0.7, 0.1, 3.0), [1e-3, 0.05, 0.1, 0.25, 0.29, 0.31, 0.5]),
    (oracle.make_components(NFW, 0.0, 0.0, 0.7, 0.1, 0.5), [5e-4, 2e-3, 0.02, 0.0995, 0.1, 0.1003, 0.3, 0.49, 0.6]),
    (oracle.make_components(SIS, 0.0, 0.0, 0.0, 0.4), [1e-3, 0.2, 1.0]),
    (oracle.make_components(DISK, 0.0, 0.0, -0.3, 0.4), [0.05, 0.39, 0.41, 1.0]),
])
def test_shape_parameter_derivatives_of_alpha(comp, radii):
    """d alpha / d p0, d p1 of one component at rays inside and outside its
    support, against central differences of or_eval_component; read through
    direct_vjp with an upstream gradient of 1 on alpha1 at one ray (a ray on
    the x axis at distance r; the derivative of alpha2 there is 0)."""
    for r in radii:
        G = np.zeros((1, 5))
        G[0, 0] = 1.0
        got = oracle.direct_vjp(comp, [r], [0.0], G, params=True)[0]
        for k, field in ((3, "p0"), (4, "p1")):
            base = comp[0][field]
            if base == 0.0:
                assert got[k] == 0.0
                continue
            h = 1e-5 * base

            def a1(d):
                cc = comp.copy()
                cc[0][field] = base + d
                return oracle.eval_component(cc[0], r, 0.0)[0]
            fd = fd4(a1, h)
            assert got[k] == pytest.approx(fd, rel=1e-7, abs=1e-9 * max(1.0, abs(fd))), (r, field)


def test_vjp_rejects_kappa_gamma_gradients():
    c, rx, ry, _ = setup()
    G = np.zeros((rx.size, 5))
    G[:, 2] = 1.0
    with pytest.raises(ValueError):
        oracle.direct_vjp(c, rx, ry, G)
