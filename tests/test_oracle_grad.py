"""Pin of the oracle gradient: the vector-Jacobian product of the direct sum
against central finite differences of the FP64 loss L = sum |alpha - alpha_t|^2
(the lens-fit loss; beta = theta - alpha, Eq. lens_eq, so source-plane
residuals equal deflection residuals).  L is quadratic in the masses, so the
mass differences are exact up to rounding."""
import numpy as np
import pytest

import oracle
from oracle import GAUSS, NFW, POINT


def setup(seed=1):
    g = np.random.default_rng(seed)
    c = oracle.concat(
        oracle.make_components(GAUSS, g.uniform(-0.5, 0.5, 12), g.uniform(-0.5, 0.5, 12),
                               g.uniform(0.1, 1, 12), 0.15, 3.0),
        oracle.make_components(POINT, g.uniform(-0.5, 0.5, 4), g.uniform(-0.5, 0.5, 4),
                               g.uniform(0.1, 1, 4)),
        oracle.make_components(NFW, 0.1, 0.05, 0.5, 0.1, 0.4))
    rx, ry = g.uniform(-0.7, 0.7, 300), g.uniform(-0.7, 0.7, 300)
    target = oracle.direct_sum(c, rx, ry)[:, :2] * (1 + 0.05 * g.standard_normal((300, 2)))
    return c, rx, ry, target


def loss(c, rx, ry, target):
    a = oracle.direct_sum(c, rx, ry)[:, :2]
    return float(((a - target) ** 2).sum())


def test_vjp_matches_central_differences():
    c, rx, ry, target = setup()
    a = oracle.direct_sum(c, rx, ry)
    G = np.zeros_like(a)
    G[:, :2] = 2 * (a[:, :2] - target)
    grad = oracle.direct_vjp(c, rx, ry, G)
    for j in range(len(c)):
        for k, field in enumerate(["m", "x", "y"]):
            h = 1e-4 * abs(c[j]["m"]) if field == "m" else 1e-6

            def shifted(d):
                cc = c.copy()
                cc[j][field] += d
                return loss(cc, rx, ry, target)
            # 4th-order central difference (point masses near rays are steep)
            fd = (-shifted(2 * h) + 8 * shifted(h) - 8 * shifted(-h) + shifted(-2 * h)) / (12 * h)
            assert grad[j, k] == pytest.approx(fd, rel=2e-6, abs=1e-7 * np.abs(grad).max())


def test_vjp_rejects_kappa_gamma_gradients():
    c, rx, ry, _ = setup()
    G = np.zeros((rx.size, 5))
    G[:, 2] = 1.0
    with pytest.raises(ValueError):
        oracle.direct_vjp(c, rx, ry, G)
