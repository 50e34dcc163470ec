"""Pins of the refinement oracle (oracle/refine.py) against the mathematics
and the paper: the App. A solve inverts an exactly affine map and agrees with
a direct solve of the printed 4x4 system; the two ways of getting A agree on
the SIS of App. B, whose det A = 1 - r_E/r; interpolated deflections on
uniform cells agree with direct shooting to a part in 1e4 (the accuracy the
paper reports for its interpolation); cells next to a point mass are not
uniform."""
import numpy as np
import pytest

import oracle
from oracle import refine as R


def grid(x0, y0, h, nx, ny):
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    return (x0 + i * h).ravel(), (y0 + j * h).ravel()


def test_app_a_inverts_an_affine_map():
    g = np.random.default_rng(1)
    M = np.array([[0.7, -0.31], [0.12, 1.4]])  # not symmetric: a21 != a12
    y0 = np.array([0.2, -0.5])
    nx, ny, h = 12, 9, 0.013
    x, y = grid(0.3, -0.2, h, nx, ny)
    # alpha = x - y(x) with y = y0 + M x
    a1 = x - (y0[0] + M[0, 0] * x + M[0, 1] * y)
    a2 = y - (y0[1] + M[1, 0] * x + M[1, 1] * y)
    cells = R.interior_cells(nx, ny)
    uni, A, ys, stat = R.refine_cells(0.3, -0.2, h, nx, ny, a1, a2, None, None, None, cells, 3, 1e-4,
                                      R.DEFLECTION)
    assert uni.all() and stat.max() < 1e-12
    # (a11, a21, a12, a22) with dy1 = a11 dx1 + a21 dx2, dy2 = a12 dx1 + a22 dx2
    np.testing.assert_allclose(A, np.broadcast_to([M[0, 0], M[0, 1], M[1, 0], M[1, 1]], A.shape), atol=1e-12)
    i, j = cells % nx, cells // nx
    d = (np.arange(3) - 1) * h / 3
    for b in range(3):
        for a in range(3):
            xs = 0.3 + i * h + d[a]
            yy = -0.2 + j * h + d[b]
            np.testing.assert_allclose(ys[:, b, a, 0], y0[0] + M[0, 0] * xs + M[0, 1] * yy, atol=1e-12)
            np.testing.assert_allclose(ys[:, b, a, 1], y0[1] + M[1, 0] * xs + M[1, 1] * yy, atol=1e-12)
    del g


def test_app_a_closed_form_matches_the_printed_linear_system():
    g = np.random.default_rng(2)
    for _ in range(50):
        dx1, dx2, dy1, dy2 = (g.normal(size=2) for _ in range(4))
        A, det = R.app_a_solve(dx1, dy1, dx2, dy2)
        # the 4x4 system of App. A: (dy1^(1), dy2^(1), dy1^(2), dy2^(2)) = X (a11, a21, a12, a22)
        X = np.array([[dx1[0], dx1[1], 0, 0], [0, 0, dx1[0], dx1[1]],
                      [dx2[0], dx2[1], 0, 0], [0, 0, dx2[0], dx2[1]]])
        sol = np.linalg.solve(X, np.array([dy1[0], dy1[1], dy2[0], dy2[1]]))
        np.testing.assert_allclose(A, sol, rtol=1e-9, atol=1e-12)


def test_sis_two_routes_to_A_and_appendix_b_magnification():
    rE = 0.5
    comps = oracle.make_components(oracle.SIS, 0.0, 0.0, 0.0, rE)
    nx = ny = 24
    h = 5e-5  # small enough that gamma (rotating as 2 phi) stays within 1e-4 across a cell
    x0, y0 = 0.8, 0.3
    x, y = grid(x0, y0, h, nx, ny)
    out = oracle.direct_sum(comps, x, y)
    cells = R.interior_cells(nx, ny)
    uk, Ak, _, _ = R.refine_cells(x0, y0, h, nx, ny, out[:, 0], out[:, 1], out[:, 2], out[:, 3], out[:, 4],
                                  cells, 3, 1e-4, R.KAPPA_GAMMA)
    ud, Ad, _, _ = R.refine_cells(x0, y0, h, nx, ny, out[:, 0], out[:, 1], None, None, None,
                                  cells, 3, 1e-4, R.DEFLECTION)
    assert uk.all() and ud.all()
    # finite differences of the deflection are second-order accurate in h
    np.testing.assert_allclose(Ad, Ak, atol=1e-6)
    r = np.hypot(x[cells], y[cells])
    det = Ak[:, 0] * Ak[:, 3] - Ak[:, 1] * Ak[:, 2]
    np.testing.assert_allclose(det, 1.0 - rE / r, rtol=1e-12)


def test_interpolation_agrees_with_direct_shooting_to_1e4():
    # an SIS plus a small NFW halo inside the grid: uniform cells away from
    # the halo's centre, non-uniform ones near it
    comps = oracle.concat(oracle.make_components(oracle.SIS, 0.0, 0.0, 0.0, 0.5),
                          oracle.make_components(oracle.NFW, [0.8026], [0.3021], [5e-9], [1e-3], [3e-3]))
    nx = ny = 48
    h = 1e-4
    x0, y0 = 0.8, 0.3
    x, y = grid(x0, y0, h, nx, ny)
    out = oracle.direct_sum(comps, x, y)
    cells = R.interior_cells(nx, ny)
    for mode in (R.KAPPA_GAMMA, R.DEFLECTION):
        uni, A, ys, _ = R.refine_cells(x0, y0, h, nx, ny, *(out[:, q] for q in range(5)), cells, 3, 1e-4, mode)
        assert 0.2 < uni.mean() < 1.0, uni.mean()
        sel = cells[uni]
        i, j = sel % nx, sel // nx
        d = (np.arange(3) - 1) * h / 3
        for b in range(3):
            for a in range(3):
                xs, yy = x0 + i * h + d[a], y0 + j * h + d[b]
                ref = oracle.direct_sum(comps, xs, yy)
                alpha_int = np.stack([xs - ys[uni, b, a, 0], yy - ys[uni, b, a, 1]], axis=1)
                err = np.hypot(*(alpha_int - ref[:, :2]).T) / np.hypot(ref[:, 0], ref[:, 1])
                assert err.max() <= 1e-4, (mode, err.max())


def test_cells_next_to_a_point_mass_are_not_uniform():
    comps = oracle.make_components(oracle.POINT, 0.5005, 0.5005, 1e-8)
    nx = ny = 32
    h = 1e-3
    x, y = grid(0.49, 0.49, h, nx, ny)
    out = oracle.direct_sum(comps, x, y)
    cells = R.interior_cells(nx, ny)
    uni, _, ys, _ = R.refine_cells(0.49, 0.49, h, nx, ny, *(out[:, q] for q in range(5)), cells, 3, 1e-4,
                                   R.DEFLECTION)
    i, j = cells % nx, cells // nx
    r = np.hypot(0.49 + i * h - 0.5005, 0.49 + j * h - 0.5005)
    assert not uni[r < 3 * h].any()
    assert uni[r > 12 * h].all()
    assert np.isnan(ys[~uni]).all() and np.isfinite(ys[uni]).all()


@pytest.mark.parametrize("k", [1, 3, 5])
def test_subcell_centres(k):
    nx = ny = 5
    a = np.zeros(nx * ny)
    cells = R.interior_cells(nx, ny)
    uni, _, ys, _ = R.refine_cells(0.0, 0.0, 1.0, nx, ny, a, a, a, a, a, cells, k, 1e-4, R.KAPPA_GAMMA)
    assert uni.all()
    c = (k - 1) // 2
    i, j = cells % nx, cells // nx
    np.testing.assert_array_equal(ys[:, c, c, 0], i * 1.0)
    np.testing.assert_array_equal(ys[:, c, c, 1], j * 1.0)
    np.testing.assert_allclose(ys[:, c, -1, 0] - ys[:, c, 0, 0], (k - 1) / k)


def test_edge_cells_are_rejected():
    a = np.zeros(16)
    with pytest.raises(ValueError):
        R.refine_cells(0.0, 0.0, 1.0, 4, 4, a, a, a, a, a, [0], 3, 1e-4, R.KAPPA_GAMMA)
