"""GPU parity of lens_refine_cells (Sec. 3.4 interpolation, App. A) against
the FP64 refinement oracle on the same grid inputs, which come from the
oracle's direct sum (no input or expected value passes through the CUDA
path).

Bars: the uniform flags are equal wherever the oracle's statistic is farther
from tol than the rounding of the GPU's comparison (FP32 for kappa/gamma and
FP32 deflections, FP64 for FP64 deflections); A within its FP32 rounding;
sub-cell source positions within the FP32 rounding of A times the sub-cell
offset; NaN exactly where a cell is not uniform.
"""
import numpy as np
import pytest

import lensgen
import oracle
from oracle import refine as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1312_1128_gb300 as L  # noqa: E402


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def lens_grid(nx, ny, x0, y0, h, seed=41, n_halos=6):
    """An SIS plus small NFW halos inside the grid, evaluated by the oracle."""
    g = lensgen.rng(seed)
    hx = x0 + g.uniform(0, nx * h, n_halos)
    hy = y0 + g.uniform(0, ny * h, n_halos)
    comps = oracle.concat(oracle.make_components(oracle.SIS, 0.0, 0.0, 0.0, 0.5),
                          oracle.make_components(oracle.NFW, hx, hy, 10 ** g.uniform(-9.5, -8, n_halos),
                                                 np.full(n_halos, 5 * h), np.full(n_halos, 15 * h)))
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    x, y = (x0 + i * h).ravel(), (y0 + j * h).ravel()
    return oracle.direct_sum(comps, x, y)


def check(out, x0, y0, h, nx, ny, cells, k, mode, adtype):
    tol = 1e-4
    a1, a2 = out[:, 0].astype(adtype), out[:, 1].astype(adtype)
    kg = [out[:, q].astype(np.float32) for q in (2, 3, 4)]
    uni, A, ys = L.refine_cells(x0, y0, h, nx, ny, cu(a1), cu(a2), *(cu(v) for v in kg), cells=cu(cells), k=k,
                                tol=tol, mode=mode)
    torch.cuda.synchronize()
    uni, A, ys = uni.cpu().numpy(), A.cpu().numpy(), ys.cpu().numpy()
    ru, rA, rys, stat = R.refine_cells(x0, y0, h, nx, ny, a1, a2, *kg, cells, k, tol, mode)
    band = 1e-12 if (mode == R.DEFLECTION and adtype == np.float64) else 1e-6
    clear = np.abs(stat - tol) > band
    assert np.array_equal(uni[clear] == 1, ru[clear])
    assert set(np.unique(uni)) <= {0, 1}
    np.testing.assert_allclose(A, rA, atol=1e-6 if mode == R.DEFLECTION and adtype == np.float32 else 3e-7)
    both = (uni == 1) & ru
    assert np.isnan(ys[uni == 0]).all() and np.isfinite(ys[uni == 1]).all()
    atol = 1e-6 * h + 4e-16 * np.abs(rys[both]).max() if both.any() else 0
    np.testing.assert_allclose(ys[both], rys[both], rtol=0, atol=atol)
    return uni


@pytest.mark.parametrize("mode", [R.KAPPA_GAMMA, R.DEFLECTION])
@pytest.mark.parametrize("adtype", [np.float32, np.float64])
@pytest.mark.parametrize("k", [1, 3, 5])
def test_refine_matches_oracle(mode, adtype, k):
    nx, ny, h, x0, y0 = 96, 80, 1e-4, 0.8, 0.3
    out = lens_grid(nx, ny, x0, y0, h)
    cells = R.interior_cells(nx, ny)
    uni = check(out, x0, y0, h, nx, ny, cells, k, mode, adtype)
    if mode == R.KAPPA_GAMMA or adtype == np.float64:
        assert 0.05 < uni.mean() < 0.999
    # FP32 deflections (ulp ~6e-8 at |alpha| ~ 0.5) cannot resolve A to 1e-4
    # from differences across h = 1e-4: the reason Sec. 3.4 computes the
    # deflection to higher precision for this test; few cells pass then


def test_refine_invalid_cells_and_empty():
    nx, ny, h = 16, 16, 1e-4
    out = lens_grid(nx, ny, 0.8, 0.3, h)
    cells = np.array([0, 5, nx + 1, nx * ny - 1, -3, nx * ny + 7, 2 * nx + 2], np.int64)
    a = [cu(out[:, q].astype(np.float32)) for q in range(5)]
    uni, A, ys = L.refine_cells(0.8, 0.3, h, nx, ny, *a, cells=cu(cells))
    uni, A, ys = uni.cpu().numpy(), A.cpu().numpy(), ys.cpu().numpy()
    bad = np.array([1, 1, 0, 1, 1, 1, 0], bool)
    assert (uni[bad] == 2).all() and (uni[~bad] < 2).all()
    assert np.isnan(A[bad]).all() and np.isnan(ys[bad]).all() and np.isfinite(A[~bad]).all()
    u0, A0, y0 = L.refine_cells(0.8, 0.3, h, nx, ny, *a, cells=cu(np.zeros(0, np.int64)))
    assert u0.numel() == 0


def test_refine_fullsize_sampled():
    """2048^2 grid, every interior cell refined on the GPU (3x3 sub-cells,
    both modes); 4,096 sampled cells against the oracle."""
    nx = ny = 2048
    h, x0, y0 = 5e-5, 0.7, 0.2
    out = lens_grid(nx, ny, x0, y0, h, seed=42, n_halos=40)
    g = lensgen.rng(43)
    allc = R.interior_cells(nx, ny)
    sample = np.sort(g.choice(allc.size, 4096, replace=False))
    for mode in (R.KAPPA_GAMMA, R.DEFLECTION):
        a = [cu(out[:, q].astype(np.float32)) for q in range(5)]
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        uni, A, ys = L.refine_cells(x0, y0, h, nx, ny, *a, k=3, mode=mode, n_nonuniform=cnt)  # implicit cells
        torch.cuda.synchronize()
        assert uni.numel() == allc.size and int(cnt.item()) == int((uni == 0).sum().item())
        # the implicit list is every interior cell in row-major order
        u2, A2, y2 = L.refine_cells(x0, y0, h, nx, ny, *a, cells=cu(allc[:70000]), k=3, mode=mode)
        assert torch.equal(u2, uni[:70000]) and torch.equal(A2, A[:70000])
        assert torch.equal(torch.nan_to_num(y2), torch.nan_to_num(ys[:70000]))
        idx = torch.from_numpy(sample).cuda()
        got_u, got_A, got_y = uni[idx].cpu().numpy(), A[idx].cpu().numpy(), ys[idx].cpu().numpy()
        kg = [out[:, q].astype(np.float32) for q in (2, 3, 4)]
        ru, rA, rys, stat = R.refine_cells(x0, y0, h, nx, ny, out[:, 0].astype(np.float32),
                                           out[:, 1].astype(np.float32), *kg, allc[sample], 3, 1e-4, mode)
        clear = np.abs(stat - 1e-4) > 1e-6
        assert np.array_equal(got_u[clear] == 1, ru[clear])
        np.testing.assert_allclose(got_A, rA, atol=1e-6)
        both = (got_u == 1) & ru
        np.testing.assert_allclose(got_y[both], rys[both], rtol=0, atol=1e-6 * h + 4e-16 * 2)
