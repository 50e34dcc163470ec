"""Parity at the workloads' full sizes, in the configuration bench.py times,
checked on sampled rays that the FP64 oracle computes one by one.

* smoothed NFW particles (1e6, r_sm = 32nd 3D neighbour, q = 3), 2048^2 grid:
  tree medians at theta = 0.3 and 0.1, kappa exact, FP32 direct sum bar;
* NFW halos + 1e6 stars, 256 uneven refinement batches (3.7e7 rays) in one
  persistent launch, eager and CUDA-graph replay;
* 1e7 stars + SIS, 4096^2 rays over a 1e-6 patch, FP64 origin + FP32
  offsets, theta = 0.1;
* the lens fit (1e5 Gaussians, 1e6 rays): tree adjoint against the oracle's
  vector-Jacobian product for 64 random particles; direct-sum adjoint against
  central differences of the FP64 loss on 64 random masses.
"""
import numpy as np
import pytest

import lensgen
import oracle
from lens_testutil import comps_gauss, comps_nfw, comps_points, rel_errors, to_np, within_fp32_bar

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1312_1128_gb300 as L  # noqa: E402


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def pick(out, idx):
    return np.stack([o[idx].double().cpu().numpy() for o in out], axis=1)


@pytest.fixture(scope="module")
def sph():
    return lensgen.workload_nfw_sph()


@pytest.mark.parametrize("theta,bar", [(0.3, 1e-3), (0.1, 1e-4)])
def test_sph_fullsize_tree(sph, theta, bar):
    w = sph
    parts = cu(w["gauss"])
    rx, ry = cu(w["rx"]), cu(w["ry"])
    lens = L.Lens([L.Species.gauss(parts, w["q"])], theta=theta)
    g = lensgen.rng(91)
    idx = lensgen.sample_indices(g, w["rx"].size, 1024)
    for gr in (32, 64):
        lens.close()
        lens = L.Lens([L.Species.gauss(parts, w["q"])], theta=theta, group_rays=gr)
        out = lens.shoot(rx, ry)
        lens.sync()
        got = pick(out, torch.from_numpy(idx).cuda())
        comps = comps_gauss(w["gauss"], w["q"])
        ref = oracle.direct_sum(comps, w["rx"][idx].astype(np.float64), w["ry"][idx].astype(np.float64))
        ea, ek, eg = rel_errors(got, ref)
        assert np.median(ea) <= bar, (gr, np.median(ea))
        assert np.median(eg) <= bar, (gr, np.median(eg))
        assert np.quantile(ek, 0.99) <= 1e-5, (gr, np.quantile(ek, 0.99))
    lens.close()


def test_sph_fullsize_direct_sample(sph):
    w = sph
    g = lensgen.rng(92)
    idx = lensgen.sample_indices(g, w["rx"].size, 512)
    lens = L.Lens([L.Species.gauss(cu(w["gauss"]), w["q"])], theta=0.3)
    out = lens.shoot(cu(w["rx"][idx]), cu(w["ry"][idx]), flags=L.DIRECT)
    lens.sync()
    got = to_np(out)
    comps = comps_gauss(w["gauss"], w["q"])
    ref, absum = oracle.direct_sum(comps, w["rx"][idx].astype(np.float64), w["ry"][idx].astype(np.float64),
                                   with_absum=True)
    ok, frac = within_fp32_bar(got, ref, absum)
    # kappa may differ where a ray sits within FP32 rounding of a support edge
    assert ok[:, [0, 2]].all() and ok[:, 1].mean() >= 0.99
    assert frac <= 0.05
    lens.close()


def test_mixed_batches_fullsize():
    w = lensgen.workload_mixed_batches()
    lens = L.Lens([L.Species.points(cu(w["points"])), L.Species.nfw(cu(w["nfw"]), w["conc"])], theta=0.3)
    dx, dy = cu(w["dx"]), cu(w["dy"])
    n = dx.numel()
    assert 3e7 < n < 4.5e7
    out = [torch.empty(n, device="cuda") for _ in range(5)]
    lens.reserve(n, len(w["offsets"]) - 1)
    lens.shoot_batches(w["offsets"], w["origins"], dx, dy, flags=L.USE_GRAPH, out=out)   # eager + capture
    lens.shoot_batches(w["offsets"], w["origins"], dx, dy, flags=L.USE_GRAPH, out=out)   # replay
    lens.sync()
    g = lensgen.rng(93)
    idx = lensgen.sample_indices(g, n, 2048)
    got = pick(out, torch.from_numpy(idx).cuda())
    b = np.searchsorted(w["offsets"], idx, side="right") - 1
    rx = w["origins"][b, 0] + w["dx"][idx].astype(np.float64)
    ry = w["origins"][b, 1] + w["dy"][idx].astype(np.float64)
    comps = oracle.concat(comps_points(w["points"]), comps_nfw(w["nfw"], w["conc"]))
    ref = oracle.direct_sum(comps, rx, ry)
    ea, ek, eg = rel_errors(got, ref)
    assert np.median(ea) <= 1e-3 and np.median(eg) <= 1e-3
    assert np.quantile(ek, 0.99) <= 1e-5
    lens.close()


def test_microlensing_fullsize():
    w = lensgen.workload_microlensing()
    lens = L.Lens([L.Species.points(cu(w["points"]))], [L.Halo.sis(0.0, 0.0, w["sis_re"])], theta=0.1)
    out = lens.shoot(cu(w["dx"]), cu(w["dy"]), origin=w["origin"])
    lens.sync()
    g = lensgen.rng(94)
    idx = lensgen.sample_indices(g, w["dx"].size, 1024)
    got = pick(out, torch.from_numpy(idx).cuda())
    comps = oracle.concat(comps_points(w["points"]), oracle.make_components(oracle.SIS, 0, 0, 0, w["sis_re"]))
    ref = oracle.direct_sum(comps, w["origin"][0] + w["dx"][idx].astype(np.float64),
                            w["origin"][1] + w["dy"][idx].astype(np.float64))
    ea, _, eg = rel_errors(got, ref)
    assert np.median(ea) <= 1e-4 and np.median(eg) <= 1e-4
    lens.close()


@pytest.fixture(scope="module")
def fit():
    return lensgen.workload_fit()


def test_fit_fullsize_adjoint_vs_oracle_vjp(fit):
    w = fit
    parts, target = w["gauss"], w["target"]
    dx, dy = cu(w["rx"]), cu(w["ry"])
    lens = L.Lens([L.Species.gauss(cu(parts), w["q"])], theta=0.1)
    tl = L.Lens([L.Species.gauss(cu(target), w["q"])], theta=0.1)
    a = lens.shoot(dx, dy, flags=L.ALPHA_ONLY)
    at = tl.shoot(dx, dy, flags=L.ALPHA_ONLY)
    G1, G2 = (2 * (a[0] - at[0])).contiguous(), (2 * (a[1] - at[1])).contiguous()
    (grad,) = lens.backward(dx, dy, G1, G2)
    grad = grad.double().cpu().numpy()
    # the oracle's VJP of a particle needs that particle alone
    g = lensgen.rng(95)
    sel = g.choice(parts.shape[0], 64, replace=False)
    G = np.zeros((w["rx"].size, 5))
    G[:, 0] = G1.double().cpu().numpy()
    G[:, 1] = G2.double().cpu().numpy()
    ref = oracle.direct_vjp(comps_gauss(parts[sel], w["q"]), w["rx"].astype(np.float64),
                            w["ry"].astype(np.float64), G)
    errs = [np.linalg.norm(grad[sel, k] - ref[:, k]) / np.linalg.norm(ref[:, k]) for k in range(3)]
    print("full-size fit: tree adjoint vs oracle VJP, rel L2 m, x, y =", errs)
    for k in range(3):
        assert errs[k] <= 5e-3, (k, errs[k])
    lens.close()
    tl.close()


def test_fit_fullsize_mass_finite_differences_fp64(fit):
    """Direct-sum adjoint with all 1e5 particles against central differences
    of the FP64 direct-sum loss on 64 random masses (2,048 sampled rays).
    The tree loss itself is only piecewise smooth in the masses (r_cut moves
    with the centre of mass, so MAC decisions can flip inside a stencil); the
    tree adjoint is checked against the oracle's VJP above and against finite
    differences where no decision flips (test_gpu_backward)."""
    w = fit
    p64 = w["gauss"].astype(np.float64)
    t64 = w["target"].astype(np.float64)
    g = lensgen.rng(96)
    idx = lensgen.sample_indices(g, w["rx"].size, 2048)
    dx, dy = cu(w["rx"][idx].astype(np.float64)), cu(w["ry"][idx].astype(np.float64))
    tl = L.Lens([L.Species.gauss(cu(t64), w["q"])], theta=0.3, precision="fp64")
    t_out = tl.shoot(dx, dy, flags=L.ALPHA_ONLY | L.DIRECT)
    alpha_t = torch.stack([t_out[0], t_out[1]], 1)

    def loss(p):
        lens = L.Lens([L.Species.gauss(cu(p), w["q"])], theta=0.3, precision="fp64")
        out = lens.shoot(dx, dy, flags=L.ALPHA_ONLY | L.DIRECT)
        v = float(((torch.stack([out[0], out[1]], 1) - alpha_t) ** 2).sum())
        lens.close()
        return v

    lens = L.Lens([L.Species.gauss(cu(p64), w["q"])], theta=0.3, precision="fp64")
    out = lens.shoot(dx, dy, flags=L.ALPHA_ONLY | L.DIRECT)
    r = torch.stack([out[0], out[1]], 1) - alpha_t
    (grad,) = lens.backward(dx, dy, (2 * r[:, 0]).contiguous(), (2 * r[:, 1]).contiguous(), flags=L.DIRECT)
    grad = grad.cpu().numpy()
    for j in g.choice(p64.shape[0], 64, replace=False):
        h = 1e-4 * p64[j, 2]

        def at(d):
            q = p64.copy()
            q[j, 2] += d
            return loss(q)
        fd = (at(h) - at(-h)) / (2 * h)
        assert grad[j, 0] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(grad[:, 0]).max())
    lens.close()
    tl.close()


def test_potential_fullsize_tree(sph):
    """The potential workload as bench.py times it (1e6 smoothed NFW particles,
    2048^2 rays, theta = 0.3, 32- and 64-ray groups): psi on 512 sampled rays
    against the oracle's direct potential at the deflection's bar (1e-3 of
    |psi| at the median ray), and the call's alpha equal to shoot()'s."""
    w = sph
    parts = cu(w["gauss"])
    rx, ry = cu(w["rx"]), cu(w["ry"])
    g = lensgen.rng(93)
    idx = lensgen.sample_indices(g, w["rx"].size, 512)
    ti = torch.from_numpy(idx).cuda()
    comps = comps_gauss(w["gauss"], w["q"])
    ref = oracle.direct_potential(comps, w["rx"][idx].astype(np.float64), w["ry"][idx].astype(np.float64))
    for gr in (32, 64):
        lens = L.Lens([L.Species.gauss(parts, w["q"])], theta=0.3, group_rays=gr)
        psi, a1, a2 = lens.potential(rx, ry)
        e = np.abs(psi[ti].double().cpu().numpy() - ref) / np.abs(ref)
        assert np.median(e) <= 1e-3, (gr, np.median(e))
        s = lens.shoot(rx, ry, flags=L.ALPHA_ONLY)
        lens.sync()
        d = (a1 - s[0]).abs().max().item()
        assert d <= 1e-4 * s[0].abs().max().item(), (gr, d)
        lens.close()


def test_images_fullsize_sis_test():
    """The image-finding workload as bench.py times it: the 62 sources of the
    Sec. 5.2 SIS test in one call; every image above mu_min found, none
    spurious, all magnifications within 0.7 % of App. B (median below 0.05 %),
    and the same result on a second call (the workspace is reused)."""
    from oracle import images as I
    src = []
    for R in (0.1, 0.01, 1e-4):
        for b in np.round(np.linspace(0.0, 2.0, 21), 6):
            if R < 1e-3 and b == 0.0:
                continue
            src.append((float(b), 0.0, R))
    lens = L.Lens([], [L.Halo.sis(0.0, 0.0, 1.0)], theta=0.3, precision="fp64")
    kw = dict(x0=-10.0, y0=-10.0, side=20.0, n=64, l_max=12, mu_min=0.01, f_area=5e-4, n_min=50,
              max_cells=1 << 26, max_images=1024)
    imgs, st = lens.find_images(src, **kw)
    errs = []
    for k, (b, _, R) in enumerate(src):
        mp, mm, ring = I.sis_finite_source_mu(b, R)
        exp = [mp + mm] if ring else ([mp, mm] if mm > 0 else [mp])
        got = sorted((im["mu"] for im in imgs if im["source"] == k), reverse=True)
        assert len(got) <= len(exp), (b, R, got)
        assert all(m < 0.01 for m in exp[len(got):]), (b, R, got, exp)
        errs += [abs(a / e - 1.0) for a, e in zip(got, exp)]
    errs = np.array(errs)
    assert errs.max() < 7e-3 and np.median(errs) < 5e-4, (errs.max(), np.median(errs))
    again, st2 = lens.find_images(src, **kw)
    assert again == imgs and st2["cells"] == st["cells"]
    lens.close()
