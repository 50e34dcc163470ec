"""GPU lensing potential (lens_shoot_potential; Eq. alpha, Eq. timedelay)
against the oracle's direct potential on the same inputs.

Bars: FP64 direct sum 1e-12 of sum |term|; FP32 direct sum within 8 FP32
roundings of sum |term| (the conditioning form used for the other outputs);
the tree's psi within 1e-3 (theta = 0.3) / 1e-4 (theta = 0.1) of |psi| at
the median ray, the bars of the deflection; the potential call's deflection
equals shoot()'s.
"""
import numpy as np
import pytest

import lensgen
import oracle
from lens_testutil import comps_gauss, comps_nfw, comps_points

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1312_1128_gb300 as L  # noqa: E402

EPS32 = 2.0 ** -24


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def halo_list():
    return ([L.Halo.sis(0.05, -0.1, 0.2), L.Halo.disk(-0.3, 0.2, 0.05, 0.3), L.Halo.nfw(0.4, 0.4, 0.02, 0.05, 0.2),
             L.Halo.gauss(-0.2, -0.5, 0.01, 0.04, 3.0), L.Halo.point(0.7, -0.6, 1e-3)],
            oracle.concat(oracle.make_components(oracle.SIS, 0.05, -0.1, 0.0, 0.2),
                          oracle.make_components(oracle.DISK, -0.3, 0.2, 0.05, 0.3),
                          oracle.make_components(oracle.NFW, 0.4, 0.4, 0.02, 0.05, 0.2),
                          oracle.make_components(oracle.GAUSS, -0.2, -0.5, 0.01, 0.04, 3.0),
                          oracle.make_components(oracle.POINT, 0.7, -0.6, 1e-3)))


def test_direct_fp64_points():
    w = lensgen.workload_point_disk()
    p = w["points"].astype(np.float64)
    lens = L.Lens([L.Species.points(cu(p))], theta=0.1, precision="fp64")
    psi, a1, a2 = lens.potential(cu(w["rx"]), cu(w["ry"]), flags=L.DIRECT)
    ref, ab = oracle.direct_potential(comps_points(p), w["rx"], w["ry"], with_absum=True)
    got = psi.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-12 * ab)
    s = lens.shoot(cu(w["rx"]), cu(w["ry"]), flags=L.DIRECT)
    np.testing.assert_allclose(a1.cpu().numpy(), s[0].cpu().numpy(), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(a2.cpu().numpy(), s[1].cpu().numpy(), rtol=1e-12, atol=1e-14)
    lens.close()


def test_direct_fp32_mixed_species_and_halos():
    g = lensgen.rng(61)
    gp = lensgen.nfw_particles(3000, 62, nsph=16)
    nfw = lensgen.nfw_test_halos(300, 63, 0.2)
    pts = lensgen.point_disk(2000, 64, total_mass=0.1)
    hl, hc = halo_list()
    lens = L.Lens([L.Species.gauss(cu(gp), 3.0), L.Species.nfw(cu(nfw), 3.0), L.Species.points(cu(pts))], hl,
                  theta=0.3)
    rx = g.uniform(-1, 1, 2048).astype(np.float32)
    ry = g.uniform(-1, 1, 2048).astype(np.float32)
    psi, a1, a2 = lens.potential(cu(rx), cu(ry), flags=L.DIRECT)
    comps = oracle.concat(comps_gauss(gp, 3.0), comps_nfw(nfw, 3.0), comps_points(pts), hc)
    ref, ab = oracle.direct_potential(comps, rx.astype(np.float64), ry.astype(np.float64), with_absum=True)
    d = np.abs(psi.cpu().numpy().astype(np.float64) - ref)
    assert np.all(d <= 8 * EPS32 * ab + 1e-7 * np.abs(ref)), (d / ab).max()
    lens.close()


@pytest.mark.parametrize("theta,bar", [(0.3, 1e-3), (0.1, 1e-4)])
def test_tree_gauss_nfw_sph(theta, bar):
    parts = lensgen.nfw_particles(20000, 7, nsph=32)
    g = lensgen.rng(8)
    rx = g.uniform(-1, 1, 4096).astype(np.float32)
    ry = g.uniform(-1, 1, 4096).astype(np.float32)
    for gr in (32, 64):
        lens = L.Lens([L.Species.gauss(cu(parts), 3.0)], theta=theta, group_rays=gr)
        psi, a1, a2 = lens.potential(cu(rx), cu(ry))
        ref = oracle.direct_potential(comps_gauss(parts, 3.0), rx.astype(np.float64), ry.astype(np.float64))
        e = np.abs(psi.cpu().numpy() - ref) / np.abs(ref)
        assert np.median(e) <= bar, (gr, np.median(e))
        s = lens.shoot(cu(rx), cu(ry))
        # same tree, same terms up to the order of summation
        np.testing.assert_allclose(a1.cpu().numpy(), s[0].cpu().numpy(), rtol=1e-4,
                                   atol=1e-5 * float(np.abs(s[0].cpu().numpy()).max()))
        lens.close()


def test_tree_fp64_points_and_halos_only():
    w = lensgen.workload_point_disk()
    p = w["points"].astype(np.float64)
    hl, hc = halo_list()
    lens = L.Lens([L.Species.points(cu(p))], hl, theta=0.1, precision="fp64")
    psi, _, _ = lens.potential(cu(w["rx"]), cu(w["ry"]))
    ref = oracle.direct_potential(oracle.concat(comps_points(p), hc), w["rx"], w["ry"])
    e = np.abs(psi.cpu().numpy() - ref) / np.abs(ref)
    assert np.median(e) <= 1e-5
    lens.close()
    h_only = L.Lens([], hl, theta=0.3)
    g = lensgen.rng(65)
    rx, ry = g.uniform(-1, 1, 500).astype(np.float32), g.uniform(-1, 1, 500).astype(np.float32)
    psi, a1, _ = h_only.potential(cu(rx), cu(ry))
    ref, ab = oracle.direct_potential(hc, rx.astype(np.float64), ry.astype(np.float64), with_absum=True)
    assert np.all(np.abs(psi.cpu().numpy() - ref) <= 8 * EPS32 * ab + 1e-7)
    assert np.isfinite(a1.cpu().numpy()).all()
    h_only.close()


def test_potential_edges():
    lens = L.Lens([L.Species.points(cu(lensgen.point_disk(100, 66)))], theta=0.3)
    e = torch.zeros(0, device="cuda")
    lens.potential(e, e)
    x = torch.zeros(8, device="cuda")
    with pytest.raises(L.LensError):
        lens.potential(x, x, flags=L.ALPHA_ONLY)
    psi, a1, a2 = lens.potential(x, x, out=[torch.empty(8, device="cuda"), None, None])
    assert a1 is None and torch.isfinite(psi).all()
    lens.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_direct_gauss_q5_both_ein_branches(prec):
    """q = 5 puts u = r^2 / (2 sigma^2) up to 12.5: both the series (u < 5)
    and the continued fraction (u >= 5) of Ein are taken."""
    gp = lensgen.nfw_particles(1500, 67, fixed_sigma=0.03)
    g = lensgen.rng(68)
    rx = g.uniform(-0.5, 0.5, 1024)
    ry = g.uniform(-0.5, 0.5, 1024)
    dt = np.float64 if prec == "fp64" else np.float32
    lens = L.Lens([L.Species.gauss(cu(gp.astype(dt)), 5.0)], theta=0.3, precision=prec)
    psi, _, _ = lens.potential(cu(rx.astype(dt)), cu(ry.astype(dt)), flags=L.DIRECT)
    ref, ab = oracle.direct_potential(comps_gauss(gp, 5.0), rx.astype(dt).astype(np.float64),
                                      ry.astype(dt).astype(np.float64), with_absum=True)
    d = np.abs(psi.cpu().numpy().astype(np.float64) - ref)
    bar = 1e-12 * ab if prec == "fp64" else 8 * EPS32 * ab + 1e-7 * np.abs(ref)
    assert np.all(d <= bar), (d / ab).max()
    lens.close()


def test_potential_timing_and_counters():
    """LENS_TIMING and LENS_COUNT on the potential walk: positive times, and
    the same interaction counts as the deflection walk over the same tree."""
    parts = lensgen.nfw_particles(20000, 7, nsph=32)
    g = lensgen.rng(9)
    rx = cu(g.uniform(-1, 1, 8192).astype(np.float32))
    ry = cu(g.uniform(-1, 1, 8192).astype(np.float32))
    lens = L.Lens([L.Species.gauss(cu(parts), 3.0)], theta=0.3, group_rays=32, walk="warp")
    lens.potential(rx, ry, flags=L.TIMING | L.COUNT)
    gm, wm = lens.last_timing()
    assert gm > 0 and wm > 0
    c_psi = lens.counters()
    lens.shoot(rx, ry, flags=L.COUNT)
    lens.sync()
    c_fwd = lens.counters()
    for k in ("groups", "visited", "cells", "leaf_particles", "big_kept", "ray_interactions"):
        assert c_psi[k] == c_fwd[k], k
    lens.close()


@pytest.mark.parametrize("q", [3.0, 3.1, 3.5])
def test_tree_ein_branches(q):
    """The packed big-list potential takes Ein by the degree-9 polynomial for
    q <= 3 (U_q <= 4.5), by the 20-term series up to U_q = 5, and the generic
    per-entry form beyond: each against the oracle's direct potential at the
    theta = 0.1 bar."""
    parts = lensgen.nfw_particles(20000, 7, nsph=32)
    g = lensgen.rng(81)
    rx = g.uniform(-1, 1, 4096).astype(np.float32)
    ry = g.uniform(-1, 1, 4096).astype(np.float32)
    lens = L.Lens([L.Species.gauss(cu(parts), q)], theta=0.1, group_rays=64)
    psi, _, _ = lens.potential(cu(rx), cu(ry))
    ref = oracle.direct_potential(comps_gauss(parts, q), rx.astype(np.float64), ry.astype(np.float64))
    e = np.abs(psi.cpu().numpy() - ref) / np.abs(ref)
    assert np.median(e) <= 1e-4 and np.quantile(e, 0.99) <= 1e-3, (q, np.median(e), np.quantile(e, 0.99))
    lens.close()
