"""GPU parity: liblens (through its C ABI) against the FP64 oracle.

Bars: direct sum FP64 <= 1e-12 relative; direct sum FP32 <= 1e-5 in alpha,
kappa and gamma; tree median alpha error <= 1e-3 at theta = 0.3 and <= 1e-4
at theta = 0.1 (error metric in lens_testutil).  Kappa from the tree is exact
up to FP32 rounding for sized particles (only particles whose support covers
the ray carry surface density, Sec. 5.1 halo test).
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


def edge_mask(comps, rx, ry, rel=1e-6):
    """Rays within a relative 1e-6 of some component's support edge, where the
    FP32 and FP64 inside/outside decisions may legitimately differ (kappa
    jumps there by the truncated profile's edge value)."""
    m = np.zeros(rx.size, bool)
    sizes = np.where(comps["type"] == oracle.GAUSS, comps["p0"] * comps["p1"],
                     np.where(comps["type"] == oracle.NFW, comps["p1"],
                              np.where(comps["type"] == oracle.DISK, comps["p0"], 0.0)))
    sel = sizes > 0
    cx, cy, s = comps["x"][sel], comps["y"][sel], sizes[sel]
    for i in range(rx.size):
        r = np.hypot(rx[i] - cx, ry[i] - cy)
        m[i] = np.any(np.abs(r / s - 1.0) < rel)
    return m


# ----------------------------------------------------------- direct sums

def test_direct_fp64_point_disk():
    """2,000 equal point masses in the unit disk, 64 x 64 grid, FP64."""
    w = lensgen.workload_point_disk()
    p = w["points"]
    lens = L.Lens([L.Species.points(cu(p))], theta=0.1, precision="fp64")
    out = lens.shoot(cu(w["rx"]), cu(w["ry"]), flags=L.DIRECT)
    lens.sync()
    got = to_np(out)
    ref = oracle.direct_sum(comps_points(p), w["rx"], w["ry"])
    ea, ek, eg = rel_errors(got, ref)
    assert ea.max() <= 1e-12 and eg.max() <= 1e-12
    assert np.all(got[:, 2] == 0.0)


def mixed_lens_inputs(seed=5):
    g = lensgen.rng(seed)
    gauss = lensgen.nfw_particles(3000, seed, nsph=16)
    nfw = lensgen.nfw_halo_field(60, seed + 1, rs_at_1e4=0.03, box=0.8)
    pts = lensgen.point_disk(300, seed + 2, total_mass=0.05)
    halos = [L.Halo.sis(0.1, -0.05, 0.15), L.Halo.disk(-0.2, 0.1, -0.02, 0.3),
             L.Halo.gauss(0.3, 0.3, 0.01, 0.05, 3.0), L.Halo.nfw(-0.4, -0.3, 0.02, 0.05, 0.2),
             L.Halo.point(0.5, -0.5, 0.003)]
    comps = oracle.concat(
        comps_gauss(gauss, 3.0), comps_nfw(nfw, 3.0), comps_points(pts),
        oracle.make_components(oracle.SIS, 0.1, -0.05, 0.0, 0.15),
        oracle.make_components(oracle.DISK, -0.2, 0.1, -0.02, 0.3),
        oracle.make_components(oracle.GAUSS, 0.3, 0.3, 0.01, 0.05, 3.0),
        oracle.make_components(oracle.NFW, -0.4, -0.3, 0.02, 0.05, 0.2),
        oracle.make_components(oracle.POINT, 0.5, -0.5, 0.003))
    rx = g.uniform(-0.9, 0.9, 1024).astype(np.float32)
    ry = g.uniform(-0.9, 0.9, 1024).astype(np.float32)
    species = [L.Species.gauss(cu(gauss), 3.0), L.Species.nfw(cu(nfw), 3.0), L.Species.points(cu(pts))]
    return species, halos, comps, rx, ry


@pytest.mark.parametrize("group_rays", [32, 64])
def test_direct_fp32_mixed(group_rays):
    species, halos, comps, rx, ry = mixed_lens_inputs()
    lens = L.Lens(species, halos, theta=0.3, group_rays=group_rays)
    out = lens.shoot(cu(rx), cu(ry), flags=L.DIRECT)
    lens.sync()
    got = to_np(out)
    ref, absum = oracle.direct_sum(comps, rx.astype(np.float64), ry.astype(np.float64), with_absum=True)
    amb = edge_mask(comps, rx.astype(np.float64), ry.astype(np.float64))
    assert amb.sum() <= 0.01 * rx.size
    ok, frac_cond = within_fp32_bar(got, ref, absum)
    bad = np.where(~ok[~amb].all(axis=1))[0]
    assert bad.size == 0, (bad, rel_errors(got, ref)[2][~amb][bad])
    assert frac_cond <= 0.02


# ------------------------------------------------------------- tree mode

@pytest.mark.parametrize("theta,bar", [(0.3, 1e-3), (0.1, 1e-4)])
def test_tree_gauss_nfw_sph(theta, bar):
    """Smoothed NFW particles, r_sm = 32nd 3D neighbour, q = 3 (Sec. 3.1)."""
    parts = lensgen.nfw_particles(20000, 7, nsph=32)
    g = lensgen.rng(8)
    rx = g.uniform(-1, 1, 4096).astype(np.float32)
    ry = g.uniform(-1, 1, 4096).astype(np.float32)
    lens = L.Lens([L.Species.gauss(cu(parts), 3.0)], theta=theta)
    got = to_np(lens.shoot(cu(rx), cu(ry)))
    lens.sync()
    comps = comps_gauss(parts, 3.0)
    ref = oracle.direct_sum(comps, rx.astype(np.float64), ry.astype(np.float64))
    ea, ek, eg = rel_errors(got, ref)
    assert np.median(ea) <= bar, np.median(ea)
    assert np.median(eg) <= bar
    amb = edge_mask(comps, rx.astype(np.float64), ry.astype(np.float64))
    assert ek[~amb].max() <= 1e-5, ek[~amb].max()


def _counters(lens):
    c = lens.counters(reset=True)
    return [int(c[k]) for k in ("groups", "visited", "cells", "leaf_particles", "big_scanned", "big_kept",
                                "ray_interactions")]


@pytest.mark.parametrize("group_rays", [32, 64])
@pytest.mark.parametrize("case", ["gauss", "nfw_halo_ao", "points_fp64"])
def test_walk_pairs_matches_warp(case, group_rays):
    """The producer/consumer walks (one consumer, or two sharing a 64-ray
    group) and the one-warp walk with the large
    near-field tile visit the same boxes and keep the same entries as the
    one-warp walk with the standard tile (interaction counters equal), and
    their totals agree up to the order of summation; all meet the oracle's
    bar."""
    g = lensgen.rng(31)
    rx = g.uniform(-1, 1, 3000).astype(np.float64)
    ry = g.uniform(-1, 1, 3000).astype(np.float64)
    flags, prec, halos = 0, "fp32", []
    if case == "gauss":
        parts = lensgen.nfw_particles(20000, 7, nsph=32)
        species, comps = [L.Species.gauss(cu(parts), 3.0)], comps_gauss(parts, 3.0)
    elif case == "nfw_halo_ao":
        h = lensgen.nfw_test_halos(3000, 22, 0.3)
        species, comps = [L.Species.nfw(cu(h), 3.0)], comps_nfw(h, 3.0)
        halos = [L.Halo.sis(0.1, -0.2, 0.05)]
        comps = oracle.concat(comps, oracle.make_components(oracle.SIS, 0.1, -0.2, 0, 0.05))
        flags = L.ALPHA_ONLY
    else:
        p = lensgen.point_disk(5000, 33)
        species, comps, prec = [L.Species.points(cu(p))], comps_points(p), "fp64"
    dtype = np.float64 if prec == "fp64" else np.float32
    dx, dy = cu(rx.astype(dtype)), cu(ry.astype(dtype))
    res, cnt = {}, {}
    ncomp = 2 if flags & L.ALPHA_ONLY else 5
    for form, walk, tile in (("warp", "warp", "standard"), ("pairs", "pairs", "standard"),
                             ("trios", "trios", "standard"), ("large", "warp", "large")):
        lens = L.Lens(species, halos, theta=0.3, precision=prec, group_rays=group_rays, walk=walk, tile=tile)
        assert lens.info()["tile"] == (tile if prec == "fp32" else "standard")
        out = lens.shoot(dx, dy, flags=flags | L.COUNT)
        res[form] = np.stack([o.double().cpu().numpy() for o in out[:ncomp]], axis=1)
        lens.sync()
        cnt[form] = _counters(lens)
        lens.close()
    assert cnt["warp"] == cnt["pairs"] == cnt["trios"] == cnt["large"], cnt
    ref, absum = oracle.direct_sum(comps, rx, ry, with_absum=True)
    a = res["warp"]
    for form in ("pairs", "trios", "large"):
        b = res[form]
        # same terms, summed in another order: a few roundings of the sum of |terms|
        eps = 1e-14 if prec == "fp64" else 1e-6
        d = np.abs(a - b) / (absum[:, :ncomp] + 1e-300)
        assert d.max() <= eps, (form, d.max(axis=0))
        ea, _, _ = rel_errors(b, ref) if ncomp == 5 else rel_errors(np.c_[b, ref[:, 2:]], ref)
        assert np.median(ea) <= 1e-3


@pytest.mark.parametrize("case", ["gauss", "points_origin"])
def test_tree_128_ray_groups(case):
    """128-ray groups (four rays per lane, the one-warp FP32 tree walk):
    within the tree's bar of the oracle, kappa of a Gaussian lens exact away
    from support edges; the calls that group at most 64 rays (direct sum,
    potential) give the 64-ray lens's bits."""
    g = lensgen.rng(41)
    origin = (0.0, 0.0)
    if case == "gauss":
        parts = lensgen.nfw_particles(20000, 7, nsph=32)
        species, comps = [L.Species.gauss(cu(parts), 3.0)], comps_gauss(parts, 3.0)
        halos = []
    else:
        # FP64 origin with FP32 offsets: the FP64-anchored grouping path
        p = lensgen.point_disk(5000, 43)
        species, comps = [L.Species.points(cu(p))], comps_points(p)
        halos = [L.Halo.sis(0.05, -0.02, 0.3)]
        comps = oracle.concat(comps, oracle.make_components(oracle.SIS, 0.05, -0.02, 0, 0.3))
        origin = (0.25, -0.125)
    dx = g.uniform(-0.6, 0.6, 5000).astype(np.float32)
    dy = g.uniform(-0.6, 0.6, 5000).astype(np.float32)
    rx, ry = origin[0] + dx.astype(np.float64), origin[1] + dy.astype(np.float64)
    lens = L.Lens(species, halos, theta=0.3, group_rays=128, walk="warp")
    assert lens.info()["group_rays"] == 128
    got = to_np(lens.shoot(cu(dx), cu(dy), origin=origin))
    lens.sync()
    ref = oracle.direct_sum(comps, rx, ry)
    ea, ek, eg = rel_errors(got, ref)
    assert np.median(ea) <= 1e-3 and np.median(eg) <= 1e-3, (np.median(ea), np.median(eg))
    if case == "gauss":
        amb = edge_mask(comps, rx, ry)
        assert ek[~amb].max() <= 1e-5, ek[~amb].max()
        # alpha only (the big entries of each half of a group, packed general
        # form where a ray may be inside a softening radius)
        ao = to_np(lens.shoot(cu(dx), cu(dy), origin=origin, flags=L.ALPHA_ONLY)[:2])
        lens.sync()
        ea_ao = rel_errors(np.concatenate([ao[:, :2], ref[:, 2:]], axis=1), ref)[0]
        assert np.median(ea_ao) <= 1e-3, np.median(ea_ao)
        assert np.max(np.abs(ao[:, :2] - got[:, :2])) <= 1e-5 * np.max(np.abs(got[:, :2]))
    l64 = L.Lens(species, halos, theta=0.3, group_rays=64, walk="warp")
    for a, b in zip(lens.shoot(cu(dx), cu(dy), origin=origin, flags=L.DIRECT),
                    l64.shoot(cu(dx), cu(dy), origin=origin, flags=L.DIRECT)):
        assert torch.equal(a, b)
    for a, b in zip(lens.potential(cu(dx), cu(dy), origin=origin), l64.potential(cu(dx), cu(dy), origin=origin)):
        assert torch.equal(a, b)
    lens.close()
    l64.close()


def test_page_locked_host_outputs():
    """Outputs in page-locked host memory receive the same bits as device
    outputs (shoot, potential, batches); other host memory is refused."""
    parts = lensgen.nfw_particles(5000, 51, nsph=32)
    g = lensgen.rng(52)
    dx = cu(g.uniform(-0.5, 0.5, 3000).astype(np.float32))
    dy = cu(g.uniform(-0.5, 0.5, 3000).astype(np.float32))
    lens = L.Lens([L.Species.gauss(cu(parts), 3.0)], theta=0.3)
    host = [torch.empty(3000, dtype=torch.float32).pin_memory() for _ in range(5)]
    ref = lens.shoot(dx, dy)
    lens.shoot(dx, dy, out=host)
    lens.sync()
    for a, b in zip(ref, host):
        assert torch.equal(a.cpu(), b)
    pref = lens.potential(dx, dy)
    lens.potential(dx, dy, out=host[:3])
    lens.sync()
    for a, b in zip(pref, host[:3]):
        assert torch.equal(a.cpu(), b)
    offs = np.array([0, 1000, 3000], np.int64)
    bref = lens.shoot_batches(offs, np.zeros((2, 2)), dx, dy)
    lens.shoot_batches(offs, np.zeros((2, 2)), dx, dy, out=host)
    lens.sync()
    for a, b in zip(bref, host):
        assert torch.equal(a.cpu(), b)
    with pytest.raises(ValueError):
        lens.shoot(dx, dy, out=[torch.empty(3000, dtype=torch.float32) for _ in range(5)])
    lens.close()


def test_tree_used_on_another_stream():
    """Shoot, potential and adjoint calls issued on a second stream right
    after a build, with no host synchronisation, wait for the build on the
    device: the same results as the same calls made once the build has
    completed (the forward bit for bit; the adjoint, which sums in FP64
    atomics, to FP64 rounding)."""
    parts = cu(lensgen.nfw_particles(200000, 61, nsph=32))
    g = lensgen.rng(62)
    n = 1 << 16
    dx = cu(g.uniform(-0.5, 0.5, n).astype(np.float32))
    dy = cu(g.uniform(-0.5, 0.5, n).astype(np.float32))
    ga = [cu(g.normal(size=n).astype(np.float32)) for _ in range(2)]
    a, b = torch.cuda.Stream(), torch.cuda.Stream()
    outs = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(5)]
    pots = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    grad = torch.zeros(parts.shape[0], 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    for rep in range(2):
        with torch.cuda.stream(a):
            lens = L.Lens([L.Species.gauss(parts, 3.0)], theta=0.3)
        if rep == 0:
            lens.shoot(dx, dy, out=outs, stream=b)
            lens.potential(dx, dy, out=pots, stream=b)
        else:
            lens.backward(dx, dy, ga[0], ga[1], grads=[grad], stream=b)
        torch.cuda.synchronize()
        if rep == 0:
            ref = lens.shoot(dx, dy)
            pref = lens.potential(dx, dy)
            lens.sync()
            for x, y in zip(ref, outs):
                assert torch.equal(x, y)
            for x, y in zip(pref, pots):
                assert torch.equal(x, y)
        else:
            gref = torch.zeros_like(grad)
            lens.backward(dx, dy, ga[0], ga[1], grads=[gref])
            lens.sync()
            gr, gg = gref.double().cpu().numpy(), grad.double().cpu().numpy()
            scale = np.abs(gr).max(axis=0) + 1e-30
            assert np.max(np.abs(gg - gr) / scale) < 1e-5
        lens.close()


def test_tree_points_fp64_theta01():
    w = lensgen.workload_point_disk()
    p = w["points"]
    lens = L.Lens([L.Species.points(cu(p))], theta=0.1, precision="fp64")
    got = to_np(lens.shoot(cu(w["rx"]), cu(w["ry"])))
    lens.sync()
    ref = oracle.direct_sum(comps_points(p), w["rx"], w["ry"])
    ea, _, eg = rel_errors(got, ref)
    assert np.median(ea) <= 1e-4 and np.median(eg) <= 1e-4
    assert np.all(got[:, 2] == 0.0)


@pytest.mark.parametrize("theta", [0.3, 0.55, 0.8])
def test_tree_halo_kappa_exact(theta):
    """Sec. 5.1 halo test: NFW halos, sizes uniform up to 0.3, c = 3: kappa
    from the tree equals the direct sum at any opening angle."""
    h = lensgen.nfw_test_halos(1000, 21, 0.3)
    g = lensgen.rng(22)
    rx = g.uniform(-1, 1, 1024).astype(np.float32)
    ry = g.uniform(-1, 1, 1024).astype(np.float32)
    lens = L.Lens([L.Species.nfw(cu(h), 3.0)], theta=theta)
    got = to_np(lens.shoot(cu(rx), cu(ry)))
    lens.sync()
    comps = comps_nfw(h, 3.0)
    ref = oracle.direct_sum(comps, rx.astype(np.float64), ry.astype(np.float64))
    amb = edge_mask(comps, rx.astype(np.float64), ry.astype(np.float64))
    _, ek, _ = rel_errors(got, ref)
    assert ek[~amb].max() <= 1e-5, ek[~amb].max()


def test_microlensing_patch_fp64_offsets():
    """Stars in the unit disk + SIS, rays on a 1e-6-wide patch at (0.5, 0):
    FP64 origin + FP32 offsets keep the patch resolved."""
    w = lensgen.workload_microlensing(n_stars=100_000, n_grid=32)
    p = w["points"]
    lens = L.Lens([L.Species.points(cu(p))], [L.Halo.sis(0.0, 0.0, w["sis_re"])], theta=0.1)
    got = to_np(lens.shoot(cu(w["dx"]), cu(w["dy"]), origin=w["origin"]))
    lens.sync()
    comps = oracle.concat(comps_points(p), oracle.make_components(oracle.SIS, 0, 0, 0, w["sis_re"]))
    rx = w["origin"][0] + w["dx"].astype(np.float64)
    ry = w["origin"][1] + w["dy"].astype(np.float64)
    ref = oracle.direct_sum(comps, rx, ry)
    ea, _, eg = rel_errors(got, ref)
    assert np.median(ea) <= 1e-4 and np.median(eg) <= 1e-4
    # across the patch the shear changes by ~1e-3 of itself; FP32 absolute
    # coordinates (ulp(0.5) ~ 6e-8) would step it in ~17 levels.  The direct
    # sum must follow the oracle ray by ray to 1e-3 of that variation.
    dirc = to_np(lens.shoot(cu(w["dx"]), cu(w["dy"]), origin=w["origin"], flags=L.DIRECT))
    lens.sync()
    for q in (3, 4):
        assert np.abs(dirc[:, q] - ref[:, q]).max() <= 1e-3 * np.ptp(ref[:, q])


def test_batches_and_graph_replay():
    """Uneven refinement batches in one launch, eager and graph-replayed."""
    w = lensgen.workload_mixed_batches(n_halos=100, n_stars=20000, n_batches=12, nmin=50, nmax=3000)
    lens = L.Lens([L.Species.points(cu(w["points"])), L.Species.nfw(cu(w["nfw"]), 3.0)], theta=0.3)
    dx, dy = cu(w["dx"]), cu(w["dy"])
    lib = L.lib()
    k0 = lib.lens_kernel_launches()
    eager = to_np(lens.shoot_batches(w["offsets"], w["origins"], dx, dy))
    per_call = lib.lens_kernel_launches() - k0
    assert per_call > 0
    outs = [torch.empty(dx.numel(), device="cuda") for _ in range(5)]
    for it in range(3):
        for o in outs:
            o.fill_(float("nan"))
        k0 = lib.lens_kernel_launches()
        lens.shoot_batches(w["offsets"], w["origins"], dx, dy, flags=L.USE_GRAPH, out=outs)
        lens.sync()
        # the first call runs eagerly and captures; a replay counts the graph's kernels
        assert lib.lens_kernel_launches() - k0 == per_call, it
        np.testing.assert_array_equal(to_np(outs), eager)
    comps = oracle.concat(comps_points(w["points"]), comps_nfw(w["nfw"], 3.0))
    b = np.repeat(np.arange(len(w["offsets"]) - 1), np.diff(w["offsets"]))
    rx = w["origins"][b, 0] + w["dx"].astype(np.float64)
    ry = w["origins"][b, 1] + w["dy"].astype(np.float64)
    sel = np.arange(0, rx.size, max(1, rx.size // 3000))
    ref = oracle.direct_sum(comps, rx[sel], ry[sel])
    ea, _, _ = rel_errors(eager[sel], ref)
    assert np.median(ea) <= 1e-3


# --------------------------------------------------- edge cases and flags

def test_empty_ragged_and_flags():
    parts = lensgen.nfw_particles(2000, 31, nsph=16)
    lens = L.Lens([L.Species.gauss(cu(parts), 3.0), L.Species.points(cu(np.zeros((0, 4), np.float32)))],
                  [L.Halo.sis(0.0, 0.0, 0.1)], theta=0.3)
    # n = 0 is a no-op
    e = torch.empty(0, device="cuda")
    lens.shoot(e, e)
    g = lensgen.rng(32)
    for n in [1, 31, 33, 65, 1000]:
        rx = g.uniform(-0.5, 0.5, n).astype(np.float32)
        ry = g.uniform(-0.5, 0.5, n).astype(np.float32)
        full = to_np(lens.shoot(cu(rx), cu(ry)))
        ao = lens.shoot(cu(rx), cu(ry), flags=L.ALPHA_ONLY)
        np.testing.assert_allclose(to_np(ao[:2]), full[:, :2], rtol=1e-6, atol=1e-7)
        acc = [cu(np.ones(n, np.float32)) for _ in range(5)]
        lens.shoot(cu(rx), cu(ry), flags=L.ACCUMULATE, out=acc)
        np.testing.assert_allclose(to_np(acc), full + 1.0, rtol=1e-6, atol=1e-6)
    lens.sync()
    # halos only
    only = L.Lens([], [L.Halo.sis(0.0, 0.0, 0.5)], theta=0.3)
    o = to_np(only.shoot(cu(np.array([0.3], np.float32)), cu(np.array([0.4], np.float32))))
    np.testing.assert_allclose(o[0, :2], [0.3, 0.4], rtol=1e-6)   # r_E * x / |x| with |x| = 0.5
    assert o[0, 2] == pytest.approx(0.5, rel=1e-6)                 # r_E / (2 r)


def test_invalid_inputs_are_rejected():
    bad = np.array([[0.0, 0.0, -1.0, 0.1]], np.float32)
    with pytest.raises(L.LensError):
        L.Lens([L.Species.gauss(cu(bad), 3.0)])
    with pytest.raises(L.LensError):
        L.Lens([], theta=-1.0)


@pytest.mark.parametrize("walk", ["warp", "pairs", "trios"])
def test_forward_is_bitwise_deterministic(walk):
    """Each ray's sum is taken by one warp in a fixed order whatever warp takes
    its group (the work counter only changes who): repeated shots and a fresh
    lens give the same bits, for both walk forms; the potential likewise."""
    parts = lensgen.nfw_particles(50000, 17, nsph=32)
    g = lensgen.rng(18)
    rx = cu(g.uniform(-1, 1, 200_000).astype(np.float32))
    ry = cu(g.uniform(-1, 1, 200_000).astype(np.float32))
    first = None
    for rep in range(3):
        lens = L.Lens([L.Species.gauss(cu(parts), 3.0)], theta=0.3, group_rays=64, walk=walk)
        for _ in range(2):
            out = [o.clone() for o in lens.shoot(rx, ry)]
            psi = lens.potential(rx, ry)[0].clone()
            if first is None:
                first = (out, psi)
            else:
                for a, b in zip(out, first[0]):
                    assert torch.equal(a, b)
                assert torch.equal(psi, first[1])
        lens.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_halos_only_per_ray_path(prec):
    """A lens of analytic components only is shot one thread per ray (no
    grouping, no walk): all five halo kinds against the oracle's direct sum,
    FP32 and FP64 ray offsets about an FP64 origin, ALPHA_ONLY and ACCUMULATE,
    and the same values as the grouped path (taken with TIMING)."""
    halos = [L.Halo.sis(0.1, -0.05, 0.15), L.Halo.disk(-0.2, 0.1, -0.02, 0.3),
             L.Halo.gauss(0.3, 0.3, 0.01, 0.05, 3.0), L.Halo.nfw(-0.4, -0.3, 0.02, 0.05, 0.2),
             L.Halo.point(0.5, -0.5, 0.003)]
    comps = oracle.concat(
        oracle.make_components(oracle.SIS, 0.1, -0.05, 0.0, 0.15),
        oracle.make_components(oracle.DISK, -0.2, 0.1, -0.02, 0.3),
        oracle.make_components(oracle.GAUSS, 0.3, 0.3, 0.01, 0.05, 3.0),
        oracle.make_components(oracle.NFW, -0.4, -0.3, 0.02, 0.05, 0.2),
        oracle.make_components(oracle.POINT, 0.5, -0.5, 0.003))
    lens = L.Lens([], halos, theta=0.3, precision=prec)
    g = lensgen.rng(71)
    origin = (0.25, -0.125)
    dx = g.uniform(-0.9, 0.9, 30000)
    dy = g.uniform(-0.9, 0.9, 30000)
    ref = oracle.direct_sum(comps, origin[0] + dx, origin[1] + dy)
    for rdt in (np.float64, np.float32):
        rx, ry = cu(dx.astype(rdt)), cu(dy.astype(rdt))
        got = to_np(lens.shoot(rx, ry, origin=origin))
        rr = oracle.direct_sum(comps, origin[0] + dx.astype(rdt).astype(np.float64),
                               origin[1] + dy.astype(rdt).astype(np.float64))
        mask = ~edge_mask(comps, origin[0] + dx.astype(rdt), origin[1] + dy.astype(rdt))
        # the halos' kappa and gamma cancel at some rays (a negative-mass
        # disk among them): bars on the conditioning, sum |term|
        _, absum = oracle.direct_sum(comps, origin[0] + dx.astype(rdt).astype(np.float64),
                                     origin[1] + dy.astype(rdt).astype(np.float64), with_absum=True)
        if prec == "fp64":
            d = np.abs(got - rr)
            ok = d <= 1e-12 * np.abs(rr) + 64 * 2.0 ** -53 * absum
            bad = np.nonzero(~ok.all(axis=1) & mask)[0]
            assert ok[:, :2].all() and bad.size == 0, [
                (origin[0] + dx[b], origin[1] + dy[b], got[b].tolist(), rr[b].tolist(), absum[b].tolist())
                for b in bad[:3]]
        else:
            ok, _ = within_fp32_bar(got, rr, absum)
            assert ok[:, 0].all() and ok[mask].all(), (rdt, (~ok[mask]).sum(axis=0))
        grouped = to_np(lens.shoot(rx, ry, origin=origin, flags=L.TIMING))
        np.testing.assert_allclose(got, grouped, rtol=1e-12 if prec == "fp64" else 1e-5,
                                   atol=1e-14 if prec == "fp64" else 1e-6)
        ao = lens.shoot(rx, ry, origin=origin, flags=L.ALPHA_ONLY)
        np.testing.assert_array_equal(to_np(ao[:2]), got[:, :2])
        dt = torch.float64 if prec == "fp64" else torch.float32
        acc = [torch.full((dx.size,), 2.0, dtype=dt, device="cuda") for _ in range(5)]
        lens.shoot(rx, ry, origin=origin, flags=L.ACCUMULATE, out=acc)
        np.testing.assert_allclose(to_np(acc), got + 2.0, rtol=1e-12 if prec == "fp64" else 1e-6, atol=1e-6)
    assert ref.shape[0] == dx.size
    lens.close()
