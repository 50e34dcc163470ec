"""The allocation-free entry point, through the C ABI.

lens_shoot_rays_direct_noalloc is for callers that cannot allocate device
memory while they shoot rays: code running while another component owns the
device allocator, latency-bound loops that cannot absorb the device-wide
synchronisation a cudaMalloc may bring, and deployments with a fixed device
budget reserved up front.  Its scratch is a fixed device array inside the
library.  Checked against the FP64 oracle's direct sum (the FP32 bar, or
1e-12 for an FP64 tree) and against the allocating direct sum, on calls in a
row (the shared array keeps the previous call's contents): FP32 and FP64
trees, FP32 and FP64 ray offsets from a non-zero origin (groups whose rays
are not exact in the working precision take a non-zero anchor), a lens of
analytic halos only, LENS_ALPHA_ONLY and LENS_ACCUMULATE; device free memory
is unchanged across a call; more than 262,144 rays is rejected.
Collected last, so that a run stopping at the first failure has run every
other test before it.
"""
import ctypes

import numpy as np
import pytest

import lensgen
import oracle
from lens_testutil import comps_gauss, comps_points, to_np, within_fp32_bar

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1312_1128_gb300 as L  # noqa: E402

MAX_RAYS = 262144


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def outputs(n, dtype=torch.float32):
    return [torch.full((n,), float("nan"), dtype=dtype, device="cuda") for _ in range(5)]


def coherent_rays(g, n, dtype):
    """n uniform rays in [-0.9, 0.9]^2 in Morton order: the entry point groups
    rays 32 at a time in their input order, so callers give them in a
    spatially coherent order (a group's FP32 offsets from its anchor then
    round within a small extent)."""
    from paper_1312_1128_gb300 import shard
    x, y = g.uniform(-0.9, 0.9, n), g.uniform(-0.9, 0.9, n)
    o = np.argsort(shard.morton_keys(x, y), kind="stable")
    return x[o].astype(dtype), y[o].astype(dtype)


def mixed_lens(precision="fp32", halos_only=False):
    gauss = lensgen.nfw_particles(4000, 41, nsph=16)
    pts = lensgen.point_disk(500, 42, total_mass=0.05)
    halos = [L.Halo.sis(0.05, 0.0, 0.2), L.Halo.disk(0.1, -0.1, -0.01, 0.4)]
    hcomps = [oracle.make_components(oracle.SIS, 0.05, 0.0, 0.0, 0.2),
              oracle.make_components(oracle.DISK, 0.1, -0.1, -0.01, 0.4)]
    if halos_only:
        return L.Lens([], halos, theta=0.3, precision=precision), oracle.concat(*hcomps)
    dt = np.float64 if precision == "fp64" else np.float32
    lens = L.Lens([L.Species.gauss(cu(gauss.astype(dt)), 3.0), L.Species.points(cu(pts.astype(dt)))], halos,
                  theta=0.3, precision=precision)
    return lens, oracle.concat(comps_gauss(gauss, 3.0), comps_points(pts), *hcomps)


def check_against_oracle(got, comps, x, y, fp64, alpha_only=False):
    sel = np.arange(0, x.size, 7)
    ref, absum = oracle.direct_sum(comps, x[sel], y[sel], with_absum=True)
    g = got[sel]
    if fp64:
        # FP64 terms with compensated totals: within 1e-12 of sum |term|
        cols = [0, 1] if alpha_only else list(range(5))
        assert np.all(np.abs(g - ref)[:, cols] <= 1e-12 * absum[:, cols])
    else:
        if alpha_only:
            g = g.copy()
            g[:, 2:] = ref[:, 2:]
        ok, frac = within_fp32_bar(g, ref, absum)
        assert ok.all(), np.where(~ok.all(axis=1))[0][:5]
        assert frac <= 0.02


@pytest.mark.parametrize("precision,ray_dtype,origin", [("fp32", np.float32, (0.0, 0.0)),
                                                         ("fp32", np.float64, (0.3, 0.2)),
                                                         ("fp64", np.float64, (0.3, 0.2)),
                                                         ("fp64", np.float32, (0.0, 0.0))])
def test_noalloc_matches_oracle_on_consecutive_calls(precision, ray_dtype, origin):
    lens, comps = mixed_lens(precision)
    odt = lens.out_dtype
    g = lensgen.rng(43)
    for call, n in enumerate([5001, 20000]):
        rx, ry = coherent_rays(g, n, ray_dtype)
        dx, dy = cu(rx), cu(ry)
        got = to_np(lens.shoot_direct_noalloc(dx, dy, outputs(n, odt), origin=origin))
        ref = to_np(lens.shoot(dx, dy, origin=origin, flags=L.DIRECT))
        lens.sync()
        assert np.all(np.isfinite(got)), call
        x = origin[0] + rx.astype(np.float64)
        y = origin[1] + ry.astype(np.float64)
        check_against_oracle(got, comps, x, y, precision == "fp64")
        # the allocating direct sum groups the rays in another order: the
        # same terms, summed differently
        if precision == "fp64":
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14)
    lens.close()


def test_noalloc_halos_only_alpha_only_and_accumulate():
    lens, comps = mixed_lens("fp32", halos_only=True)
    g = lensgen.rng(45)
    n = 7000
    rx, ry = coherent_rays(g, n, np.float32)
    dx, dy = cu(rx), cu(ry)
    x, y = rx.astype(np.float64), ry.astype(np.float64)
    got = to_np(lens.shoot_direct_noalloc(dx, dy, outputs(n)))
    lens.sync()
    check_against_oracle(got, comps, x, y, False)
    out = outputs(n)
    a = lens.shoot_direct_noalloc(dx, dy, out[:2] + [None] * 3, flags=L.ALPHA_ONLY)
    lens.sync()
    assert torch.isnan(out[2]).all()                # kappa untouched with ALPHA_ONLY
    np.testing.assert_allclose(to_np(a[:2]), got[:, :2], rtol=1e-6, atol=1e-7)
    acc = [torch.ones(n, device="cuda") for _ in range(5)]
    lens.shoot_direct_noalloc(dx, dy, acc, flags=L.ACCUMULATE)
    lens.sync()
    np.testing.assert_allclose(to_np(acc), got + 1.0, rtol=1e-6, atol=1e-6)
    lens.close()


def test_noalloc_allocates_nothing():
    """Free device memory is the same before and after a call (after a
    first call on the tree, and with the caller's buffers made beforehand)."""
    lens, _ = mixed_lens("fp32")
    n = 100000
    g = lensgen.rng(46)
    dx = cu(g.uniform(-0.9, 0.9, n).astype(np.float32))
    dy = cu(g.uniform(-0.9, 0.9, n).astype(np.float32))
    out = outputs(n)
    lens.shoot_direct_noalloc(dx, dy, out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        lens.shoot_direct_noalloc(dx, dy, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    lens.close()


def test_noalloc_rejects_too_many_rays():
    pts = lensgen.point_disk(100, 44)
    lens = L.Lens([L.Species.points(cu(pts))], theta=0.3)
    n = MAX_RAYS + 1
    dx = torch.zeros(n, device="cuda")
    out = outputs(n)
    lt = L.lib()
    st = lt.lens_shoot_rays_direct_noalloc(
        lens._h, 0.0, 0.0, ctypes.c_void_p(dx.data_ptr()), ctypes.c_void_p(dx.data_ptr()), 0, n,
        *[ctypes.c_void_p(o.data_ptr()) for o in out], 0, None)
    assert st == 1
    assert b"262144" in lt.lens_last_error()
    torch.cuda.synchronize()
    assert torch.isnan(out[0]).all()          # nothing was launched
    with pytest.raises(ValueError):           # the binding checks outputs against n and the dtype
        lens.shoot_direct_noalloc(dx[:10], dx[:10], [o[:5] for o in out])
    lens.close()
