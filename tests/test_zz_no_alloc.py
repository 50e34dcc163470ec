"""The allocation-free entry point, through the C ABI.

lens_shoot_rays_direct_noalloc serves callers that cannot allocate device
memory while they shoot rays (another component owns the allocator, a
latency-bound loop, a fixed pre-reserved budget).  Its scratch is a fixed
device array inside the library.  Checked against the regular direct sum
(lens_shoot_rays with LENS_DIRECT) on two calls in a row, since the shared
array keeps the previous call's contents, and for the size limit.
Collected last so that a run stopping at the first failure has run every
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


def outputs(n):
    return [torch.full((n,), float("nan"), dtype=torch.float32, device="cuda") for _ in range(5)]


def test_noalloc_matches_direct_sum_on_consecutive_calls():
    gauss = lensgen.nfw_particles(4000, 41, nsph=16)
    pts = lensgen.point_disk(500, 42, total_mass=0.05)
    lens = L.Lens([L.Species.gauss(cu(gauss), 3.0), L.Species.points(cu(pts))],
                  [L.Halo.sis(0.05, 0.0, 0.2), L.Halo.disk(0.1, -0.1, -0.01, 0.4)], theta=0.3)
    g = lensgen.rng(43)
    for call, n in enumerate([5001, 20000]):
        rx = g.uniform(-0.9, 0.9, n).astype(np.float32)
        ry = g.uniform(-0.9, 0.9, n).astype(np.float32)
        dx, dy = cu(rx), cu(ry)
        ref = to_np(lens.shoot(dx, dy, flags=L.DIRECT))
        got = to_np(lens.shoot_direct_noalloc(dx, dy, outputs(n)))
        lens.sync()
        assert np.all(np.isfinite(got)), call
        # both are FP32 direct sums of the same terms; they may differ by rounding
        comps = oracle.concat(comps_gauss(gauss, 3.0), comps_points(pts),
                              oracle.make_components(oracle.SIS, 0.05, 0.0, 0.0, 0.2),
                              oracle.make_components(oracle.DISK, 0.1, -0.1, -0.01, 0.4))
        sel = np.arange(0, n, 7)
        _, absum = oracle.direct_sum(comps, rx[sel].astype(np.float64), ry[sel].astype(np.float64),
                                     with_absum=True)
        ok, _ = within_fp32_bar(got[sel], ref[sel], absum)
        assert ok.all(), (call, np.where(~ok.all(axis=1))[0][:5])
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
    lens.close()
