"""The multi-GPU split of one problem through the CUDA kernels, on one GPU:
two Morton-contiguous ray ranges shot by two calls on the same (replicated)
tree, as two ranks would.  The direct sum of each ray does not depend on its
range, so the split forward equals the one-call forward bit for bit; the
tree forward of the split meets the tree tolerance against the oracle; the
two ranges' adjoints, summed as the all-reduce sums them, equal the one-call
adjoint to rounding.  (The collective itself is tested with gloo ranks in
test_shard.py.)"""
import numpy as np
import pytest

import lensgen
import oracle
from lens_testutil import comps_gauss, rel_errors, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1312_1128_gb300 as L  # noqa: E402
from paper_1312_1128_gb300 import shard  # noqa: E402


def test_two_range_split_on_one_gpu():
    """327,680 rays: each range still gives every SM enough ray groups, so no
    call splits its direct sum over particle slices (a split sums in another
    order)."""
    parts = lensgen.nfw_particles(3000, 51, nsph=16)
    g = lensgen.rng(52)
    n = 327680
    rx = g.uniform(-0.8, 0.8, n).astype(np.float32)
    ry = g.uniform(-0.8, 0.8, n).astype(np.float32)
    dx, dy = torch.from_numpy(rx).cuda(), torch.from_numpy(ry).cuda()
    lens = L.Lens([L.Species.gauss(torch.from_numpy(parts).cuda(), 3.0)], theta=0.3)
    order, bounds = shard.ray_ranges(rx, ry, 2)
    full_d = to_np(lens.shoot(dx, dy, flags=L.DIRECT))
    split_d = np.zeros_like(full_d)
    split_t = np.zeros_like(full_d)
    for r in range(2):
        idx = shard.rank_indices(order, bounds, r)
        split_d[idx] = to_np(shard.shoot_rank(lens, dx, dy, idx, flags=L.DIRECT))
        split_t[idx] = to_np(shard.shoot_rank(lens, dx, dy, idx))
    np.testing.assert_array_equal(split_d, full_d)
    sel = np.arange(0, rx.size, 100)
    ref = oracle.direct_sum(comps_gauss(parts, 3.0), rx[sel].astype(np.float64), ry[sel].astype(np.float64))
    ea, _, eg = rel_errors(split_t[sel], ref)
    assert np.median(ea) <= 1e-3 and np.median(eg) <= 1e-3
    # the direct-sum adjoint: each range's share, accumulated into the same
    # gradient (the sum the all-reduce forms), against the one-call adjoint
    ga = torch.from_numpy(2 * full_d[:, 0].astype(np.float32)).cuda(), \
        torch.from_numpy(2 * full_d[:, 1].astype(np.float32)).cuda()
    (full_g,) = lens.backward(dx, dy, *ga, flags=L.DIRECT)
    acc = [torch.zeros_like(full_g)]
    for r in range(2):
        idx = shard.rank_indices(order, bounds, r)
        i = torch.from_numpy(idx).cuda()
        lens.backward(dx[i].contiguous(), dy[i].contiguous(), ga[0][i].contiguous(), ga[1][i].contiguous(),
                      grads=acc, flags=L.DIRECT)
    torch.testing.assert_close(acc[0], full_g, rtol=1e-4, atol=1e-6 * float(full_g.abs().max()))
    lens.close()
