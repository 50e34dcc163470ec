"""Failure detection without a GPU fault: a bounded wait that runs out.

The producer/consumer walk (LENS_WALK_PAIRS) hands buffers between two warps
through mbarrier phases, and every wait has a limit in SM clock cycles
(lens_set_wait_limit).  With a limit of a few hundred cycles the waits run out
long before the partner warp arrives: both warps must return, the call's
status word must report LENS_ERR_TIMEOUT through lens_sync_status, and the
tree and the CUDA context must stay usable (the next call, with the default
limit, gives the bits of the same walk form on an undisturbed tree).
"""
import numpy as np
import pytest

import lensgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1312_1128_gb300 as L  # noqa: E402

TIMEOUT = 4


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("walk", ["pairs", "trios"])
def test_pairs_walk_wait_runs_out_and_reports_timeout(walk):
    parts = lensgen.nfw_particles(20000, 91, nsph=16)
    g = lensgen.rng(92)
    dx = cu(g.uniform(-0.8, 0.8, 40000).astype(np.float32))
    dy = cu(g.uniform(-0.8, 0.8, 40000).astype(np.float32))
    ref_lens = L.Lens([L.Species.gauss(cu(parts), 3.0)], theta=0.3, walk=walk, group_rays=64)
    ref = ref_lens.shoot(dx, dy)
    ref_lens.sync()
    lens = L.Lens([L.Species.gauss(cu(parts), 3.0)], theta=0.3, walk=walk, group_rays=64)
    assert lens.info()["walk"] == walk
    lens.set_wait_limit(200)
    lens.shoot(dx, dy)
    with pytest.raises(L.LensError) as e:
        lens.sync()
    assert e.value.status == TIMEOUT, str(e.value)
    lens.sync()                      # the error word was cleared
    lens.set_wait_limit(0)           # back to the default (about 2 s)
    out = lens.shoot(dx, dy)
    lens.sync()
    for a, b in zip(out, ref):
        assert torch.equal(a, b)     # the form is deterministic: an undisturbed tree's bits
    with pytest.raises(L.LensError):
        lens.set_wait_limit(-1)
    lens.close()
    ref_lens.close()


OOM = 3


def until_success(call, max_fail=400):
    """Fail the 1st, 2nd, ... device allocation that `call` makes, one try
    each: every try must raise LENS_ERR_OOM until one gets all it asks for.
    Returns (failed tries, the successful result)."""
    for after in range(max_fail):
        L.fail_allocations(after)
        try:
            res = call()
        except L.LensError as e:
            assert e.status == OOM, str(e)
            continue
        finally:
            L.fail_allocations(-1)
        return after, res
    raise AssertionError("the call kept failing")


def same(a, b):
    for x, y in zip(a, b):
        if x is not None:
            torch.testing.assert_close(x, y, rtol=0, atol=0)


def test_every_entry_point_reports_oom_and_the_tree_stays_usable():
    """The host-side failure-injection hook fails each device allocation of
    each entry point in turn: the call returns LENS_ERR_OOM and releases what
    it had allocated, and the same call then succeeds on the same tree with
    the results of an undisturbed tree."""
    parts = lensgen.nfw_particles(20000, 93, nsph=16)
    pts = lensgen.point_disk(3000, 94, total_mass=0.05)
    g = lensgen.rng(95)
    n = 30000
    dx = cu(g.uniform(-0.8, 0.8, n).astype(np.float32))
    dy = cu(g.uniform(-0.8, 0.8, n).astype(np.float32))
    halos = [L.Halo.sis(0.0, 0.0, 0.3)]

    def build():
        return L.Lens([L.Species.gauss(cu(parts), 3.0), L.Species.points(cu(pts))], halos, theta=0.3)

    ref_lens = build()
    ref = ref_lens.shoot(dx, dy)
    ref_psi = ref_lens.potential(dx, dy)
    ga = (2 * ref[0]).contiguous(), (2 * ref[1]).contiguous()
    ref_grad = ref_lens.backward(dx, dy, *ga)
    offsets = np.array([0, 10000, 30000], np.int64)
    origins = np.zeros((2, 2))
    ref_b = ref_lens.shoot_batches(offsets, origins, dx, dy)
    torch.cuda.synchronize()

    tries, lens = until_success(build)
    assert tries > 10                       # the build makes dozens of allocations
    same(lens.shoot(dx, dy), ref)           # a fresh tree: its ray scratch is allocated here

    lens2 = build()
    tries, out = until_success(lambda: lens2.shoot(dx, dy))
    assert tries >= 1
    same(out, ref)
    lens3 = build()
    tries, psi = until_success(lambda: lens3.potential(dx, dy))
    assert tries >= 1
    same(psi, ref_psi)
    tries, grad = until_success(lambda: lens2.backward(dx, dy, *ga))
    assert tries >= 4                       # four accumulators per species
    for a, b in zip(grad, ref_grad):
        torch.testing.assert_close(a, b, rtol=1e-5, atol=1e-6 * float(b.abs().max()))
    lens4 = build()
    tries, outb = until_success(lambda: lens4.shoot_batches(offsets, origins, dx, dy))
    assert tries >= 1
    same(outb, ref_b)
    lens5 = build()
    tries, _ = until_success(lambda: lens5.autotune(dx, dy))
    assert tries >= 1
    lens5.sync()
    tries, _ = until_success(lambda: lens5.reserve(2 * n))
    # the autotuned group size or walk form may sum in another order
    for a, b in zip(lens5.shoot(dx, dy), ref):
        torch.testing.assert_close(a, b, rtol=1e-4, atol=1e-5 * float(b.abs().max()))

    sis = L.Lens([], [L.Halo.sis(0.0, 0.0, 1.0)], theta=0.3, precision="fp64")
    ref_imgs, _ = sis.find_images([(0.5, 0.0, 0.1)], -10.0, -10.0, 20.0, 64)
    sis2 = L.Lens([], [L.Halo.sis(0.0, 0.0, 1.0)], theta=0.3, precision="fp64")
    tries, (imgs, _) = until_success(lambda: sis2.find_images([(0.5, 0.0, 0.1)], -10.0, -10.0, 20.0, 64))
    assert tries >= 1 and imgs == ref_imgs

    xyz = torch.from_numpy(lensgen.nfw_positions_3d(5000, 96)).cuda()
    ref_r = L.smoothing_lengths(xyz, 16)
    tries, r = until_success(lambda: L.smoothing_lengths(xyz, 16))
    assert tries >= 1
    torch.testing.assert_close(r, ref_r, rtol=0, atol=0)
    for x in (ref_lens, lens, lens2, lens3, lens4, lens5, sis, sis2):
        x.sync()
        x.close()
