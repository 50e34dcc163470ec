"""GPU smoothing lengths (lens_smoothing_lengths, Sec. 3.1) against the FP64
oracle on the same float32 positions.  Distances are formed in FP32 from
exact coordinate differences (Sterbenz), so the k-th distance agrees to a few
ulps; where two neighbours tie within rounding either may be the k-th, which
moves the value by no more than that rounding."""
import numpy as np
import pytest

import lensgen
from oracle import knn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1312_1128_gb300 as L  # noqa: E402


def gpu(xyz, k):
    r = L.smoothing_lengths(torch.from_numpy(np.ascontiguousarray(xyz, np.float32)).cuda(), k)
    torch.cuda.synchronize()
    return r.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("k", [1, 8, 32, 64])
def test_clustered_points_match_brute_force(k):
    xyz = lensgen.nfw_positions_3d(3000, 12)
    np.testing.assert_allclose(gpu(xyz, k), knn.kth_neighbour_distance_brute(xyz, k), rtol=1e-6)


def test_lattice_shells_exact():
    g = np.arange(9, dtype=np.float32) * np.float32(0.25)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    p = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    centre = (np.abs(p / 0.25 - 4) <= 2).all(axis=1)
    r = gpu(p, 32)
    assert (r[centre] == 0.5).all()  # 6 + 12 + 8 shells inside, the 32nd at 2a
    np.testing.assert_allclose(r, knn.kth_neighbour_distance_brute(p, 32), rtol=1e-7)


def test_duplicates_and_tiny_sets():
    g = np.random.default_rng(4)
    p = g.normal(size=(300, 3)).astype(np.float32)
    q = np.concatenate([p, p[:40]])
    r = gpu(q, 1)
    assert (r[:40] == 0).all() and (r[300:] == 0).all() and (r[40:300] > 0).all()
    small = g.uniform(size=(9, 3)).astype(np.float32)
    np.testing.assert_allclose(gpu(small, 8), knn.kth_neighbour_distance_brute(small, 8), rtol=1e-6)
    with pytest.raises(L.LensError):
        gpu(small, 9)


def test_fullsize_nfw_million():
    """The headline's 1e6 NFW particles, k = 32: every particle against the
    k-d tree on the same float32 positions, and against the smoothing lengths
    the workload generator stores (k-d tree on the FP64 positions)."""
    xyz = lensgen.nfw_positions_3d(1_000_000, 2)
    r = gpu(xyz, 32)
    np.testing.assert_allclose(r, knn.kth_neighbour_distance_tree(xyz, 32), rtol=1e-6)
    stored = lensgen.workload_nfw_sph(n_grid=4)["gauss"][:, 3].astype(np.float64)
    np.testing.assert_allclose(r, stored, rtol=2e-5)
