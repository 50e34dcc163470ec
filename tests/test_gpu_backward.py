"""GPU adjoint (lens_shoot_rays_backward) checks for the lens-fit loss
L = sum |alpha - alpha_t|^2 (source-plane residuals, beta = theta - alpha,
Eq. lens_eq):

* against 4th-order central differences of the FP64 tree forward on 64
  random masses (the tree approximation is smooth in the masses: they move
  no particle between boxes);
* in direct-sum mode against the FP64 oracle gradient (masses and
  positions);
* the tree gradient against the FP64 oracle gradient within the tree's own
  accuracy;
* through torch.autograd.
"""
import numpy as np
import pytest

import lensgen
import oracle
from lens_testutil import comps_gauss, comps_points

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1312_1128_gb300 as L  # noqa: E402


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def fit_problem(n=3000, nr=2048, seed=61, precision="fp32"):
    parts = lensgen.nfw_particles(n, seed, fixed_sigma=0.01)
    pts = lensgen.point_disk(200, seed + 1, total_mass=0.02)
    g = lensgen.rng(seed + 2)
    rx = g.uniform(-0.6, 0.6, nr)
    ry = g.uniform(-0.6, 0.6, nr)
    dt = np.float64 if precision == "fp64" else np.float32
    target = parts.astype(np.float64).copy()
    target[:, 2] *= np.exp(0.05 * g.standard_normal(n))
    return parts, pts, target, rx.astype(dt), ry.astype(dt)


def loss_and_grad(lens, dx, dy, alpha_t, flags=0):
    out = lens.shoot(dx, dy, flags=flags | L.ALPHA_ONLY)
    a = torch.stack([out[0], out[1]], 1).double()
    r = a - alpha_t
    Lval = float((r * r).sum())
    g = (2 * r).to(lens.out_dtype)
    grads = lens.backward(dx, dy, g[:, 0].contiguous(), g[:, 1].contiguous(),
                          flags=flags & L.DIRECT)
    return Lval, [x.double().cpu().numpy() for x in grads]


def test_tree_adjoint_matches_mass_finite_differences_fp64():
    parts, pts, target, rx, ry = fit_problem(precision="fp64")
    p64 = parts.astype(np.float64)
    dx, dy = cu(rx), cu(ry)
    tl = L.Lens([L.Species.gauss(cu(target), 3.0)], theta=0.3, precision="fp64")
    t_out = tl.shoot(dx, dy, flags=L.ALPHA_ONLY)
    alpha_t = torch.stack([t_out[0], t_out[1]], 1).double()

    def lossf(p):
        lens = L.Lens([L.Species.gauss(cu(p), 3.0), L.Species.points(cu(pts.astype(np.float64)))],
                      theta=0.3, precision="fp64")
        out = lens.shoot(dx, dy, flags=L.ALPHA_ONLY)
        a = torch.stack([out[0], out[1]], 1).double()
        v = float(((a - alpha_t) ** 2).sum())
        lens.close()
        return v

    lens = L.Lens([L.Species.gauss(cu(p64), 3.0), L.Species.points(cu(pts.astype(np.float64)))],
                  theta=0.3, precision="fp64")
    _, (gg, gp) = loss_and_grad(lens, dx, dy, alpha_t)
    g = lensgen.rng(7)
    for j in g.choice(p64.shape[0], 64, replace=False):
        h = 1e-3 * p64[j, 2]

        def at(d):
            q = p64.copy()
            q[j, 2] += d
            return lossf(q)
        fd = (-at(2 * h) + 8 * at(h) - 8 * at(-h) + at(-2 * h)) / (12 * h)
        assert gg[j, 0] == pytest.approx(fd, rel=1e-3, abs=1e-6 * np.abs(gg[:, 0]).max())


def test_direct_adjoint_matches_oracle_gradient():
    parts, pts, target, rx, ry = fit_problem(n=2000, nr=1024)
    comps = oracle.concat(comps_gauss(parts, 3.0), comps_points(pts))
    tcomps = oracle.concat(comps_gauss(target, 3.0), comps_points(pts))
    rx64, ry64 = rx.astype(np.float64), ry.astype(np.float64)
    a_ref = oracle.direct_sum(comps, rx64, ry64)
    a_t = oracle.direct_sum(tcomps, rx64, ry64)[:, :2]
    G = np.zeros_like(a_ref)
    G[:, :2] = 2 * (a_ref[:, :2] - a_t)
    ref = oracle.direct_vjp(comps, rx64, ry64, G)
    lens = L.Lens([L.Species.gauss(cu(parts), 3.0), L.Species.points(cu(pts))], theta=0.3)
    _, grads = loss_and_grad(lens, cu(rx), cu(ry), torch.from_numpy(a_t).cuda(), flags=L.DIRECT)
    got = np.concatenate(grads)
    scale = np.abs(ref).max(axis=0)
    np.testing.assert_allclose(got, ref, rtol=1e-3, atol=1e-4 * scale.max())
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref)


@pytest.mark.parametrize("theta,bar", [(0.3, 2e-2), (0.1, 3e-3)])
def test_tree_adjoint_close_to_oracle_gradient(theta, bar):
    parts, pts, target, rx, ry = fit_problem(n=20000, nr=4096, seed=71)
    comps = comps_gauss(parts, 3.0)
    tcomps = comps_gauss(target, 3.0)
    rx64, ry64 = rx.astype(np.float64), ry.astype(np.float64)
    a_ref = oracle.direct_sum(comps, rx64, ry64)
    a_t = oracle.direct_sum(tcomps, rx64, ry64)[:, :2]
    G = np.zeros_like(a_ref)
    G[:, :2] = 2 * (a_ref[:, :2] - a_t)
    ref = oracle.direct_vjp(comps, rx64, ry64, G)
    lens = L.Lens([L.Species.gauss(cu(parts), 3.0)], theta=theta)
    # feed the oracle's upstream gradient: only the adjoint's own error remains
    gt = cu(G[:, :2].astype(np.float32))
    (got,) = lens.backward(cu(rx), cu(ry), gt[:, 0].contiguous(), gt[:, 1].contiguous())
    got = got.double().cpu().numpy()
    for k in range(3):
        err = np.linalg.norm(got[:, k] - ref[:, k]) / np.linalg.norm(ref[:, k])
        assert err <= bar, (k, err)


def test_autograd_function():
    parts, pts, target, rx, ry = fit_problem(n=1500, nr=512)
    data = cu(parts).requires_grad_(True)
    lens = L.Lens([L.Species.gauss(data.detach(), 3.0)], theta=0.3)
    dx, dy = cu(rx), cu(ry)
    alpha = L.shoot(lens, dx, dy, species_data=[data])
    loss = (alpha.double() ** 2).sum()
    (gd,) = torch.autograd.grad(loss, [data])
    g = (2 * alpha.detach()).contiguous()
    (ref,) = lens.backward(dx, dy, g[:, 0].contiguous(), g[:, 1].contiguous())
    np.testing.assert_allclose(gd[:, 2].cpu().numpy(), ref[:, 0].cpu().numpy(), rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(gd[:, 0].cpu().numpy(), ref[:, 1].cpu().numpy(), rtol=1e-5, atol=1e-6)
    assert torch.all(gd[:, 3] == 0)


def test_halo_gradient_direct():
    """Analytic halos: dL/d(r_E, x, y) of an SIS against the oracle."""
    pts = lensgen.point_disk(100, 81, total_mass=0.01)
    g = lensgen.rng(82)
    rx = g.uniform(-0.5, 0.5, 512).astype(np.float32)
    ry = g.uniform(-0.5, 0.5, 512).astype(np.float32)
    lens = L.Lens([L.Species.points(cu(pts))], [L.Halo.sis(0.05, -0.03, 0.2)], theta=0.3)
    comps = oracle.concat(comps_points(pts), oracle.make_components(oracle.SIS, 0.05, -0.03, 0.0, 0.2))
    ref_a = oracle.direct_sum(comps, rx.astype(np.float64), ry.astype(np.float64))
    G = np.zeros_like(ref_a)
    G[:, :2] = 2 * ref_a[:, :2]
    gsum = cu(G[:, :2].astype(np.float32))
    gh = torch.zeros(1, 3, dtype=torch.float64, device="cuda")
    lens.backward(cu(rx), cu(ry), gsum[:, 0].contiguous(), gsum[:, 1].contiguous(), g_halos=gh,
                  flags=L.DIRECT)
    # the oracle's mass slot is dL/dm; for the SIS the strength is r_E:
    # alpha is linear in r_E, so dL/dr_E = sum G.alpha_SIS / r_E
    sis = oracle.make_components(oracle.SIS, 0.05, -0.03, 0.0, 0.2)
    a_sis = oracle.direct_sum(sis, rx.astype(np.float64), ry.astype(np.float64))
    d_re = float((G[:, :2] * a_sis[:, :2]).sum()) / 0.2
    pos = oracle.direct_vjp(oracle.make_components(oracle.POINT, 0.05, -0.03, 1.0), rx.astype(np.float64),
                            ry.astype(np.float64), np.zeros_like(G))  # shape check only
    assert pos.shape == (1, 3)
    got = gh.cpu().numpy()[0]
    assert got[0] == pytest.approx(d_re, rel=1e-4)
    # positions: -sum G.J with the SIS Jacobian from its kappa, gamma
    k, g1_, g2_ = a_sis[:, 2], a_sis[:, 3], a_sis[:, 4]
    gx = -np.sum(G[:, 0] * (k + g1_) + G[:, 1] * g2_)
    gy = -np.sum(G[:, 0] * g2_ + G[:, 1] * (k - g1_))
    assert got[1] == pytest.approx(gx, rel=1e-4)
    assert got[2] == pytest.approx(gy, rel=1e-4)
