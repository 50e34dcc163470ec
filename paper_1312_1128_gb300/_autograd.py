"""torch.autograd wrapper: alpha from lens_shoot_rays, its vector-Jacobian
product from lens_shoot_rays_backward.  Argument marshalling only."""
from __future__ import annotations

import torch


class _ShootAlpha(torch.autograd.Function):
    @staticmethod
    def forward(ctx, lens, dx, dy, origin, *species_data):
        from . import ALPHA_ONLY, KEEP_LISTS
        if not lens.built_from(species_data):
            lens.rebuild(species_data)   # new values: the old tree's moments are stale
        # the walk's interaction lists are kept for the adjoint (dx, dy are
        # saved: autograd refuses a backward after they change in place)
        out = lens.shoot(dx, dy, origin=origin, flags=ALPHA_ONLY | KEEP_LISTS)
        ctx.lens = lens
        ctx.origin = origin
        ctx.save_for_backward(dx, dy)
        return torch.stack([out[0], out[1]], dim=1)

    @staticmethod
    def backward(ctx, g):
        dx, dy = ctx.saved_tensors
        lens = ctx.lens
        g = g.to(lens.out_dtype)
        g1, g2 = g[:, 0].contiguous(), g[:, 1].contiguous()
        from . import KEEP_LISTS
        grads = lens.backward(dx, dy, g1, g2, origin=ctx.origin, flags=KEEP_LISTS)
        out = []
        for s, gr in zip(lens.species, grads):
            gd = torch.zeros_like(s.data)
            gd[:, 0] = gr[:, 1].to(gd.dtype)   # x
            gd[:, 1] = gr[:, 2].to(gd.dtype)   # y
            gd[:, 2] = gr[:, 0].to(gd.dtype)   # m
            gd[:, 3] = gr[:, 3].to(gd.dtype)   # size (r_sm or r_s; 0 for points)
            out.append(gd)
        return (None, None, None, None, *out)


def shoot_alpha(lens, dx, dy, origin=(0.0, 0.0), species_data=None):
    """alpha (n, 2) at rays origin + (dx, dy); differentiable w.r.t. the
    species tensors (columns x, y, m, size); the lens is rebuilt from them
    when they are not its current data."""
    data = species_data if species_data is not None else [s.data for s in lens.species]
    return _ShootAlpha.apply(lens, dx, dy, tuple(origin), *data)
