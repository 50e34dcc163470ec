"""One ray-shooting problem over several GPUs (Sec. 3.3: the rays are
distributed among the processors, every processor uses the whole tree).

Every rank holds a replica of the lens, built from the same particles, and
shoots one Morton-contiguous range of the rays: the forward pass exchanges
nothing, and a spatially compact range keeps the rank's ray groups (and so
its interaction lists) as tight as in a one-GPU call.  Range boundaries fall
on multiples of the ray-group size of the Morton order.  The backward pass
sums the ranks' particle and halo gradients with one all-reduce.

This module plans the split on the host and issues the collective; every ray
still goes through lens_shoot_rays / lens_shoot_rays_backward on its rank's
GPU.  One process per GPU, launched by torch.distributed.run.
"""
from __future__ import annotations

import numpy as np

_BITS = 16


def _spread16(v):
    """Put the 16 low bits of v at the even bit positions of a uint32."""
    v = v.astype(np.uint32) & np.uint32(0xFFFF)
    v = (v | (v << np.uint32(8))) & np.uint32(0x00FF00FF)
    v = (v | (v << np.uint32(4))) & np.uint32(0x0F0F0F0F)
    v = (v | (v << np.uint32(2))) & np.uint32(0x33333333)
    v = (v | (v << np.uint32(1))) & np.uint32(0x55555555)
    return v


def morton_keys(x, y):
    """32-bit Morton keys (x in the even bits) of 2D points, quantised to
    2^16 cells per side of their bounding square."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    if x.size == 0:
        return np.zeros(0, np.uint32)
    x0, y0 = x.min(), y.min()
    side = max(x.max() - x0, y.max() - y0)
    scale = (2 ** _BITS - 1) / side if side > 0 else 0.0
    qx = np.floor((x - x0) * scale).astype(np.int64)
    qy = np.floor((y - y0) * scale).astype(np.int64)
    return _spread16(qx) | (_spread16(qy) << np.uint32(1))


def ray_ranges(x, y, world: int, align: int = 64):
    """Split rays into `world` Morton-contiguous ranges.  Returns (order,
    bounds): order is the stable Morton order of the rays (indices into x, y)
    and rank r owns order[bounds[r]:bounds[r + 1]]; every inner boundary is a
    multiple of `align` (the ray-group size), so no group straddles two
    ranks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    n = np.asarray(x).size
    order = np.argsort(morton_keys(x, y), kind="stable")
    per = -(-n // world)                      # ceil
    per = -(-per // align) * align            # rounded up to whole groups
    bounds = np.minimum(np.arange(world + 1, dtype=np.int64) * per, n)
    return order, bounds


def rank_indices(order, bounds, rank: int):
    """The rays (indices into the caller's arrays) that `rank` shoots."""
    return order[bounds[rank]:bounds[rank + 1]]


def allreduce_sum(tensors, group=None):
    """Sum every tensor over the ranks in place (one all-reduce each): the
    particle and halo gradients of the backward pass."""
    import torch.distributed as dist
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors


def shoot_rank(lens, dx, dy, idx, origin=(0.0, 0.0), flags: int = 0):
    """Shoot this rank's rays (device tensors dx, dy indexed by the int64
    index array idx); returns the five outputs for those rays."""
    import torch
    i = torch.as_tensor(np.ascontiguousarray(idx), dtype=torch.int64, device=dx.device)
    return lens.shoot(dx[i].contiguous(), dy[i].contiguous(), origin=origin, flags=flags)


def backward_rank(lens, dx, dy, idx, g_alpha1, g_alpha2, origin=(0.0, 0.0), flags: int = 0,
                  g_halos=None, group=None):
    """This rank's share of the vector-Jacobian product (its rays' upstream
    gradients g_alpha1, g_alpha2, given in idx order), summed over the ranks:
    every rank returns the whole job's particle gradients (and g_halos)."""
    import torch
    i = torch.as_tensor(np.ascontiguousarray(idx), dtype=torch.int64, device=dx.device)
    grads = lens.backward(dx[i].contiguous(), dy[i].contiguous(), g_alpha1, g_alpha2, origin=origin,
                          flags=flags, g_halos=g_halos)
    allreduce_sum(grads + ([g_halos] if g_halos is not None else []), group)
    return grads
