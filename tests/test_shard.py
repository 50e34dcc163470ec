"""The multi-GPU split of one problem (Sec. 3.3: rays distributed among the
processors, the tree replicated), on the CPU with two gloo ranks.

The host logic of paper_1312_1128_gb300.shard -- Morton-contiguous ray
ranges aligned to the ray-group size, and the sum all-reduce of particle
gradients -- runs with the FP64 oracle standing in for each rank's GPU: the
split forward must equal the one-rank forward bit for bit (each ray's sum
does not depend on which rank shoots it), and the reduced gradient must equal
the one-rank gradient to rounding.  The same split through the CUDA kernels
on one GPU is in test_gpu_shard.py; on several GPUs it is unmeasured.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")

from paper_1312_1128_gb300 import shard  # noqa: E402


def test_morton_keys_interleave_x_in_even_bits():
    x = np.array([0.0, 1.0, 0.0, 1.0, 0.5])
    y = np.array([0.0, 0.0, 1.0, 1.0, 0.0])
    k = shard.morton_keys(x, y)
    assert k[0] == 0
    assert k[1] == 0x55555555          # x = 2^16 - 1 in the even bits
    assert k[2] == 0xAAAAAAAA          # y in the odd bits
    assert k[3] == 0xFFFFFFFF
    # x = 0.5 -> floor(0.5 * 65535) = 32767 = 0x7FFF: the even bits of 0x15555555
    assert k[4] == 0x15555555


def test_ray_ranges_cover_align_and_are_morton_contiguous():
    g = np.random.default_rng(3)
    for n, world in [(10000, 2), (10000, 3), (777, 4), (64, 5), (0, 2)]:
        x, y = g.uniform(-1, 1, n), g.uniform(0, 2, n)
        order, bounds = shard.ray_ranges(x, y, world)
        assert np.array_equal(np.sort(order), np.arange(n))
        assert bounds[0] == 0 and bounds[-1] == n and np.all(np.diff(bounds) >= 0)
        assert np.all(bounds[1:-1][bounds[1:-1] < n] % 64 == 0)
        k = shard.morton_keys(x, y)
        for r in range(world - 1):
            a, b = shard.rank_indices(order, bounds, r), shard.rank_indices(order, bounds, r + 1)
            if a.size and b.size:
                assert k[a].max() <= k[b].min()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import lensgen
    import oracle
    parts = lensgen.nfw_particles(800, 31, fixed_sigma=0.02)
    p = parts.astype(np.float64)
    comps = oracle.make_components(oracle.GAUSS, p[:, 0], p[:, 1], p[:, 2], p[:, 3], 3.0)
    g = lensgen.rng(32)
    rx, ry = g.uniform(-0.5, 0.5, 1500), g.uniform(-0.5, 0.5, 1500)
    target = oracle.direct_sum(comps, rx, ry)[:, :2] * (1 + 0.05 * g.standard_normal((1500, 2)))
    return comps, rx, ry, target


def _rank_main(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1312_1128_gb300 import shard as S
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        comps, rx, ry, target = _problem()
        order, bounds = S.ray_ranges(rx, ry, ws)
        idx = S.rank_indices(order, bounds, rank)
        # this rank's forward (the oracle in the role of the rank's GPU)
        out = oracle.direct_sum(comps, rx[idx], ry[idx], nthreads=1)
        G = np.zeros_like(out)
        G[:, :2] = 2 * (out[:, :2] - target[idx])
        grad = torch.from_numpy(oracle.direct_vjp(comps, rx[idx], ry[idx], G, nthreads=1))
        S.allreduce_sum([grad])
        q.put((rank, idx, out, grad.numpy()))
    finally:
        dist.destroy_process_group()


def test_split_forward_bitwise_and_reduced_gradient_two_gloo_ranks():
    import oracle
    import torch.multiprocessing as mp
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    comps, rx, ry, target = _problem()
    full = oracle.direct_sum(comps, rx, ry, nthreads=1)
    G = np.zeros_like(full)
    G[:, :2] = 2 * (full[:, :2] - target)
    gfull = oracle.direct_vjp(comps, rx, ry, G, nthreads=1)
    seen = np.zeros(rx.size, bool)
    for rank, idx, out, grad in got:
        assert np.array_equal(out, full[idx])           # the split forward, bit for bit
        seen[idx] = True
        np.testing.assert_allclose(grad, gfull, rtol=1e-11, atol=1e-13 * np.abs(gfull).max())
    assert seen.all()
    np.testing.assert_array_equal(got[0][3], got[1][3])  # every rank holds the same sum
