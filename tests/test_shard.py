"""Host logic of the multi-GPU path: LPT sharding of independent images and
the one exchange step of the reverse mode (parameter gradients), checked on
CPU with gloo ranks."""
import itertools
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1212_2245_b300 import shard, synth
from paper_1212_2245_b300.params import Params


def test_lpt_assigns_every_image_once():
    rng = np.random.default_rng(0)
    costs = rng.integers(1, 1000, 137).tolist()
    for m in (1, 2, 3, 8):
        parts = shard.lpt_partition(costs, m)
        assert len(parts) == m
        flat = sorted(itertools.chain.from_iterable(parts))
        assert flat == list(range(len(costs)))
        assert all(p == sorted(p) for p in parts)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("m", [2, 3])
def test_lpt_within_graham_bound(seed, m):
    """Makespan of LPT <= (4/3 - 1/(3m)) x the optimum, found by brute force
    over all assignments of 8 images."""
    rng = np.random.default_rng(seed)
    costs = rng.integers(1, 50, 8).tolist()
    parts = shard.lpt_partition(costs, m)
    lpt = max(sum(costs[i] for i in p) for p in parts)
    best = min(max(sum(c for c, r in zip(costs, a) if r == k) for k in range(m))
               for a in itertools.product(range(m), repeat=len(costs)))
    assert lpt <= (4.0 / 3.0 - 1.0 / (3 * m)) * best + 1e-9


def test_lpt_known_instance_and_ties():
    # Graham's tight example for m = 2: 3,3,2,2,2 -> LPT 7, optimum 6
    parts = shard.lpt_partition([3, 3, 2, 2, 2], 2)
    assert parts == [[0, 2, 4], [1, 3]]
    assert shard.lpt_partition([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]
    costs = shard.image_costs([(128, 256), (1024, 1024), (300, 200)], 10)
    assert costs == [327680.0, 10485760.0, 600000.0]
    assert shard.rank_images(costs, 2, 0) == [1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _tiny_batch():
    rng = np.random.default_rng(7)
    h = synth.raised_cosine_1d(5)
    gs = [synth.scene(12, 16, rng).astype(np.float32) for _ in range(5)]
    fs = [synth.degrade(g, h, 2.0, rng) for g in gs]
    return np.stack(fs), np.stack(gs), h


def _grads(f, g, h, p, iters):
    taps = torch.tensor(h, dtype=torch.float64, requires_grad=True)
    alpha = torch.tensor(p.alpha, dtype=torch.float64, requires_grad=True)
    K = torch.tensor(p.K, dtype=torch.float64, requires_grad=True)
    loss = oracle.wr3l_loss(torch.as_tensor(f, dtype=torch.float64), torch.as_tensor(g, dtype=torch.float64),
                            taps, alpha, K, p, iters)
    loss.backward()
    return [taps.grad.clone(), alpha.grad.reshape(1).clone(), K.grad.reshape(1).clone()]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        f, g, h = _tiny_batch()
        p = Params(alpha=0.01)
        mine = shard.rank_images(shard.image_costs([x.shape for x in f], 3), world, rank)
        grads = _grads(f[mine], g[mine], h, p, 3)
        shard.combine_param_grads(grads, len(mine), len(f))
        out[rank] = [x.numpy() for x in grads]
    finally:
        dist.destroy_process_group()


def test_sharded_gradients_equal_full_batch():
    """Two gloo ranks, each with its LPT share of 5 images: the combined
    parameter gradients equal the full-batch FP64 gradients."""
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    f, g, h = _tiny_batch()
    full = _grads(f, g, h, Params(alpha=0.01), 3)
    for r in range(world):
        for a, b in zip(res[r], full):
            np.testing.assert_allclose(a, b.numpy(), rtol=1e-10, atol=1e-14)
