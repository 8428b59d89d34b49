"""Multi-process host logic on CPU (gloo, world size 2): trajectory sharding,
gradient averaging of data-parallel training (checked against the
single-process full-batch gradient of the oracle objective), and the max-over-
ranks timing."""

import os
import socket

import numpy as np
import pytest

from oracle import train as T
from paper_2507_01975_gb300.shard import trajectory_shard

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("total,world", [(16, 2), (17, 2), (3, 4), (0, 3), (512, 8)])
def test_sharding_covers_every_trajectory_once(total, world):
    seen = []
    for r in range(world):
        s = trajectory_shard(r, world, total)
        seen.extend(s)
        assert len(s) in (total // world, total // world + 1)
    assert seen == list(range(total))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, total, out):
    import torch.distributed as dist

    from paper_2507_01975_gb300.shard import average_gradients, max_over_ranks

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(0)
    pred, tgt = rng.standard_normal((2, total, 2, 8, 8))
    idx = list(trajectory_shard(rank, world, total))
    # per-rank gradient of the mean-over-samples MSE w.r.t. an additive bias theta
    # of the prediction: d/dtheta mean((pred + theta - t)^2) = mean(2 (pred - t))
    _, g = T.mse_loss(pred[idx], tgt[idx])
    grad = torch.tensor([g.sum()], dtype=torch.float64)
    average_gradients(grad, len(idx))
    t = max_over_ranks(float(rank + 1))
    out[rank] = (float(grad.item()), t)
    dist.destroy_process_group()


def test_data_parallel_gradient_equals_full_batch_gradient():
    import torch.multiprocessing as mp

    world, total = 2, 5  # ragged shards: 3 + 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, total, out), nprocs=world, join=True)
        res = dict(out)
    rng = np.random.default_rng(0)
    pred, tgt = rng.standard_normal((2, total, 2, 8, 8))
    _, g = T.mse_loss(pred, tgt)
    full = g.sum()
    for r in range(world):
        assert abs(res[r][0] - full) <= 1e-12 * max(1.0, abs(full))
        assert res[r][1] == 2.0
