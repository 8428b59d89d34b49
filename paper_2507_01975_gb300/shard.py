"""Host-side logic of running the path on several GPUs (one process per GPU).

The forward path shards by trajectory: every rank advances its own batch and no
data crosses ranks. Data-parallel training has one real exchange step: the
parameter gradients of the ranks' batches are averaged (weighted by the number
of samples) before the optimiser step, so that every rank applies the update of
the full batch (the objective is a mean over samples, Sec. 4 Model Training).
"""

from __future__ import annotations


def trajectory_shard(rank: int, world: int, total: int) -> range:
    """Contiguous trajectory indices of ``rank`` out of ``total`` (ragged split:
    the first ``total % world`` ranks take one more)."""
    if not (0 <= rank < world) or total < 0:
        raise ValueError("need 0 <= rank < world and total >= 0")
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def average_gradients(grad, n_local: int, group=None):
    """In place: grad <- sum_r n_r grad_r / sum_r n_r over the ranks of ``group``
    (torch.distributed; gloo on CPU tensors, NCCL on device tensors)."""
    import torch
    import torch.distributed as dist

    grad.mul_(float(n_local))
    dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    n = torch.tensor([float(n_local)], dtype=torch.float64, device=grad.device)
    dist.all_reduce(n, op=dist.ReduceOp.SUM, group=group)
    grad.div_(float(n.item()))
    return grad


def max_over_ranks(seconds: float, group=None) -> float:
    """The job's time: the slowest rank's."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([seconds], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
