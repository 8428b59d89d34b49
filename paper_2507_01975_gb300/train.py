"""Unrolled training of the learnable module through the hand-written adjoint.

Host-side orchestration only: every numerical step runs in ``libldfv.so``
(fd_rollout, fd_rollout_adjoint, fd_train_step, fd_adam_step,
fd_set_params_device, fd_downsample). torch supplies device memory and streams.

* ``Rollout``: a ``torch.autograd.Function`` mapping (u0, theta) to the states
  u_1 .. u_n of an n-step rollout; its backward is fd_rollout_adjoint with
  checkpoints every ``ckpt_every`` steps.
* ``Trainer``: the paper's training loop (Sec. 4, Model Training; App. training
  details): autoregressive rollouts of ``k_s`` steps from label states, MSE
  against the coarse-grained labels, Adam.
* ``make_labels``: fine-grid plain-FV trajectories coarse-grained in space
  (face averages) and time (every ``ratio_t``-th fine step) into labels.
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

from . import fd


def _torch():
    import torch

    return torch


class Rollout:
    """``Rollout.apply(solver, u0, theta, n_steps, ckpt_every) -> traj[n, B, 2, N, N]``.

    theta is the device float32 parameter tensor the solver was last given
    (fd_set_params_device); its gradient is the parameter gradient of the
    rollout. Built lazily so that importing this module needs no torch.
    """

    _fn = None

    @classmethod
    def apply(cls, solver: fd.Solver, u0, theta, n_steps: int, ckpt_every: int):
        if cls._fn is None:
            torch = _torch()

            class _RolloutFn(torch.autograd.Function):
                @staticmethod
                def forward(ctx, u0, theta, solver, n_steps, ckpt_every):
                    traj = torch.empty((n_steps,) + tuple(u0.shape), dtype=u0.dtype, device=u0.device)
                    last = torch.empty_like(u0)
                    solver.rollout(u0, last, n_steps, traj=traj, save_every=1)
                    ctx.solver, ctx.n, ctx.k = solver, n_steps, ckpt_every
                    ctx.save_for_backward(u0, theta)
                    return traj

                @staticmethod
                def backward(ctx, grad_traj):
                    u0, theta = ctx.saved_tensors
                    lam0 = torch.empty_like(u0)
                    dtheta = torch.zeros_like(theta) if theta is not None else None
                    ctx.solver.rollout_adjoint(u0, ctx.n, ctx.k, grad_traj.contiguous(), lam0, dtheta)
                    return lam0, dtheta, None, None, None

            cls._fn = _RolloutFn
        return cls._fn.apply(u0, theta, solver, n_steps, ckpt_every)


def make_labels(fine: fd.Solver, u0_fine, n_coarse_steps: int, ratio_x: int, ratio_t: int):
    """Labels [n_coarse_steps + 1, B, 2, n/ratio_x, n/ratio_x]: the coarse-grained
    initial state followed by the coarse-grained fine state every ratio_t fine steps."""
    torch = _torch()
    b, _, n, _ = u0_fine.shape
    nc = n // ratio_x
    out = torch.empty((n_coarse_steps + 1, b, 2, nc, nc), dtype=u0_fine.dtype, device=u0_fine.device)
    fd.downsample(u0_fine, out[0], ratio_x)
    traj = torch.empty((n_coarse_steps,) + tuple(u0_fine.shape), dtype=u0_fine.dtype, device=u0_fine.device)
    last = torch.empty_like(u0_fine)
    fine.rollout(u0_fine, last, n_coarse_steps * ratio_t, traj=traj, save_every=ratio_t)
    for k in range(n_coarse_steps):
        fd.downsample(traj[k], out[k + 1], ratio_x)
    return out


@dataclass
class TrainConfig:
    unroll: int = 32          # k_s, rollout steps per sample
    ckpt_every: int = 8
    lr: float = 1e-4          # the paper's learning rate
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8


class Trainer:
    """Adam on the parameters of a learned solver, one fused training step per iteration."""

    def __init__(self, solver: fd.Solver, params0, cfg: Optional[TrainConfig] = None, group=None):
        """``group``: a torch.distributed process group for data-parallel training
        (one process per GPU, each with its own batch); the gradients are averaged
        over the ranks, weighted by batch size, before every Adam step."""
        torch = _torch()
        self.solver = solver
        self.group = group
        self.cfg = cfg or TrainConfig()
        self.theta = torch.as_tensor(params0, dtype=torch.float32).to("cuda").contiguous()
        self.grad = torch.zeros_like(self.theta)
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.t = 0
        solver.set_params_device(self.theta)

    def step(self, u0, targets):
        """One iteration: loss of the unrolled rollout from u0 against targets[unroll]
        (device), gradient, Adam update, parameter upload. Returns the loss tensor."""
        c = self.cfg
        self.solver.train_step(u0, targets, c.unroll, c.ckpt_every, self.grad, self.loss)
        if self.group is not None:
            from .shard import average_gradients

            average_gradients(self.grad, int(u0.shape[0]), self.group)
        self.t += 1
        fd.adam_step(self.theta, self.grad, self.m, self.v, self.t, c.lr, c.beta1, c.beta2, c.eps, zero_grads=True)
        self.solver.set_params_device(self.theta)
        return self.loss

    def evaluate(self, u0, targets):
        """Loss of the rollout against targets without a parameter update."""
        torch = _torch()
        n = self.cfg.unroll
        traj = torch.empty((n,) + tuple(u0.shape), dtype=u0.dtype, device=u0.device)
        last = torch.empty_like(u0)
        self.solver.rollout(u0, last, n, traj=traj, save_every=1)
        out = torch.zeros(1, dtype=torch.float64, device=u0.device)
        self.solver.mse_loss(traj, targets[:n], out)
        return out
