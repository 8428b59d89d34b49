"""FP64 oracle of the training pieces: coarse-graining, the MSE objective, the
reverse mode of a rollout, and Adam.

TEST INFRASTRUCTURE ONLY -- see the package docstring.

* ``face_average``: the fine-to-coarse downsampling of the training labels
  (Sec. 4, Simulation Datasets; App. C.1 Table of dataset settings). The paper
  says only that the fine fields are downsampled in space and time; the reading
  used here is the face average of the staggered grid (a coarse face value is
  the mean of the fine face values that tile the coarse face), the
  coarse-graining that keeps the discrete divergence of the MAC grid.
* ``mse_loss``: the objective of Sec. 4 (Model Training), the mean over
  samples of the per-sample MSE, i.e. the mean over every rollout step,
  trajectory and element for samples of equal length.
* ``rollout_vjp``: composition of ``adjoint.step_vjp`` over the steps of a
  rollout (no checkpointing: the oracle keeps every state).
* ``adam_step``: Adam (Kingma & Ba, 2015, Algorithm 1), the optimiser of the
  paper's training details.
"""

from __future__ import annotations

from typing import Optional

import numpy as np

from . import adjoint as A
from .fv import LearnedModel, Problem, learned_step, rk4_step


def face_average(U: np.ndarray, r: int) -> np.ndarray:
    """Coarse state [2, n/r, n/r] from a fine state [2, n, n]."""
    _, ny, nx = U.shape
    nyc, nxc = ny // r, nx // r
    out = np.zeros((2, nyc, nxc))
    for J in range(nyc):
        for I in range(nxc):
            # u on the west face of coarse cell (I, J): fine west faces i = r I, rows r J .. r J + r - 1
            out[0, J, I] = np.mean([U[0, r * J + k, r * I] for k in range(r)])
            # v on the south face: fine south faces j = r J, columns r I .. r I + r - 1
            out[1, J, I] = np.mean([U[1, r * J, r * I + k] for k in range(r)])
    return out


def mse_loss(pred: np.ndarray, target: np.ndarray):
    """(loss, gradient) of mean((pred - target)^2) over all elements."""
    d = pred - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def step(U: np.ndarray, p: Problem, model: Optional[LearnedModel]) -> np.ndarray:
    return rk4_step(U, p) if model is None else learned_step(U, p, model)


def rollout_vjp(U0: np.ndarray, p: Problem, n: int, lam_traj: np.ndarray, model: Optional[LearnedModel] = None):
    """Reverse mode of U0 -> (U_1 .. U_n) for the cotangents lam_traj[k] of U_{k+1}.

    Returns ``(lam0, grads)``; grads is None for the plain step and
    ``(W_L_bar, stencil_grads)`` summed over the steps for the learned one.
    """
    states = [U0]
    for _ in range(n):
        states.append(step(states[-1], p, model))
    lam = np.zeros_like(U0)
    acc = None
    for k in range(n - 1, -1, -1):
        lam = lam + lam_traj[k]
        lam, g = A.step_vjp(states[k], p, lam, model)
        if g is not None:
            if acc is None:
                acc = (g[0].copy(), [(dW.copy(), db.copy()) for dW, db in g[1]])
            else:
                acc = (acc[0] + g[0], [(a + dW, b + db) for (a, b), (dW, db) in zip(acc[1], g[1])])
    return lam, acc


def adam_step(p: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, t: int, lr: float = 1e-4,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update; returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
