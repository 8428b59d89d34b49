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
* ``rollout_vjp`` / ``rollout_vjp_full``: composition of ``adjoint.step_vjp``
  and ``adjoint.temporal_correction_vjp`` over the steps of a rollout (no
  checkpointing: the oracle keeps every state); ``flat_grads`` lays the
  parameter gradients out like the parameter array.
* ``adam_step``: Adam (Kingma & Ba, 2015, Algorithm 1), the optimiser of the
  paper's training details.
"""

from __future__ import annotations

from typing import Optional

import numpy as np

from . import adjoint as A
from .fv import LearnedModel, Problem, learned_step, rk4_step, temporal_correction


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
    """Reverse mode of U0 -> (U_1 .. U_n) for the cotangents lam_traj[k] of U_{k+1},
    for a model without a temporal correction (see ``rollout_vjp_full``).

    Returns ``(lam0, grads)``; grads is None for the plain step and
    ``(W_L_bar, stencil_grads)`` summed over the steps for the learned one.
    """
    lam, g = rollout_vjp_full(U0, p, n, lam_traj, model)
    return lam, (None if g is None else (g["W_L"], g["stencil"]))


def _has_tc(model: Optional[LearnedModel]) -> bool:
    return model is not None and model.k_c > 0 and (model.tc_fno is not None or len(model.tc) > 0)


def rollout_states(U0: np.ndarray, p: Problem, n: int, model: Optional[LearnedModel] = None):
    """States u_0 .. u_n of a rollout (``oracle.fv.rollout``) and, for each k, the FV
    output before the temporal correction (Sec. 3.2: at k = M k_c,
    u_k = P(FV(u_{k-1}) + TC(u_{k-k_c} .. u_{k-1}) - mean))."""
    states, fv_out = [np.array(U0, dtype=np.float64)], [None]
    for k in range(1, n + 1):
        V = step(states[-1], p, model)
        fv_out.append(V)
        if _has_tc(model) and k % model.k_c == 0:
            V = temporal_correction(V, states[k - model.k_c:k], p, model)
        states.append(V)
    return states, fv_out


def _add(a, b):
    """Sum of two gradients of the same kind (arrays, lists of (dW, db), FNOParams)."""
    if a is None:
        return b
    if isinstance(a, np.ndarray):
        return a + b
    if isinstance(a, list):
        return [(x0 + y0, x1 + y1) for (x0, x1), (y0, y1) in zip(a, b)]
    return A._fno_sum(a, b)


def rollout_vjp_full(U0: np.ndarray, p: Problem, n: int, lam_traj: np.ndarray, model: Optional[LearnedModel] = None):
    """Reverse mode of U0 -> (U_1 .. U_n), the temporal correction included.

    lam_traj[k] is the cotangent of U_{k+1}. A corrected state u_k (k = M k_c) sends
    P(lam_k) into the FV step that produced it (``adjoint.step_vjp``; P is
    idempotent and that step already ends with P) and, through
    ``adjoint.temporal_correction_vjp``, cotangents to each of u_{k-k_c} .. u_{k-1};
    every state's cotangent is the sum of what reaches it.

    Returns ``(lam0, grads)``; grads is None for the plain step, else a dict with
    'W_L', 'stencil' (list of (dW, db)), 'fno' (FNOParams or None) and 'tc' (list
    of (dW, db) for the CNN head, FNOParams for the FNO correction, None without a
    correction), each summed over the steps.
    """
    states, fv_out = rollout_states(U0, p, n, model)
    pending = [np.zeros_like(states[0]) for _ in range(n + 1)]
    g = None if model is None else {"W_L": None, "stencil": None, "fno": None, "tc": None}
    for k in range(n, 0, -1):
        lam = pending[k] + lam_traj[k - 1]
        if _has_tc(model) and k % model.k_c == 0:
            lam, hbars, tg = A.temporal_correction_vjp(fv_out[k], states[k - model.k_c:k], p, model, lam)
            for s, hb in enumerate(hbars):
                pending[k - model.k_c + s] = pending[k - model.k_c + s] + hb
            g["tc"] = _add(g["tc"], tg)
        lam_in, sg = A.step_vjp(states[k - 1], p, lam, model)
        pending[k - 1] = pending[k - 1] + lam_in
        if sg is not None:
            g["W_L"] = _add(g["W_L"], sg[0])
            g["stencil"] = _add(g["stencil"], sg[1])
            if len(sg) > 2:
                g["fno"] = _add(g["fno"], sg[2])
    return pending[0], g


def flat_grads(g: dict, model: LearnedModel) -> np.ndarray:
    """A gradient dict of ``rollout_vjp_full`` as one flat array in the parameter
    layout of the library's parameter upload: W_L, the stencil layers (W then b),
    the temporal correction (CNN layers, or the FNO operator), then O_F. An
    operator is P_w, P_b, per layer R as [2M][M][Cin][Cout][re, im] (the real and
    imaginary partial derivatives), W, b, then Q_w, Q_b. Absent gradients of
    present parameters are zero."""
    def operator(f, like):
        if f is None:
            f = like
            zero = True
        else:
            zero = False
        out = [f.P_w.ravel(), f.P_b.ravel()]
        for R, W, b in zip(f.R, f.W, f.Wb):
            out += [np.stack([R.real, R.imag], axis=-1).ravel(), W.ravel(), b.ravel()]
        out += [f.Q_w.ravel(), f.Q_b.ravel()]
        v = np.concatenate(out)
        return np.zeros_like(v) if zero else v

    parts = [np.asarray(g["W_L"] if g["W_L"] is not None else np.zeros_like(model.W_L)).ravel()]
    st = g["stencil"] if g["stencil"] is not None else [(np.zeros_like(W), np.zeros_like(b)) for W, b in model.stencil]
    for dW, db in st:
        parts += [dW.ravel(), db.ravel()]
    if _has_tc(model):
        if model.tc_fno is not None:
            parts.append(operator(g["tc"], model.tc_fno))
        else:
            tc = g["tc"] if g["tc"] is not None else [(np.zeros_like(W), np.zeros_like(b)) for W, b in model.tc]
            for dW, db in tc:
                parts += [dW.ravel(), db.ravel()]
    if model.fno is not None:
        parts.append(operator(g["fno"], model.fno))
    return np.concatenate(parts)


def adam_step(p: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, t: int, lr: float = 1e-4,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update; returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def rollout_scalar_states(U0: np.ndarray, S0: np.ndarray, p: Problem, D: float, n: int,
                          model: Optional[LearnedModel] = None):
    """States (u_k, s_k), k = 0 .. n, of the joint rollout (``oracle.scalar.rollout_scalar``)
    and each step's velocity before its temporal correction."""
    from .fv import temporal_correction
    from .scalar import rk4_step_scalar

    U, S = np.array(U0, dtype=np.float64), np.array(S0, dtype=np.float64)
    states, fv_out = [(U, S)], [None]
    for k in range(1, n + 1):
        U1, S1 = rk4_step_scalar(U, S, p, D, model)
        fv_out.append(U1)
        if _has_tc(model) and k % model.k_c == 0:
            U1 = temporal_correction(U1, [states[m][0] for m in range(k - model.k_c, k)], p, model)
        U, S = U1, S1
        states.append((U, S))
    return states, fv_out


def rollout_scalar_vjp(U0: np.ndarray, S0: np.ndarray, p: Problem, D: float, n: int, lamU_traj: np.ndarray,
                       lamS_traj: np.ndarray, model: Optional[LearnedModel] = None):
    """Reverse mode of the joint rollout (u_0, s_0) -> (u_k, s_k), k = 1 .. n, with
    the velocity's temporal correction: lamU_traj[k - 1], lamS_traj[k - 1] are the
    cotangents of (u_k, s_k). Composition of the joint step's VJP
    (``adjoint.rk4_step_scalar_vjp``) and the correction's
    (``adjoint.temporal_correction_vjp``), each state's cotangent the sum of what
    reaches it. Returns (lamU0, lamS0, grads) with grads a dict of 'W_L', 'W_Ls',
    'stencil' and 'tc' (None for the plain step)."""
    states, fv_out = rollout_scalar_states(U0, S0, p, D, n, model)
    pu = [np.zeros_like(states[0][0]) for _ in range(n + 1)]
    ps = [np.zeros_like(states[0][1]) for _ in range(n + 1)]
    g = None if model is None else {"W_L": None, "W_Ls": None, "stencil": None, "tc": None}
    for k in range(n, 0, -1):
        lu = pu[k] + lamU_traj[k - 1]
        ls = ps[k] + lamS_traj[k - 1]
        if _has_tc(model) and k % model.k_c == 0:
            lu, hbars, tg = A.temporal_correction_vjp(fv_out[k], [states[m][0] for m in range(k - model.k_c, k)], p,
                                                      model, lu)
            for s, hb in enumerate(hbars):
                pu[k - model.k_c + s] = pu[k - model.k_c + s] + hb
            g["tc"] = _add(g["tc"], tg)
        out = A.rk4_step_scalar_vjp(states[k - 1][0], states[k - 1][1], p, D, lu, ls, model)
        pu[k - 1] = pu[k - 1] + out[0]
        ps[k - 1] = ps[k - 1] + out[1]
        if model is not None:
            wl, wls, st = out[2]
            g["W_L"] = _add(g["W_L"], wl)
            g["W_Ls"] = _add(g["W_Ls"], wls)
            g["stencil"] = _add(g["stencil"], st)
    return pu[0], ps[0], g
