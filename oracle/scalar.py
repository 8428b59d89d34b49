"""Passive scalar of the shear flow, FP64 reference.

Test infrastructure only: imported by tests/, smoke() and bench.py's CPU arms,
never by the CUDA path.

The shear flow couples the incompressible momentum equation with the transport
of a passive scalar s (App. C.1, shear flow): s_t - D lap s = -u . grad s, with
D in {0.001, 0.002}. Reading (the paper gives the equation, not its finite-volume
form): s lives at the cell centres of the MAC grid and is advanced in flux form,
s_t = -div(u s_f - D grad_f s), where the face value s_f and the face derivative
grad_f s come from the physics kernels (App. B.2) along x at the u-faces and
along y at the v-faces -- four more operator instances beside the eight of the
momentum flux block. For a discretely divergence-free velocity the flux form and
the advective form differ by s div u = 0, and the flux form conserves the total
scalar exactly (finite-volume conservation, App. B.1). The scalar is not
projected; RK4 takes its stages from the same (projected) stage velocities as
the momentum equation (App. B.5).

Learned scalar (reading; the paper says the model learns the scalar's transport
but not how): the learnable flux block extends to the scalar's four instances
exactly as to the velocity's eight (Sec. 3.4): per-face kernels W_P + proj(W_Ls
+ C_s) / h^deriv on the same 5 x 4 tap grid, with a learnable conv W_Ls of their
own and the correction C_s from the same stencil network, which then reads
(u, v, s) and emits 80 more channels. The temporal correction stays on the
velocity.
"""

from __future__ import annotations

import numpy as np

from .fv import (FLOW_NAVIER_STOKES, N_COEF, Problem, apply_axial, cnn_forward, consistency_project,
                 learned_kernels, physics_kernel, project, shifted, temporal_correction, tendency)

#: the scalar's operator instances: (axis, kind) with kind 0 interpolation,
#: 1 derivative; output at the face between cells i-1 and i (taps i-2 .. i+1)
SCALAR_INSTANCES = [(0, 0), (0, 1), (1, 0), (1, 1)]
SCALAR_SHIFT = -2
#: first channel of the scalar instances in the network output of a model that
#: learns the scalar: instance m's tap (r, c) is channel SCALAR_COEF0 + 20 m + 4 r + c
SCALAR_COEF0 = N_COEF
N_COEF_SCALAR = N_COEF + 4 * 20


def scalar_face_values(S: np.ndarray, p: Problem, kernels=None) -> list:
    """s and its normal derivative at the u-faces (axis 0) and v-faces (axis 1);
    ``kernels[m]`` (optional, [5, 4] or per face [5, 4, ny, nx]) replaces instance
    m's physics kernel."""
    out = []
    for m, (axis, kind) in enumerate(SCALAR_INSTANCES):
        h = p.dx if axis == 0 else p.dy
        K = physics_kernel(kind, p.deriv_order, h) if kernels is None else kernels[m]
        out.append(apply_axial(S, K, axis, SCALAR_SHIFT))
    return out


def learned_scalar_kernels(C: np.ndarray, p: Problem, model) -> list:
    """Per-face kernels of the scalar's four instances, the reading of the learned
    flux block (Sec. 3.4) for the scalar: K_f = W_P + proj(W_Ls[kind, axis] +
    C_s,f) with the learned derivative part divided by the spacing along the
    instance's axis, C_s the network's scalar channels (``C`` its whole output)."""
    ny, nx = C.shape[1:]
    ks = []
    for m, (axis, kind) in enumerate(SCALAR_INSTANCES):
        h = p.dx if axis == 0 else p.dy
        c0 = SCALAR_COEF0 + 20 * m
        L = model.W_Ls[kind, axis][:, :, None, None] + C[c0:c0 + 20].reshape(5, 4, ny, nx)
        L = consistency_project(L)
        if kind == 1:
            L = L / h
        ks.append(physics_kernel(kind, p.deriv_order, h)[:, :, None, None] + L)
    return ks


def scalar_tendency(U: np.ndarray, S: np.ndarray, p: Problem, D: float, kernels=None) -> np.ndarray:
    """-div(u s_f - D grad_f s) at the cell centres for the velocity U[2, ny, nx]
    (u on the west faces, v on the south faces of each cell); ``kernels`` as in
    scalar_face_values."""
    sx, gx, sy, gy = scalar_face_values(S, p, kernels)
    Fx = U[0] * sx - D * gx
    Fy = U[1] * sy - D * gy
    return -(shifted(Fx, 0, 1) - Fx) / p.dx - (shifted(Fy, 1, 0) - Fy) / p.dy


def rk4_step_scalar(U: np.ndarray, S: np.ndarray, p: Problem, D: float, model=None):
    """One joint update (u_k, s_k) -> (u_{k+1}, s_{k+1}): the momentum stages of the
    FV step (projected for Navier-Stokes), the scalar's stages from the same
    stage velocities (App. B.5). With a model that learns the scalar (``W_Ls``
    set) every stage runs the network on (w, z) once: its first 160 channels give
    the velocity's learned kernels, the last 80 the scalar's."""
    P = (lambda W: project(W, p)) if p.flow == FLOW_NAVIER_STOKES else (lambda W: W)
    dt = p.dt

    def H(W, Z):
        if model is None:
            return tendency(W, p), scalar_tendency(W, Z, p, D)
        C = cnn_forward(np.concatenate([W, Z[None]], axis=0), model.stencil)
        return (tendency(W, p, learned_kernels(W, p, model, C=C)),
                scalar_tendency(W, Z, p, D, learned_scalar_kernels(C, p, model)))

    r1, q1 = H(U, S)
    w, z = P(U + 0.5 * dt * r1), S + 0.5 * dt * q1
    r2, q2 = H(w, z)
    w, z = P(U + 0.5 * dt * r2), S + 0.5 * dt * q2
    r3, q3 = H(w, z)
    w, z = P(U + dt * r3), S + dt * q3
    r4, q4 = H(w, z)
    return (P(U + (dt / 6.0) * (r1 + 2.0 * r2 + 2.0 * r3 + r4)),
            S + (dt / 6.0) * (q1 + 2.0 * q2 + 2.0 * q3 + q4))


def rollout_scalar(U0: np.ndarray, S0: np.ndarray, p: Problem, D: float, n_steps: int, model=None):
    """n_steps joint updates of the velocity and the scalar; with a model, the
    learned joint step and, every k_c steps, the velocity's temporal correction
    from the last k_c velocities (the scalar is not corrected)."""
    U, S = np.array(U0, dtype=np.float64), np.array(S0, dtype=np.float64)
    hist = [U.copy()]
    for k in range(1, n_steps + 1):
        U, S = rk4_step_scalar(U, S, p, D, model)
        if model is not None and model.k_c > 0 and k % model.k_c == 0:
            U = temporal_correction(U, hist[-model.k_c:], p, model)
        hist.append(U.copy())
        if len(hist) > 16:
            hist.pop(0)
    return U, S
