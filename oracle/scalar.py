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
"""

from __future__ import annotations

import numpy as np

from .fv import (FLOW_NAVIER_STOKES, Problem, apply_axial, physics_kernel, project, shifted,
                 tendency)

#: the scalar's operator instances: (axis, kind) with kind 0 interpolation,
#: 1 derivative; output at the face between cells i-1 and i (taps i-2 .. i+1)
SCALAR_INSTANCES = [(0, 0), (0, 1), (1, 0), (1, 1)]
SCALAR_SHIFT = -2


def scalar_face_values(S: np.ndarray, p: Problem) -> list:
    """s and its normal derivative at the u-faces (axis 0) and v-faces (axis 1)."""
    out = []
    for axis, kind in SCALAR_INSTANCES:
        h = p.dx if axis == 0 else p.dy
        out.append(apply_axial(S, physics_kernel(kind, p.deriv_order, h), axis, SCALAR_SHIFT))
    return out


def scalar_tendency(U: np.ndarray, S: np.ndarray, p: Problem, D: float) -> np.ndarray:
    """-div(u s_f - D grad_f s) at the cell centres for the velocity U[2, ny, nx]
    (u on the west faces, v on the south faces of each cell)."""
    sx, gx, sy, gy = scalar_face_values(S, p)
    Fx = U[0] * sx - D * gx
    Fy = U[1] * sy - D * gy
    return -(shifted(Fx, 0, 1) - Fx) / p.dx - (shifted(Fy, 1, 0) - Fy) / p.dy


def rk4_step_scalar(U: np.ndarray, S: np.ndarray, p: Problem, D: float):
    """One joint update (u_k, s_k) -> (u_{k+1}, s_{k+1}): the momentum stages of the
    plain FV step (projected for Navier-Stokes), the scalar's stages from the same
    stage velocities (App. B.5)."""
    P = (lambda W: project(W, p)) if p.flow == FLOW_NAVIER_STOKES else (lambda W: W)
    dt = p.dt
    r1, q1 = tendency(U, p), scalar_tendency(U, S, p, D)
    w, z = P(U + 0.5 * dt * r1), S + 0.5 * dt * q1
    r2, q2 = tendency(w, p), scalar_tendency(w, z, p, D)
    w, z = P(U + 0.5 * dt * r2), S + 0.5 * dt * q2
    r3, q3 = tendency(w, p), scalar_tendency(w, z, p, D)
    w, z = P(U + dt * r3), S + dt * q3
    r4, q4 = tendency(w, p), scalar_tendency(w, z, p, D)
    return (P(U + (dt / 6.0) * (r1 + 2.0 * r2 + 2.0 * r3 + r4)),
            S + (dt / 6.0) * (q1 + 2.0 * q2 + 2.0 * q3 + q4))


def rollout_scalar(U0: np.ndarray, S0: np.ndarray, p: Problem, D: float, n_steps: int):
    """n_steps joint updates of the velocity and the scalar."""
    U, S = np.array(U0, dtype=np.float64), np.array(S0, dtype=np.float64)
    for _ in range(n_steps):
        U, S = rk4_step_scalar(U, S, p, D)
    return U, S

