"""FP64 oracle of the adjoint (vector-Jacobian product) of one FV step.

TEST INFRASTRUCTURE ONLY -- see the package docstring. Hand-derived reverse
mode of ``oracle.fv``: given u_n and lam = dL/du_{n+1}, returns dL/du_n and
dL/dtheta for the learnable parameters (W_L, the stencil network). The
solver's differentiability is what the paper's training relies on (Sec. 4.1,
Eq. for the loss; the "differentiable solver backbone" of the introduction);
the paper gives no derivation, so every rule here is the transpose of the
corresponding forward line in ``oracle.fv``:

* periodic shift  g = shifted(f, a, b)      ->  f_bar += shifted(g_bar, -a, -b)
* face operator   v = sum_rc K_rc tap_rc(f) ->  f_bar += sum_rc tap_rc^T(K_rc v_bar),
                                                K_bar_rc = v_bar tap_rc(f)
* projection      P symmetric (P^T = P)
* consistency projection (orthogonal projector) -> L_bar = proj(K_bar) * scale
* conv3x3 / GELU: transposed convolution, weight correlation, GELU'.

Pinned in ``tests/test_oracle_adjoint.py`` by dot-product tests against a
fourth-order finite-difference Jacobian-vector product and by central
differences on the parameters.
"""

from __future__ import annotations

from typing import Optional

import numpy as np

from .fv import (
    FLOW_BURGERS,
    FLOW_NAVIER_STOKES,
    INSTANCES,
    LearnedModel,
    Problem,
    apply_axial,
    cnn_forward,
    consistency_project,
    face_values,
    gelu_grad,
    learned_kernels,
    physics_kernel,
    plain_kernels,
    project,
    shifted,
    shifted_c,
    tendency,
)


def unshift(g: np.ndarray, dj: int, di: int) -> np.ndarray:
    """Adjoint of ``shifted(f, dj, di)``: ``shifted(g, -dj, -di)``."""
    return shifted(g, -dj, -di)


def tendency_vjp(U: np.ndarray, p: Problem, kernels, Tbar: np.ndarray, want_kbar: bool = False,
                 extra: Optional[np.ndarray] = None, want_vbar: bool = False):
    """Reverse mode of ``oracle.fv.tendency`` for fixed kernels (and fixed extra
    face values, the frequency-domain operator's output, when given).

    Returns ``(Ubar, Kbar)``: the gradient with respect to the state through
    the face-operator taps and the direct terms, and (when ``want_kbar``) the
    per-location kernel gradients ``Kbar[q][5, 4, ny, nx]``; with ``want_vbar``
    also the face-value cotangents ``vbar[q]`` (what flows into ``extra``).
    """
    dx, dy = p.dx, p.dy
    fv = face_values(U, kernels)
    if extra is not None:
        fv = [f + extra[q] for q, f in enumerate(fv)]
    Uc, Gxc, Uk, Gyu, Vk, Gxv, Vc, Gyc = fv
    Tu, Tv = Tbar[0], Tbar[1]
    vbar = [None] * 8
    # advection of u: -(Uc^2 - W(Uc^2)) / dx
    A_bar = -Tu / dx + unshift(Tu, 0, -1) / dx
    vbar[0] = 2.0 * Uc * A_bar
    # corner products P = Uk Vk in both equations
    P_bar = (-unshift(Tu, 1, 0) + Tu) / dy + (-unshift(Tv, 0, 1) + Tv) / dx
    vbar[2] = P_bar * Vk
    vbar[4] = P_bar * Uk
    # advection of v: -(Vc^2 - S(Vc^2)) / dy
    B_bar = -Tv / dy + unshift(Tv, -1, 0) / dy
    vbar[6] = 2.0 * Vc * B_bar
    # diffusion
    vbar[1] = p.nu * (Tu - unshift(Tu, 0, -1)) / dx
    vbar[3] = p.nu * (unshift(Tu, 1, 0) - Tu) / dy
    vbar[5] = p.nu * (unshift(Tv, 0, 1) - Tv) / dx
    vbar[7] = p.nu * (Tv - unshift(Tv, -1, 0)) / dy
    Ubar = np.zeros_like(U)
    if p.flow == FLOW_BURGERS:
        divc = Gxc + Gyc
        Ubar[0] += Tu * 0.5 * (shifted(divc, 0, -1) + divc)
        Ubar[1] += Tv * 0.5 * (shifted(divc, -1, 0) + divc)
        hu = 0.5 * Tu * U[0]
        hv = 0.5 * Tv * U[1]
        divc_bar = unshift(hu, 0, -1) + hu + unshift(hv, -1, 0) + hv
        vbar[1] = vbar[1] + divc_bar
        vbar[7] = vbar[7] + divc_bar
    if p.forcing_kind == 1:
        Ubar[0] += -p.drag * Tu
        Ubar[1] += -p.drag * Tv
    # face operators
    Kbar = [None] * 8
    for q, (fld, axis, _kind, shift) in enumerate(INSTANCES):
        K = kernels[q]
        if want_kbar:
            Kbar[q] = np.zeros((5, 4) + U.shape[1:])
        for r in range(5):
            for c in range(4):
                if axis == 0:
                    a, b = r - 2, c + shift
                else:
                    a, b = c + shift, r - 2
                Ubar[fld] += unshift(K[r, c] * vbar[q], a, b)
                if want_kbar:
                    Kbar[q][r, c] = vbar[q] * shifted(U[fld], a, b)
    return (Ubar, Kbar, vbar) if want_vbar else (Ubar, Kbar)


def cnn_vjp(x: np.ndarray, layers, ybar: np.ndarray):
    """Reverse mode of ``oracle.fv.cnn_forward``: returns (xbar, [(dW, db)])."""
    _, pre = cnn_forward(x, layers, keep=True)
    n_layers = len(layers)
    acts = [x] + [None] * n_layers
    from .fv import gelu

    for l in range(n_layers - 1):
        acts[l + 1] = gelu(pre[l])
    grads = [None] * n_layers
    zbar = ybar
    for l in range(n_layers - 1, -1, -1):
        W, _b = layers[l]
        h = acts[l]
        dW = np.zeros_like(W)
        for a in (-1, 0, 1):
            for e in (-1, 0, 1):
                dW[:, :, a + 1, e + 1] = np.einsum("oji,cji->oc", zbar, shifted_c(h, a, e))
        db = zbar.sum(axis=(1, 2))
        grads[l] = (dW, db)
        hbar = np.zeros_like(h)
        for a in (-1, 0, 1):
            for e in (-1, 0, 1):
                hbar += shifted_c(np.einsum("oc,oji->cji", W[:, :, a + 1, e + 1], zbar), -a, -e)
        if l > 0:
            zbar = hbar * gelu_grad(pre[l - 1])
        else:
            zbar = hbar
    return zbar, grads


def learned_tendency_vjp(U: np.ndarray, p: Problem, model: LearnedModel, Tbar: np.ndarray):
    """Reverse mode of H(U) = tendency(U, learned_kernels(U), O_F(U)).

    Returns ``(Ubar, W_L_bar, stencil_grads, fno_grads)``; fno_grads is None without
    a frequency-domain operator. The ablation variants follow the forward: without
    the physics convolution the learned kernel is not projected, so neither is its
    gradient; with the frequency operator only, the kernels are zero and the stencil
    network's gradients are zero.
    """
    extra = None
    if model.fno is not None:
        from .fno import fno_forward

        extra = fno_forward(U, model.fno)
    ks = learned_kernels(U, p, model)
    Ubar, Kbar, vbar = tendency_vjp(U, p, ks, Tbar, want_kbar=model.ablation != 2, extra=extra, want_vbar=True)
    ny, nx = U.shape[1:]
    WLbar = np.zeros_like(model.W_L)
    if model.ablation == 2:
        grads = [(np.zeros_like(W), np.zeros_like(b)) for W, b in model.stencil]
    else:
        Cbar = np.zeros((160, ny, nx))
        for q, (_fld, axis, kind, _shift) in enumerate(INSTANCES):
            h = p.dx if axis == 0 else p.dy
            scale = 1.0 / h if kind == 1 else 1.0
            Lbar = (consistency_project(Kbar[q]) if model.ablation == 0 else Kbar[q]) * scale
            Cbar[q * 20:(q + 1) * 20] = Lbar.reshape(20, ny, nx)
            WLbar[kind, axis] += Lbar.sum(axis=(2, 3))
        xbar, grads = cnn_vjp(U, model.stencil, Cbar)
        Ubar = Ubar + xbar
    fno_grads = None
    if model.fno is not None:
        from .fno import fno_vjp

        Ub_f, fno_grads = fno_vjp(U, model.fno, np.stack(vbar))
        Ubar = Ubar + Ub_f
    return Ubar, WLbar, grads, fno_grads


def step_vjp(U: np.ndarray, p: Problem, lam: np.ndarray, model: Optional[LearnedModel] = None):
    """Reverse mode of one RK4 step (``oracle.fv.rk4_step`` / ``learned_step``).

    u' = P(u + dt/6 (r1 + 2 r2 + 2 r3 + r4)), r_s = H(w_s), w_1 = u,
    w_2 = P(u + dt/2 r1), w_3 = P(u + dt/2 r2), w_4 = P(u + dt r3).
    Returns ``(lam_in, grads)`` where ``grads`` is None for the plain step,
    ``(W_L_bar, stencil_grads)`` for the learned step, and ``(W_L_bar,
    stencil_grads, fno_grads)`` when the model has a frequency-domain operator.
    """
    ns = p.flow == FLOW_NAVIER_STOKES
    P = (lambda W: project(W, p)) if ns else (lambda W: W)

    def H(W):
        if model is None:
            return tendency(W, p)
        if model.fno is not None:
            from .fno import fno_forward

            return tendency(W, p, learned_kernels(W, p, model), fno_forward(W, model.fno))
        return tendency(W, p, learned_kernels(W, p, model))

    def H_vjp(W, Tb):
        if model is None:
            Ub, _ = tendency_vjp(W, p, plain_kernels(p), Tb)
            return Ub, None
        Ub, wlb, g, fg = learned_tendency_vjp(W, p, model, Tb)
        return Ub, (wlb, g, fg)

    # forward stage states
    w1 = U
    r1 = H(w1)
    w2 = P(U + 0.5 * p.dt * r1)
    r2 = H(w2)
    w3 = P(U + 0.5 * p.dt * r2)
    r3 = H(w3)
    w4 = P(U + p.dt * r3)
    # reverse
    g = P(lam)
    lam_in = g.copy()
    rb4 = p.dt / 6.0 * g
    rb3 = p.dt / 3.0 * g
    rb2 = p.dt / 3.0 * g
    rb1 = p.dt / 6.0 * g
    acc_wl = np.zeros((2, 2, 5, 4)) if model is not None else None
    acc_g = None
    acc_f = None

    def add(grads):
        nonlocal acc_wl, acc_g, acc_f
        if grads is None:
            return
        wlb, g_, fg = grads
        acc_wl += wlb
        if acc_g is None:
            acc_g = [(dW.copy(), db.copy()) for dW, db in g_]
        else:
            acc_g = [(a0 + dW, a1 + db) for (a0, a1), (dW, db) in zip(acc_g, g_)]
        if fg is not None:
            acc_f = fg if acc_f is None else _fno_sum(acc_f, fg)

    wb4, gr = H_vjp(w4, rb4)
    add(gr)
    y = P(wb4)
    lam_in += y
    rb3 = rb3 + p.dt * y
    wb3, gr = H_vjp(w3, rb3)
    add(gr)
    y = P(wb3)
    lam_in += y
    rb2 = rb2 + 0.5 * p.dt * y
    wb2, gr = H_vjp(w2, rb2)
    add(gr)
    y = P(wb2)
    lam_in += y
    rb1 = rb1 + 0.5 * p.dt * y
    wb1, gr = H_vjp(w1, rb1)
    add(gr)
    lam_in += wb1
    if model is None:
        return lam_in, None
    return lam_in, ((acc_wl, acc_g) if model.fno is None else (acc_wl, acc_g, acc_f))


def _fno_sum(a, b):
    """Sum of two FNOParams-shaped gradients."""
    from .fno import FNOParams

    return FNOParams(P_w=a.P_w + b.P_w, P_b=a.P_b + b.P_b, R=[x + y for x, y in zip(a.R, b.R)],
                     W=[x + y for x, y in zip(a.W, b.W)], Wb=[x + y for x, y in zip(a.Wb, b.Wb)],
                     Q_w=a.Q_w + b.Q_w, Q_b=a.Q_b + b.Q_b)


def temporal_correction_vjp(U: np.ndarray, hist, p: Problem, model: LearnedModel, gbar: np.ndarray):
    """Reverse mode of ``oracle.fv.temporal_correction`` (Sec. 3.2, 3.5):
    out = P(U + c - mean(c)), c = TC(concat(hist)), TC the CNN head or the FNO.
    Returns (Ubar, [hist_bar per state], grads) with grads the CNN's [(dW, db)] or
    the FNO's gradient FNOParams. The mean removal (identity minus the per-component
    average) and the projection are symmetric, so each is its own transpose."""
    g = project(gbar, p) if p.flow == FLOW_NAVIER_STOKES else gbar
    cbar = g - g.mean(axis=(1, 2), keepdims=True)
    x = np.concatenate([h for h in hist], axis=0)
    if model.tc_fno is not None:
        from .fno import fno_vjp

        xbar, grads = fno_vjp(x, model.tc_fno, cbar)
    else:
        xbar, grads = cnn_vjp(x, model.tc, cbar)
    return g.copy(), [xbar[2 * s:2 * s + 2] for s in range(len(hist))], grads


def scalar_tendency_vjp(U: np.ndarray, S: np.ndarray, p: Problem, D: float, qbar: np.ndarray, kernels=None,
                        want_kbar: bool = False):
    """Reverse mode of ``oracle.scalar.scalar_tendency``: (Ubar, Sbar) for the
    cotangent qbar of -div(u s_f - D grad_f s); every rule is the transpose of a
    forward line (flux difference, product with the face velocity, face operators).
    ``kernels`` as in the forward (per-face learned kernels); with ``want_kbar``
    also the kernel cotangents Kbar[m][5, 4, ny, nx] of the four instances."""
    from .scalar import SCALAR_INSTANCES, SCALAR_SHIFT, scalar_face_values

    sx, _gx, sy, _gy = scalar_face_values(S, p, kernels)
    Fx_bar = (qbar - shifted(qbar, 0, -1)) / p.dx
    Fy_bar = (qbar - shifted(qbar, -1, 0)) / p.dy
    Ubar = np.stack([Fx_bar * sx, Fy_bar * sy])
    face_bar = [Fx_bar * U[0], -D * Fx_bar, Fy_bar * U[1], -D * Fy_bar]
    Sbar = np.zeros_like(S)
    Kbar = [None] * 4
    for m, ((axis, kind), vb) in enumerate(zip(SCALAR_INSTANCES, face_bar)):
        K = physics_kernel(kind, p.deriv_order, p.dx if axis == 0 else p.dy) if kernels is None else kernels[m]
        if want_kbar:
            Kbar[m] = np.zeros((5, 4) + S.shape)
        for r in range(5):
            for c in range(4):
                if kernels is None and K[r, c] == 0.0 and not want_kbar:
                    continue
                a, b = (r - 2, c + SCALAR_SHIFT) if axis == 0 else (c + SCALAR_SHIFT, r - 2)
                Sbar += unshift(K[r, c] * vb, a, b)
                if want_kbar:
                    Kbar[m][r, c] = vb * shifted(S, a, b)
    return (Ubar, Sbar, Kbar) if want_kbar else (Ubar, Sbar)


def learned_joint_tendency_vjp(U: np.ndarray, S: np.ndarray, p: Problem, D: float, model: LearnedModel,
                               rbar: np.ndarray, qbar: np.ndarray):
    """Reverse mode of one stage of the learned joint step (a model that learns the
    scalar): r = tendency(U, K(C)), q = scalar_tendency(U, S, K_s(C)) with C the
    network on (u, v, s). The kernel cotangents of the eight velocity and four
    scalar instances pass through the consistency projection and 1/h to the 240
    network-output channels, W_L and W_Ls; the network's input cotangent splits
    into the velocity's two channels and the scalar's. Returns (Ubar, Sbar,
    (W_L_bar, W_Ls_bar, stencil_grads))."""
    from .scalar import N_COEF_SCALAR, SCALAR_COEF0, SCALAR_INSTANCES, learned_scalar_kernels

    assert model.ablation == 0, "a model that learns the scalar takes the full operator"
    x = np.concatenate([U, S[None]], axis=0)
    C = cnn_forward(x, model.stencil)
    ks = learned_kernels(U, p, model, C=C)
    kss = learned_scalar_kernels(C, p, model)
    Ub, Kbar = tendency_vjp(U, p, ks, rbar, want_kbar=True)
    Uq, Sb, Ksbar = scalar_tendency_vjp(U, S, p, D, qbar, kernels=kss, want_kbar=True)
    ny, nx = S.shape
    Cbar = np.zeros((N_COEF_SCALAR, ny, nx))
    WLbar, WLsbar = np.zeros_like(model.W_L), np.zeros_like(model.W_Ls)
    for q, (_fld, axis, kind, _shift) in enumerate(INSTANCES):
        scale = 1.0 / (p.dx if axis == 0 else p.dy) if kind == 1 else 1.0
        Lbar = consistency_project(Kbar[q]) * scale
        Cbar[q * 20:(q + 1) * 20] = Lbar.reshape(20, ny, nx)
        WLbar[kind, axis] += Lbar.sum(axis=(2, 3))
    for m, (axis, kind) in enumerate(SCALAR_INSTANCES):
        scale = 1.0 / (p.dx if axis == 0 else p.dy) if kind == 1 else 1.0
        Lbar = consistency_project(Ksbar[m]) * scale
        c0 = SCALAR_COEF0 + 20 * m
        Cbar[c0:c0 + 20] = Lbar.reshape(20, ny, nx)
        WLsbar[kind, axis] += Lbar.sum(axis=(2, 3))
    xbar, grads = cnn_vjp(x, model.stencil, Cbar)
    return Ub + Uq + xbar[:2], Sb + xbar[2], (WLbar, WLsbar, grads)


def rk4_step_scalar_vjp(U: np.ndarray, S: np.ndarray, p: Problem, D: float, lamU: np.ndarray, lamS: np.ndarray,
                        model: Optional[LearnedModel] = None):
    """Reverse mode of ``oracle.scalar.rk4_step_scalar``: (Ubar, Sbar) for the
    cotangents of (u_{k+1}, s_{k+1}). The scalar's stages depend on the stage
    velocities, so every stage's velocity cotangent collects the scalar term too.
    With a model that learns the scalar also the parameter gradients: returns
    (Ubar, Sbar, (W_L_bar, W_Ls_bar, stencil_grads)) summed over the stages."""
    from .scalar import rk4_step_scalar, scalar_tendency  # noqa: F401

    ns = p.flow == FLOW_NAVIER_STOKES
    P = (lambda W: project(W, p)) if ns else (lambda W: W)
    dt = p.dt

    def H(W, Z):
        if model is None:
            return tendency(W, p), scalar_tendency(W, Z, p, D)
        from .scalar import learned_scalar_kernels

        C = cnn_forward(np.concatenate([W, Z[None]], axis=0), model.stencil)
        return (tendency(W, p, learned_kernels(W, p, model, C=C)),
                scalar_tendency(W, Z, p, D, learned_scalar_kernels(C, p, model)))

    w1, z1 = U, S
    r1, q1 = H(w1, z1)
    w2, z2 = P(U + 0.5 * dt * r1), S + 0.5 * dt * q1
    r2, q2 = H(w2, z2)
    w3, z3 = P(U + 0.5 * dt * r2), S + 0.5 * dt * q2
    r3, q3 = H(w3, z3)
    w4, z4 = P(U + dt * r3), S + dt * q3
    g = P(lamU)
    Ubar, Sbar = g.copy(), lamS.copy()
    rb = [dt / 6.0 * g, dt / 3.0 * g, dt / 3.0 * g, dt / 6.0 * g]
    qb = [dt / 6.0 * lamS, dt / 3.0 * lamS, dt / 3.0 * lamS, dt / 6.0 * lamS]
    ws, zs = [w1, w2, w3, w4], [z1, z2, z3, z4]
    coef = [None, 0.5 * dt, 0.5 * dt, dt]  # w_s = P(U + coef_s r_{s-1}), z_s = S + coef_s q_{s-1}
    acc = None
    for s in (3, 2, 1, 0):
        if model is None:
            wq, zb = scalar_tendency_vjp(ws[s], zs[s], p, D, qb[s])
            wb = tendency_vjp(ws[s], p, plain_kernels(p), rb[s])[0] + wq
        else:
            wb, zb, gr = learned_joint_tendency_vjp(ws[s], zs[s], p, D, model, rb[s], qb[s])
            acc = gr if acc is None else (acc[0] + gr[0], acc[1] + gr[1],
                                          [(a + dW, b + db) for (a, b), (dW, db) in zip(acc[2], gr[2])])
        if s == 0:
            Ubar += wb
            Sbar += zb
        else:
            Sbar += zb
            qb[s - 1] = qb[s - 1] + coef[s] * zb
            y = P(wb)
            Ubar += y
            rb[s - 1] = rb[s - 1] + coef[s] * y
    return (Ubar, Sbar) if model is None else (Ubar, Sbar, acc)
