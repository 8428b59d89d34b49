"""Pins of the oracle's learned scalar operators (shear flow's passive scalar,
CPU only): the scalar's four instances with per-face kernels W_P + proj(W_Ls +
C_s) / h^deriv, C_s from the stencil network run on (u, v, s).

* geometry: a single unit tap (r, c) of instance m returns s at the cell centre
  (c - 3/2) cells along the instance's axis and (r - 2) cells across it from the
  face (found from the MAC coordinates, not from the oracle's shifts);
* consistency: any learned part that passed the projection still interpolates
  (differentiates) a linear s exactly at every face away from the periodic wrap;
* conservation: the flux form keeps the total scalar for any learned kernels;
* reduction: a zero module gives the plain joint step;
* symmetry: the learned joint step commutes with periodic translations.
A dropped consistency projection and a row/column swap for the y-axis instances,
planted in the oracle, each fail one of these.
"""

import math

import numpy as np
import pytest

import oracle as O
import oracle.scalar as OS
from paper_2507_01975_gb300 import inputs as I

NX, NY = 16, 12
LX, LY = 4.0, 3.7


def problem(**kw):
    base = dict(nx=NX, ny=NY, lx=LX, ly=LY, nu=1e-3, dt=2e-2)
    base.update(kw)
    return O.Problem(**base)


def model(seed, last_scale=0.3, ws_std=0.05, kc=0):
    st = I.random_conv_stack(seed, 3, O.CNN_HIDDEN, OS.N_COEF_SCALAR, last_scale=last_scale)
    rng = np.random.default_rng(seed + 7)
    return O.LearnedModel(W_L=I.random_wl(seed + 1, 1e-2), stencil=st, W_Ls=rng.standard_normal((2, 2, 5, 4)) * ws_std,
                          k_c=kc, tc=I.random_conv_stack(seed + 2, 2 * kc, O.CNN_HIDDEN, 2, last_scale=0.02) if kc else [])


def velocity(p, seed):
    rng = np.random.default_rng(seed)
    return O.project(rng.standard_normal((2, p.ny, p.nx)) * 0.3, p)


def centres(p):
    return np.meshgrid((np.arange(p.nx) + 0.5) * p.dx, (np.arange(p.ny) + 0.5) * p.dy)


def single_tap_error(m, r, c):
    """Deviation of a single-unit-tap kernel from the geometric lookup."""
    p = problem()
    axis, _kind = OS.SCALAR_INSTANCES[m]
    rng = np.random.default_rng(7 + 20 * m + 4 * r + c)
    S = rng.standard_normal((p.ny, p.nx))
    K = np.zeros((5, 4))
    K[r, c] = 1.0
    ks = [np.zeros((5, 4)) for _ in range(4)]
    ks[m] = K
    got = OS.scalar_face_values(S, p, ks)[m]
    j = np.arange(p.ny)[:, None] * np.ones((1, p.nx), dtype=int)
    i = np.ones((p.ny, 1), dtype=int) * np.arange(p.nx)[None, :]
    # face of instance m at cell (j, i): the west face (x = i dx, y = (j + 1/2) dy) for
    # axis 0, the south face (x = (i + 1/2) dx, y = j dy) for axis 1
    fx = i * p.dx if axis == 0 else (i + 0.5) * p.dx
    fy = (j + 0.5) * p.dy if axis == 0 else j * p.dy
    ax, tr = (c - 1.5), (r - 2)
    px = fx + (ax if axis == 0 else tr) * p.dx
    py = fy + (tr if axis == 0 else ax) * p.dy
    ci = np.rint(px / p.dx - 0.5).astype(int)
    cj = np.rint(py / p.dy - 0.5).astype(int)
    assert np.max(np.abs(px / p.dx - 0.5 - ci)) < 1e-9 and np.max(np.abs(py / p.dy - 0.5 - cj)) < 1e-9
    return float(np.max(np.abs(got - S[cj % p.ny, ci % p.nx])))


@pytest.mark.parametrize("m", range(4))
def test_single_tap_geometry(m):
    for r in range(5):
        for c in range(4):
            assert single_tap_error(m, r, c) < 1e-14


def linear_field_error(seed=3):
    """Max error of the learned scalar kernels on s = a + b x + c y at interior faces."""
    p = problem()
    mdl = model(seed)
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((OS.N_COEF_SCALAR, p.ny, p.nx))
    ks = OS.learned_scalar_kernels(C, p, mdl)
    a, b, c = 0.3, -1.1, 0.7
    x, y = centres(p)
    S = a + b * x + c * y
    vals = OS.scalar_face_values(S, p, ks)
    jj, ii = np.meshgrid(np.arange(p.ny), np.arange(p.nx), indexing="ij")
    inner = (ii >= 3) & (ii <= p.nx - 3) & (jj >= 3) & (jj <= p.ny - 3)
    xu, yu = ii * p.dx, (jj + 0.5) * p.dy          # west faces
    xv, yv = (ii + 0.5) * p.dx, jj * p.dy          # south faces
    exact = [a + b * xu + c * yu, np.full_like(xu, b), a + b * xv + c * yv, np.full_like(xv, c)]
    return max(float(np.max(np.abs(v - e)[inner])) for v, e in zip(vals, exact))


def test_consistency_on_a_linear_field():
    assert linear_field_error() < 1e-11


def test_learned_scalar_conserves_the_total():
    p = problem()
    mdl = model(5)
    U = velocity(p, 1)
    S = np.random.default_rng(2).standard_normal((p.ny, p.nx))
    C = O.cnn_forward(np.concatenate([U, S[None]]), mdl.stencil)
    q = OS.scalar_tendency(U, S, p, 2e-3, OS.learned_scalar_kernels(C, p, mdl))
    assert abs(q.sum()) <= 1e-12 * np.abs(q).sum()
    U1, S1 = OS.rk4_step_scalar(U, S, p, 2e-3, mdl)
    assert abs(S1.sum() - S.sum()) <= 1e-12 * np.abs(S).sum()
    # the learned part changed the scalar's step
    _, S0 = OS.rk4_step_scalar(U, S, p, 2e-3)
    assert np.abs(S1 - S0).max() > 1e-6


def test_zero_module_is_the_plain_joint_step():
    p = problem()
    st = I.random_conv_stack(9, 3, O.CNN_HIDDEN, OS.N_COEF_SCALAR, last_scale=0.0)
    zero = O.LearnedModel(W_L=np.zeros((2, 2, 5, 4)), stencil=st, W_Ls=np.zeros((2, 2, 5, 4)))
    U = velocity(p, 3)
    S = np.random.default_rng(4).standard_normal((p.ny, p.nx))
    Ua, Sa = OS.rk4_step_scalar(U, S, p, 1e-3, zero)
    Ub, Sb = OS.rk4_step_scalar(U, S, p, 1e-3)
    assert np.abs(Ua - Ub).max() < 1e-13 and np.abs(Sa - Sb).max() < 1e-13


def test_learned_joint_step_commutes_with_translation():
    p = problem()
    mdl = model(11)
    U = velocity(p, 5)
    S = np.random.default_rng(6).standard_normal((p.ny, p.nx))
    Ua, Sa = OS.rk4_step_scalar(U, S, p, 1e-3, mdl)
    sh = (3, 5)
    Ub, Sb = OS.rk4_step_scalar(np.roll(U, sh, axis=(1, 2)), np.roll(S, sh, axis=(0, 1)), p, 1e-3, mdl)
    assert np.abs(np.roll(Ua, sh, axis=(1, 2)) - Ub).max() < 1e-12
    assert np.abs(np.roll(Sa, sh, axis=(0, 1)) - Sb).max() < 1e-12


def test_planted_mistakes_fail(monkeypatch):
    # a dropped consistency projection breaks the exactness on linear fields
    monkeypatch.setattr(OS, "consistency_project", lambda L: L)
    assert linear_field_error() > 1e-3
    monkeypatch.undo()
    assert linear_field_error() < 1e-11
    # a row / column swap for the y-axis instances breaks the geometry
    orig = OS.apply_axial

    def swapped(f, K, axis, shift):
        if axis == 1 and K.shape[:2] == (5, 4) and np.count_nonzero(K) == 1:
            r, c = np.argwhere(K)[0]
            if r < 4:
                K2 = np.zeros_like(K)
                K2[c, r] = K[r, c]
                K = K2
        return orig(f, K, axis, shift)

    monkeypatch.setattr(OS, "apply_axial", swapped)
    assert max(single_tap_error(2, r, c) for r in range(5) for c in range(4)) > 1e-3


# --- reverse mode of the learned joint step -----------------------------------
def narrow_scalar_model(seed, ws_std=0.05):
    """The stencil network at width 8 (3 -> 8 x 5 -> 240) keeps the finite differences cheap."""
    st = I.random_conv_stack(seed, 3, 8, OS.N_COEF_SCALAR, last_scale=0.3)
    rng = np.random.default_rng(seed + 7)
    return O.LearnedModel(W_L=I.random_wl(seed + 1, 2e-2), stencil=st, W_Ls=rng.standard_normal((2, 2, 5, 4)) * ws_std)


GRIDS = {
    "ns16x8": dict(nx=16, ny=8, lx=2.0, ly=1.3, nu=1e-2, dt=1e-2),
    "burgers13x9": dict(nx=13, ny=9, lx=1.0, ly=0.8, nu=1e-2, dt=2e-3, flow=O.FLOW_BURGERS),
}


def joint_state(p, seed):
    rng = np.random.default_rng(seed)
    U = 0.3 * rng.standard_normal((2, p.ny, p.nx))
    if p.flow == O.FLOW_NAVIER_STOKES:
        U = O.project(U, p)
    return U, rng.standard_normal((p.ny, p.nx))


@pytest.mark.parametrize("grid", list(GRIDS))
def test_learned_joint_step_vjp_dot_product(grid):
    from oracle import adjoint as A

    p = O.Problem(**GRIDS[grid])
    mdl = narrow_scalar_model(21)
    U, S = joint_state(p, 22)
    rng = np.random.default_rng(23)
    dU, dS = rng.standard_normal(U.shape), rng.standard_normal(S.shape)
    if p.flow == O.FLOW_NAVIER_STOKES:
        dU = O.project(dU, p)
    lamU, lamS = rng.standard_normal(U.shape), rng.standard_normal(S.shape)
    D, eps = 2e-3, 1e-3

    def f(t):
        u1, s1 = OS.rk4_step_scalar(U + t * dU, S + t * dS, p, D, mdl)
        return np.sum(u1 * lamU) + np.sum(s1 * lamS)

    jv = (-f(2 * eps) + 8 * f(eps) - 8 * f(-eps) + f(-2 * eps)) / (12 * eps)
    Ub, Sb, _ = A.rk4_step_scalar_vjp(U, S, p, D, lamU, lamS, mdl)
    rhs = np.sum(dU * Ub) + np.sum(dS * Sb)
    assert abs(jv - rhs) <= 1e-9 * (abs(jv) + 1.0)


@pytest.mark.parametrize("grid", list(GRIDS))
def test_learned_joint_step_parameter_gradients(grid):
    """Central differences on W_L, W_Ls (both kinds and axes), the first layer's
    weights on the s channel and the last layer's scalar channels."""
    from oracle import adjoint as A

    p = O.Problem(**GRIDS[grid])
    mdl = narrow_scalar_model(31)
    U, S = joint_state(p, 32)
    rng = np.random.default_rng(33)
    lamU, lamS = rng.standard_normal(U.shape), rng.standard_normal(S.shape)
    D, eps = 2e-3, 1e-3
    _, _, (wlb, wlsb, grads) = A.rk4_step_scalar_vjp(U, S, p, D, lamU, lamS, mdl)

    def loss(m):
        u1, s1 = OS.rk4_step_scalar(U, S, p, D, m)
        return np.sum(u1 * lamU) + np.sum(s1 * lamS)

    def bumped(which, idx, s):
        wl, wls = mdl.W_L.copy(), mdl.W_Ls.copy()
        st = [(W.copy(), b.copy()) for W, b in mdl.stencil]
        if which == "wl":
            wl[idx] += s
        elif which == "wls":
            wls[idx] += s
        else:
            st[which][0][idx] += s
        return O.LearnedModel(W_L=wl, stencil=st, W_Ls=wls)

    checks = [("wl", (0, 1, 3, 2), wlb), ("wls", (0, 0, 2, 1), wlsb), ("wls", (1, 0, 1, 3), wlsb),
              ("wls", (0, 1, 4, 0), wlsb), ("wls", (1, 1, 2, 2), wlsb),
              (0, (5, 2, 1, 0), grads[0][0]), (5, (170, 3, 1, 1), grads[5][0]), (5, (233, 6, 2, 0), grads[5][0])]
    for which, idx, g in checks:
        fd = (loss(bumped(which, idx, eps)) - loss(bumped(which, idx, -eps))) / (2 * eps)
        assert abs(fd - g[idx]) <= 1e-6 * max(1e-2, abs(fd)), (which, idx, fd, g[idx])


def test_planted_mistake_in_the_joint_reverse_mode_fails(monkeypatch):
    """Dropping the consistency projection from the kernel cotangents (the forward
    keeps it) breaks the dot-product identity."""
    from oracle import adjoint as A

    monkeypatch.setattr(A, "consistency_project", lambda L: L)
    with pytest.raises(AssertionError):
        test_learned_joint_step_vjp_dot_product("ns16x8")


def test_joint_rollout_vjp_with_corrections_dot_product():
    """The joint rollout's reverse mode with the velocity's temporal correction
    (k_c = 2, four steps): the dot product with a finite-difference JVP through
    ``rollout_scalar`` in the initial velocity and scalar."""
    from oracle import train as T

    p = O.Problem(**GRIDS["ns16x8"])
    kc = 2
    mdl = narrow_scalar_model(41)
    mdl = O.LearnedModel(W_L=mdl.W_L, stencil=mdl.stencil, W_Ls=mdl.W_Ls, k_c=kc,
                         tc=I.random_conv_stack(42, 2 * kc, 8, 2, last_scale=0.2))
    U, S = joint_state(p, 43)
    rng = np.random.default_rng(44)
    n, D, eps = 4, 1e-3, 1e-3
    lu = rng.standard_normal((n,) + U.shape)
    ls = rng.standard_normal((n,) + S.shape)
    dU, dS = O.project(rng.standard_normal(U.shape), p), rng.standard_normal(S.shape)

    def f(t):
        states, _ = T.rollout_scalar_states(U + t * dU, S + t * dS, p, D, n, mdl)
        return sum(np.sum(states[k][0] * lu[k - 1]) + np.sum(states[k][1] * ls[k - 1]) for k in range(1, n + 1))

    jv = (-f(2 * eps) + 8 * f(eps) - 8 * f(-eps) + f(-2 * eps)) / (12 * eps)
    lu0, ls0, g = T.rollout_scalar_vjp(U, S, p, D, n, lu, ls, mdl)
    rhs = np.sum(dU * lu0) + np.sum(dS * ls0)
    assert abs(jv - rhs) <= 1e-9 * (abs(jv) + 1.0)
    # the final states equal the forward rollout's
    Un, Sn = OS.rollout_scalar(U, S, p, D, n, model=mdl)
    states, _ = T.rollout_scalar_states(U, S, p, D, n, mdl)
    assert np.abs(states[n][0] - Un).max() < 1e-13 and np.abs(states[n][1] - Sn).max() < 1e-13
    # a correction-network weight by central differences
    def loss(m):
        st, _ = T.rollout_scalar_states(U, S, p, D, n, m)
        return sum(np.sum(st[k][0] * lu[k - 1]) + np.sum(st[k][1] * ls[k - 1]) for k in range(1, n + 1))

    idx = (1, 3, 0, 2)
    def bump(s):
        tc = [(W.copy(), b.copy()) for W, b in mdl.tc]
        tc[0][0][idx] += s
        return O.LearnedModel(W_L=mdl.W_L, stencil=mdl.stencil, W_Ls=mdl.W_Ls, k_c=kc, tc=tc)
    fd = (loss(bump(eps)) - loss(bump(-eps))) / (2 * eps)
    assert abs(fd - g["tc"][0][0][idx]) <= 1e-6 * max(1e-2, abs(fd))
