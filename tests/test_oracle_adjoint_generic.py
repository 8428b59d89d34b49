"""Pins of the adjoint oracle on the grids of the generic-grid path (CPU):
non-power-of-two and rectangular grids with unequal spacings, where a swapped
dx / dy, a transposed operand or a wrong wrap in the reverse mode would cancel
on a square grid. Dot products against a fourth-order finite-difference JVP,
central differences on the learnable parameters (W_L entries of both axes, a
network weight and bias), for the plain and the learned step, both ablation
variants of the stencil path, Burgers and Navier-Stokes, and the temporal
correction."""

import numpy as np
import pytest

import oracle as O
from oracle import adjoint as A
from paper_2507_01975_gb300 import inputs as I


def fd4_jvp(f, x, d, eps):
    return (-f(x + 2 * eps * d) + 8 * f(x + eps * d) - 8 * f(x - eps * d) + f(x - 2 * eps * d)) / (12 * eps)


def narrow_model(seed, kc=0, ablation=0):
    st = I.random_conv_stack(seed, 2, 8, O.N_COEF, last_scale=0.2)
    tc = I.random_conv_stack(seed + 1, 2 * kc, 8, 2, last_scale=0.05) if kc else []
    return O.LearnedModel(W_L=I.random_wl(seed + 2, 2e-2), stencil=st, tc=tc, k_c=kc, ablation=ablation)


def smooth(nx, ny, seed, ncomp=2):
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.arange(ny) / ny, np.arange(nx) / nx, indexing="ij")
    out = np.zeros((ncomp, ny, nx))
    for c in range(ncomp):
        for _ in range(4):
            kx, ky = rng.integers(-2, 3, size=2)
            out[c] += rng.standard_normal() * np.sin(2 * np.pi * (kx * x + ky * y) + rng.uniform(0, 2 * np.pi))
    return out


CASES = {
    # Burgers on an odd, rectangular grid with unequal spacings
    "burgers13x9": dict(nx=13, ny=9, lx=1.0, ly=0.8, nu=1e-2, dt=2e-3, flow=O.FLOW_BURGERS),
    # Navier-Stokes on a rectangular power-of-two grid with unequal spacings
    "ns16x8": dict(nx=16, ny=8, lx=2.0, ly=1.3, nu=1e-2, dt=1e-2, flow=O.FLOW_NAVIER_STOKES),
}


def setup(case, seed):
    p = O.Problem(**CASES[case])
    U = 0.5 * smooth(p.nx, p.ny, seed)
    if p.flow == O.FLOW_NAVIER_STOKES:
        U = O.project(U, p)
    return p, U


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("learned", [False, True])
def test_step_dot_product_on_rectangular_grids(case, learned):
    p, U = setup(case, 3)
    rng = np.random.default_rng(4)
    du = rng.standard_normal(U.shape)
    if p.flow == O.FLOW_NAVIER_STOKES:
        du = O.project(du, p)
    lam = rng.standard_normal(U.shape)
    model = narrow_model(5) if learned else None
    f = (lambda x: O.learned_step(x, p, model)) if learned else (lambda x: O.rk4_step(x, p))
    jv = fd4_jvp(f, U, du, 1e-3)
    lam_in, _ = A.step_vjp(U, p, lam, model)
    lhs, rhs = np.sum(jv * lam), np.sum(du * lam_in)
    assert abs(lhs - rhs) <= 1e-10 * np.abs(jv * lam).sum()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("ablation", [0, 1])
def test_parameter_gradients_on_rectangular_grids(case, ablation):
    p, U = setup(case, 6)
    model = narrow_model(7, ablation=ablation)
    lam = np.random.default_rng(8).standard_normal(U.shape)
    _, (wlb, grads) = A.step_vjp(U, p, lam, model)

    def loss(mod):
        return np.sum(O.learned_step(U, p, mod) * lam)

    def with_wl(idx, s):
        wl = model.W_L.copy()
        wl[idx] += s
        return O.LearnedModel(W_L=wl, stencil=model.stencil, ablation=ablation)

    def with_w(l, idx, s, bias=False):
        st = [(W.copy(), b.copy()) for W, b in model.stencil]
        (st[l][1] if bias else st[l][0])[idx] += s
        return O.LearnedModel(W_L=model.W_L, stencil=st, ablation=ablation)

    eps = 1e-3
    # W_L of both kinds and both axes: the y-axis derivative part carries 1/dy
    for idx in [(0, 0, 2, 1), (1, 0, 1, 3), (0, 1, 4, 0), (1, 1, 2, 2)]:
        fd = (loss(with_wl(idx, eps)) - loss(with_wl(idx, -eps))) / (2 * eps)
        assert abs(fd - wlb[idx]) <= 1e-6 * max(1e-2, abs(fd)), (idx, fd, wlb[idx])
    for l, idx in [(0, (2, 1, 0, 2)), (5, (63, 4, 2, 1)), (5, (130, 7, 0, 0))]:
        fd = (loss(with_w(l, idx, eps)) - loss(with_w(l, idx, -eps))) / (2 * eps)
        assert abs(fd - grads[l][0][idx]) <= 1e-6 * max(1e-2, abs(fd)), (l, idx, fd, grads[l][0][idx])
    fd = (loss(with_w(5, (97,), eps, True)) - loss(with_w(5, (97,), -eps, True))) / (2 * eps)
    assert abs(fd - grads[5][1][97]) <= 1e-6 * max(1e-2, abs(fd))


@pytest.mark.parametrize("case", list(CASES))
def test_temporal_correction_vjp_on_rectangular_grids(case):
    p, U = setup(case, 9)
    kc = 2
    model = narrow_model(11, kc=kc)
    hist = [0.5 * smooth(p.nx, p.ny, 20 + s) for s in range(kc)]
    rng = np.random.default_rng(12)
    gbar = rng.standard_normal(U.shape)
    Vbar, hbar, tc_grads = A.temporal_correction_vjp(U, hist, p, model, gbar)[:3]
    # the state and every history state, by a JVP dot product
    dU = rng.standard_normal(U.shape)
    dh = [rng.standard_normal(U.shape) for _ in range(kc)]

    def f(t):
        return O.temporal_correction(U + t * dU, [h + t * d for h, d in zip(hist, dh)], p, model)

    eps = 1e-3
    jv = (-f(2 * eps) + 8 * f(eps) - 8 * f(-eps) + f(-2 * eps)) / (12 * eps)
    lhs = np.sum(jv * gbar)
    rhs = np.sum(dU * Vbar) + sum(np.sum(d * hb) for d, hb in zip(dh, hbar))
    assert abs(lhs - rhs) <= 1e-9 * np.abs(jv * gbar).sum()

    def with_tc(l, idx, s):
        tc = [(W.copy(), b.copy()) for W, b in model.tc]
        tc[l][0][idx] += s
        return O.LearnedModel(W_L=model.W_L, stencil=model.stencil, tc=tc, k_c=kc)

    for l, idx in [(0, (3, 2, 1, 0)), (5, (1, 6, 2, 2))]:
        fd = (np.sum(O.temporal_correction(U, hist, p, with_tc(l, idx, eps)) * gbar) -
              np.sum(O.temporal_correction(U, hist, p, with_tc(l, idx, -eps)) * gbar)) / (2 * eps)
        assert abs(fd - tc_grads[l][0][idx]) <= 1e-6 * max(1e-2, abs(fd))
