"""Pins of the oracle's passive scalar (shear flow, App. C.1): closed forms for
uniform advection and pure diffusion of a Fourier mode, the RK4 amplification
factor, exact conservation, a constant scalar staying constant in any
divergence-free flow, and transposition / translation symmetry."""

import math

import numpy as np
import pytest

import oracle as O
from oracle.scalar import rk4_step_scalar, scalar_tendency
from paper_2507_01975_gb300 import inputs as I


def grid(nx=16, ny=12, lx=4.0, ly=3.0, **kw):
    return O.Problem(nx=nx, ny=ny, lx=lx, ly=ly, **kw)


def centres(p):
    return np.meshgrid((np.arange(p.nx) + 0.5) * p.dx, (np.arange(p.ny) + 0.5) * p.dy)


def test_uniform_advection_of_a_mode():
    """u = c: the linear face interpolation gives -c (s_{i+1} - s_{i-1}) / (2 dx), so
    for s = cos(k x) the tendency is c sin(k x) sin(k dx) / dx."""
    p = grid()
    x, y = centres(p)
    k, c = 2 * math.pi * 3 / p.lx, 0.7
    S = np.cos(k * x)
    U = np.stack([np.full((p.ny, p.nx), c), np.zeros((p.ny, p.nx))])
    got = scalar_tendency(U, S, p, 0.0)
    assert np.abs(got - c * np.sin(k * x) * math.sin(k * p.dx) / p.dx).max() < 1e-12


@pytest.mark.parametrize("order", [2, 4])
def test_pure_diffusion_of_a_mode(order):
    """u = 0: the face-derivative differences have the symbol
    -(2/h) sin(kh/2) g(k) with g = 2 sin(kh/2)/h (2nd order) or
    (27 sin(kh/2) - sin(3kh/2)) / (12 h) (4th order), per axis."""
    p = grid(deriv_order=order)
    x, y = centres(p)
    kx, ky = 2 * math.pi * 2 / p.lx, 2 * math.pi * 1 / p.ly
    S = np.cos(kx * x) * np.cos(ky * y)
    D = 0.01

    def lam(k, h):
        g = 2 * math.sin(k * h / 2) / h if order == 2 else (27 * math.sin(k * h / 2) - math.sin(1.5 * k * h)) / (12 * h)
        return -(2 / h) * math.sin(k * h / 2) * g

    got = scalar_tendency(np.zeros((2, p.ny, p.nx)), S, p, D)
    assert np.abs(got - D * (lam(kx, p.dx) + lam(ky, p.dy)) * S).max() < 1e-12


def test_rk4_amplification_factor():
    """Uniform advection of e^{ikx}: one step multiplies the mode by the RK4
    polynomial R(z), z = -i c dt sin(k dx) / dx."""
    p = grid(dt=0.05, flow=O.FLOW_BURGERS, nu=0.0)
    x, _ = centres(p)
    k, c = 2 * math.pi * 2 / p.lx, 0.8
    U = np.stack([np.full((p.ny, p.nx), c), np.zeros((p.ny, p.nx))])
    _, S1 = rk4_step_scalar(U, np.cos(k * x), p, 0.0)
    z = -1j * c * p.dt * math.sin(k * p.dx) / p.dx
    R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    assert np.abs(S1 - np.real(R * np.exp(1j * k * x))).max() < 1e-13


def test_conservation_and_constant_scalar():
    p = grid()
    rng = np.random.default_rng(3)
    U = rng.standard_normal((2, p.ny, p.nx))
    S = rng.standard_normal((p.ny, p.nx))
    assert abs(scalar_tendency(U, S, p, 0.01).sum()) < 1e-11 * np.abs(S).sum() / p.dx
    Up = O.project(U, p)
    assert np.abs(scalar_tendency(Up, np.full((p.ny, p.nx), 2.5), p, 0.01)).max() < 1e-11
    # a full step keeps the total scalar
    _, S1 = rk4_step_scalar(Up, S, dataclass_replace(p, dt=1e-2), 0.01)
    assert abs(S1.sum() - S.sum()) < 1e-11 * np.abs(S).sum()


def dataclass_replace(p, **kw):
    import dataclasses

    return dataclasses.replace(p, **kw)


def test_transposition_and_translation_symmetry():
    """Swapping the axes (u <-> v, nx <-> ny, lx <-> ly) transposes the scalar
    update; a periodic shift commutes with it."""
    pa = grid(nx=10, ny=14, lx=2.0, ly=3.5, dt=1e-2)
    pb = grid(nx=14, ny=10, lx=3.5, ly=2.0, dt=1e-2)
    rng = np.random.default_rng(4)
    U = O.project(rng.standard_normal((2, pa.ny, pa.nx)) * 0.3, pa)
    S = rng.standard_normal((pa.ny, pa.nx))
    Ua, Sa = rk4_step_scalar(U, S, pa, 0.02)
    Ub, Sb = rk4_step_scalar(np.stack([U[1].T, U[0].T]), S.T, pb, 0.02)
    assert np.abs(Sb.T - Sa).max() < 1e-13
    Us, Ss = rk4_step_scalar(np.roll(U, (2, 3), axis=(1, 2)), np.roll(S, (2, 3), axis=(0, 1)), pa, 0.02)
    assert np.abs(Ss - np.roll(Sa, (2, 3), axis=(0, 1))).max() < 1e-13


def test_shear_flow_initial_state():
    """The shear-flow state: periodic tanh layers, the scalar between 0 and 1 and
    aligned with them; after projection a few joint steps stay bounded and keep
    the total scalar."""
    U, S = I.shear_scalar_ic(64, 32, seed=1)
    assert U.shape == (2, 32, 64) and S.shape == (32, 64)
    assert S.min() > -1e-9 and S.max() < 1 + 1e-9
    p = O.Problem(nx=64, ny=32, lx=8.0, ly=4.0, nu=1e-3, dt=1e-2)
    U = O.project(U, p)
    total = S.sum()
    for _ in range(5):
        U, S = rk4_step_scalar(U, S, p, 0.001)
    assert abs(S.sum() - total) < 1e-10 * abs(total)
    assert np.abs(S).max() < 1.5


@pytest.mark.parametrize("flow", [O.FLOW_NAVIER_STOKES, O.FLOW_BURGERS])
def test_joint_step_vjp_dot_product(flow):
    """Reverse mode of the joint velocity-scalar step against a fourth-order
    finite-difference JVP of (u, s) -> (u', s')."""
    from oracle.adjoint import rk4_step_scalar_vjp, scalar_tendency_vjp

    p = grid(nx=10, ny=8, lx=2.5, ly=2.0, nu=0.02, dt=0.02, flow=flow)
    rng = np.random.default_rng(17)
    U = rng.standard_normal((2, p.ny, p.nx)) * 0.5
    if flow == O.FLOW_NAVIER_STOKES:
        U = O.project(U, p)
    S = rng.standard_normal((p.ny, p.nx))
    dU = rng.standard_normal(U.shape)
    if flow == O.FLOW_NAVIER_STOKES:
        dU = O.project(dU, p)
    dS = rng.standard_normal(S.shape)
    lamU, lamS = rng.standard_normal(U.shape), rng.standard_normal(S.shape)
    D, e = 0.01, 1e-3

    def f(t):
        u1, s1 = rk4_step_scalar(U + t * dU, S + t * dS, p, D)
        return np.sum(u1 * lamU) + np.sum(s1 * lamS)

    jvp = (-f(2 * e) + 8 * f(e) - 8 * f(-e) + f(-2 * e)) / (12 * e)
    Ub, Sb = rk4_step_scalar_vjp(U, S, p, D, lamU, lamS)
    assert abs(jvp - (np.sum(Ub * dU) + np.sum(Sb * dS))) <= 1e-10 * abs(jvp)
    # the tendency's reverse mode alone: a dot product in both arguments
    qb = rng.standard_normal(S.shape)
    g = lambda t: np.sum(scalar_tendency(U + t * dU, S + t * dS, p, D) * qb)
    jv = (-g(2 * e) + 8 * g(e) - 8 * g(-e) + g(-2 * e)) / (12 * e)
    tu, ts = scalar_tendency_vjp(U, S, p, D, qb)
    assert abs(jv - (np.sum(tu * dU) + np.sum(ts * dS))) <= 1e-10 * abs(jv)
