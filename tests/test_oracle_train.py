"""Pins of the training oracle (CPU): closed forms of the face average, the
divergence it preserves, the rollout reverse mode against a finite-difference
directional derivative, and Adam against its first-step closed form."""

import math

import numpy as np

import oracle as O
from oracle import train as T
from paper_2507_01975_gb300 import inputs as I


def test_face_average_of_taylor_green_is_dirichlet_kernel_closed_form():
    # u = sin x cos y sampled at fine west faces; the mean over r fine rows of a
    # coarse face is sin(X) cos(Y_c) sin(r h / 2) / (r sin(h / 2)) with Y_c the
    # coarse face centre (a geometric sum of exponentials)
    n, r = 64, 8
    U = I.taylor_green(n)
    C = T.face_average(U, r)
    h, H = 2 * math.pi / n, 2 * math.pi / (n // r)
    damp = math.sin(r * h / 2) / (r * math.sin(h / 2))
    (xu, yu), (xv, yv) = I.face_coords(n // r, n // r)
    assert np.max(np.abs(C[0] - np.sin(xu) * np.cos(yu) * damp)) < 1e-13
    assert np.max(np.abs(C[1] + np.cos(xv) * np.sin(yv) * damp)) < 1e-13
    assert abs(H - r * h) < 1e-15


def test_face_average_keeps_divergence_free_fields_divergence_free():
    n, r = 32, 4
    p = O.Problem(nx=n, ny=n)
    U = O.project(np.random.default_rng(1).standard_normal((2, n, n)), p)
    assert np.max(np.abs(O.divergence(U, p.dx, p.dy))) < 1e-11
    C = T.face_average(U, r)
    assert np.max(np.abs(O.divergence(C, r * p.dx, r * p.dy))) < 1e-11
    # and a constant field is reproduced
    K = np.ones((2, n, n)) * np.array([0.3, -1.2])[:, None, None]
    assert np.allclose(T.face_average(K, r), np.ones((2, n // r, n // r)) * np.array([0.3, -1.2])[:, None, None])


def test_mse_loss_gradient_is_exact():
    rng = np.random.default_rng(2)
    a, b = rng.standard_normal((2, 3, 5))
    loss, g = T.mse_loss(a, b)
    assert abs(loss - np.sum((a - b) ** 2) / a.size) < 1e-15
    d = rng.standard_normal(a.shape)
    fd = (T.mse_loss(a + 1e-6 * d, b)[0] - T.mse_loss(a - 1e-6 * d, b)[0]) / 2e-6
    assert abs(fd - np.sum(g * d)) < 1e-8


def test_rollout_vjp_dot_product():
    n = 16
    p = O.Problem(nx=n, ny=n, nu=0.02, dt=0.02, forcing_kind=1)
    U = I.kolmogorov_ic(n, 5)
    rng = np.random.default_rng(3)
    du = O.project(rng.standard_normal(U.shape), p)
    lam_traj = rng.standard_normal((3,) + U.shape)

    def traj(x):
        out, s = [], x
        for _ in range(3):
            s = O.rk4_step(s, p)
            out.append(s)
        return np.stack(out)

    eps = 1e-3
    jv = (-traj(U + 2 * eps * du) + 8 * traj(U + eps * du) - 8 * traj(U - eps * du) + traj(U - 2 * eps * du)) / (12 * eps)
    lam0, _ = T.rollout_vjp(U, p, 3, lam_traj)
    lhs, rhs = np.sum(jv * lam_traj), np.sum(du * lam0)
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_adam_first_step_moves_each_parameter_by_lr():
    # with zero moments the bias-corrected first step is -lr g / (|g| + eps)
    rng = np.random.default_rng(4)
    p, g = rng.standard_normal(10), rng.standard_normal(10)
    q, m, v = T.adam_step(p, g, np.zeros(10), np.zeros(10), 1, lr=1e-3, eps=1e-8)
    assert np.allclose(q - p, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # a constant gradient keeps the step at lr (bias corrections cancel the decay)
    for t in range(2, 6):
        q2, m, v = T.adam_step(q, g, m, v, t, lr=1e-3, eps=0.0)
        assert np.allclose(q2 - q, -1e-3 * np.sign(g), rtol=1e-12, atol=1e-15)
        q = q2
