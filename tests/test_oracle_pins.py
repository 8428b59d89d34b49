"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test checks the oracle against something the paper or the mathematics
fixes: Fourier symbols of the printed stencils, convergence orders, closed-form
solutions (Taylor-Green, Cole-Hopf Burgers, the Kolmogorov laminar state, a
single decaying shear mode), exact discrete invariants (divergence after the
projection, mean momentum), a dense direct Poisson solve on an 8x8 grid, and
brute-force convolution loops.
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_2507_01975_gb300 import inputs as I


def prob(n, **kw):
    return O.Problem(nx=n, ny=n, **kw)


# ----------------------------------------------------------------------------
# face operators: symbols on single Fourier modes (App. B.2 kernels)
# ----------------------------------------------------------------------------
# output location of each instance relative to the input grid, in cells:
# centre outputs sit half a cell after the u (x) / v (y) samples, corners half before.
@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("q", range(8))
def test_instance_symbols(q, order):
    n = 16
    p = prob(n, deriv_order=order)
    h = p.dx
    fld, axis, kind, shift = O.INSTANCES[q]
    kx, ky = 3, 2
    (xu, yu), (xv, yv) = I.face_coords(n, n)
    x, y = (xu, yu) if fld == 0 else (xv, yv)
    f = np.exp(1j * (kx * x + ky * y))
    U = np.zeros((2, n, n), dtype=complex)
    U[fld] = f
    out = O.face_values(U, O.plain_kernels(p))[q]
    # output location: shift -1 -> +1/2 cell along the axis, shift -2 -> -1/2 cell
    off = 0.5 if shift == -1 else -0.5
    k = kx if axis == 0 else ky
    if axis == 0:
        xo, yo = x + off * h, y
    else:
        xo, yo = x, y + off * h
    th = k * h
    if kind == 0:
        sym = math.cos(th / 2)
    elif order == 4:
        sym = 1j * (27 * math.sin(th / 2) - math.sin(3 * th / 2)) / (12 * h)
    else:
        sym = 2j * math.sin(th / 2) / h
    expect = sym * np.exp(1j * (kx * xo + ky * yo))
    assert np.max(np.abs(out - expect)) < 1e-12 * max(1.0, abs(sym))


@pytest.mark.parametrize("kind,order,expect", [(0, 2, 2.0), (1, 4, 4.0), (1, 2, 2.0)])
def test_operator_order_of_accuracy(kind, order, expect):
    errs = []
    for n in (16, 32, 64):
        p = prob(n, deriv_order=order)
        (xu, yu), _ = I.face_coords(n, n)
        g = np.exp(np.sin(xu)) * np.cos(yu)
        U = np.stack([g, np.zeros_like(g)])
        q = 0 if kind == 0 else 1
        out = O.face_values(U, O.plain_kernels(p))[q]
        xc = xu + 0.5 * p.dx
        exact = (np.exp(np.sin(xc)) if kind == 0 else np.cos(xc) * np.exp(np.sin(xc))) * np.cos(yu)
        errs.append(np.max(np.abs(out - exact)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert abs(rates[-1] - expect) < 0.15, rates


# ----------------------------------------------------------------------------
# projection (App. B.3, B.4)
# ----------------------------------------------------------------------------
def test_projection_divergence_free_idempotent_symmetric():
    n = 32
    p = prob(n)
    rng = np.random.default_rng(1)
    a = rng.standard_normal((2, n, n))
    b = rng.standard_normal((2, n, n))
    Pa = O.project(a, p)
    assert np.max(np.abs(O.divergence(Pa, p.dx, p.dy))) < 1e-12 * np.max(np.abs(a)) / p.dx
    assert np.max(np.abs(O.project(Pa, p) - Pa)) < 1e-13
    lhs = np.sum(Pa * b)
    rhs = np.sum(a * O.project(b, p))
    assert abs(lhs - rhs) < 1e-12 * np.sum(np.abs(a) * np.abs(b))


def test_projection_rectangular_grid_against_dense_solve():
    """On a rectangular 12 x 8 grid with unequal spacings the spectral projection
    equals the projection with the Poisson system solved densely: D2 and G2
    assembled entry by entry, the zero-mean constraint appended, least squares."""
    nx, ny, lx, ly = 12, 8, 3.0, 4.0
    p = O.Problem(nx=nx, ny=ny, lx=lx, ly=ly)
    dx, dy = lx / nx, ly / ny
    rng = np.random.default_rng(13)
    U = rng.standard_normal((2, ny, nx))
    N = nx * ny
    c = lambda j, i: (j % ny) * nx + (i % nx)
    D = np.zeros((N, 2 * N))
    G = np.zeros((2 * N, N))
    for j in range(ny):
        for i in range(nx):
            D[c(j, i), c(j, i + 1)] += 1 / dx
            D[c(j, i), c(j, i)] -= 1 / dx
            D[c(j, i), N + c(j + 1, i)] += 1 / dy
            D[c(j, i), N + c(j, i)] -= 1 / dy
            G[c(j, i), c(j, i)] += 1 / dx
            G[c(j, i), c(j, i - 1)] -= 1 / dx
            G[N + c(j, i), c(j, i)] += 1 / dy
            G[N + c(j, i), c(j - 1, i)] -= 1 / dy
    A = np.vstack([D @ G, np.ones((1, N))])
    rhs = np.concatenate([D @ U.reshape(-1), [0.0]])
    pc = np.linalg.lstsq(A, rhs, rcond=None)[0]
    want = U.reshape(-1) - G @ pc
    got = O.project(U, p).reshape(-1)
    assert np.abs(got - want).max() < 1e-11
    assert np.abs(D @ got).max() < 1e-11


def _dense_ops(n, h):
    """D2 and G2 written out as dense matrices by index arithmetic."""
    N = n * n
    D = np.zeros((N, 2 * N))
    G = np.zeros((2 * N, N))
    c = lambda j, i: (j % n) * n + (i % n)
    for j in range(n):
        for i in range(n):
            r = c(j, i)
            # div at centre (i, j): u[j, i+1] - u[j, i] + v[j+1, i] - v[j, i]
            D[r, c(j, i + 1)] += 1 / h
            D[r, c(j, i)] -= 1 / h
            D[r, N + c(j + 1, i)] += 1 / h
            D[r, N + c(j, i)] -= 1 / h
            # gradient: u-face (i, j) between centres (i-1, j) and (i, j)
            G[c(j, i), c(j, i)] += 1 / h
            G[c(j, i), c(j, i - 1)] -= 1 / h
            G[N + c(j, i), c(j, i)] += 1 / h
            G[N + c(j, i), c(j - 1, i)] -= 1 / h
    return D, G


def _gauss_solve(A, b):
    """Gaussian elimination with partial pivoting (no library solver)."""
    A = A.copy()
    b = b.copy()
    m = len(b)
    for k in range(m):
        piv = k + int(np.argmax(np.abs(A[k:, k])))
        A[[k, piv]] = A[[piv, k]]
        b[[k, piv]] = b[[piv, k]]
        for r in range(k + 1, m):
            f = A[r, k] / A[k, k]
            A[r, k:] -= f * A[k, k:]
            b[r] -= f * b[k]
    x = np.zeros(m)
    for k in range(m - 1, -1, -1):
        x[k] = (b[k] - A[k, k + 1:] @ x[k + 1:]) / A[k, k]
    return x


def test_dense_8x8_poisson_and_projection():
    n = 8
    p = prob(n)
    h = p.dx
    D, G = _dense_ops(n, h)
    rng = np.random.default_rng(7)
    w = rng.standard_normal((2, n, n))
    rhs = D @ w.reshape(-1)
    # bordered system [L 1; 1^T 0] [p; lam] = [rhs; 0] fixes the mean of p to zero
    N = n * n
    A = np.zeros((N + 1, N + 1))
    A[:N, :N] = D @ G
    A[:N, N] = 1.0
    A[N, :N] = 1.0
    sol = _gauss_solve(A, np.concatenate([rhs, [0.0]]))
    p_dense = sol[:N].reshape(n, n)
    p_fft = O.poisson_solve(O.divergence(w, h, h), p)
    assert np.max(np.abs(p_fft - p_dense)) < 1e-12 * max(1.0, np.max(np.abs(p_dense)))
    w_dense = w - (G @ sol[:N]).reshape(2, n, n)
    assert np.max(np.abs(O.project(w, p) - w_dense)) < 1e-12
    # library cross-check of the same bordered system
    sol2 = np.linalg.solve(A, np.concatenate([rhs, [0.0]]))
    assert np.max(np.abs(sol2[:N].reshape(n, n) - p_dense)) < 1e-12


def test_continuous_symbol_projection_leaves_small_divergence():
    # paper-literal continuous symbol: not the inverse of D2 G2, so the residual
    # divergence is O(h^2) for a smooth field, and zero for the matched symbol
    res = []
    for n in (16, 32, 64):
        p = prob(n, poisson_symbol=1)
        (xu, yu), (xv, yv) = I.face_coords(n, n)
        w = np.stack([np.sin(xu) * np.cos(2 * yu), np.cos(xv) * np.sin(yv)])
        res.append(np.max(np.abs(O.divergence(O.project(w, p), p.dx, p.dy))))
    assert res[0] > 1e-6
    assert abs(math.log2(res[1] / res[2]) - 2.0) < 0.2


# ----------------------------------------------------------------------------
# time integration: single decaying shear mode, exact RK4 amplification
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("order", [2, 4])
def test_shear_mode_rk4_amplification_exact(order):
    n, k, nu, dt, steps = 16, 2, 0.05, 0.05, 10
    p = prob(n, nu=nu, dt=dt, deriv_order=order)
    (xu, yu), _ = I.face_coords(n, n)
    U = np.stack([np.sin(k * yu), np.zeros((n, n))])
    out, _ = O.rollout(U, p, steps)
    h = p.dy
    th = k * h
    if order == 4:
        dcorner = (27 * math.sin(th / 2) - math.sin(3 * th / 2)) / (12 * h)
    else:
        dcorner = 2 * math.sin(th / 2) / h
    lam = -nu * dcorner * 2 * math.sin(th / 2) / h
    z = lam * dt
    R = 1 + z + z * z / 2 + z**3 / 6 + z**4 / 24
    assert np.max(np.abs(out[0] - R**steps * U[0])) < 1e-13
    assert np.max(np.abs(out[1])) < 1e-14


def test_rk4_temporal_order_four():
    # Burgers, smooth field, Richardson in dt: error(dt) / error(dt/2) ~ 16
    n = 16
    U0 = I.burgers_ic(n, 3)
    T = 0.2

    def run(dt):
        p = prob(n, nu=0.05, dt=dt, flow=O.FLOW_BURGERS, deriv_order=2)
        return O.rollout(U0, p, int(round(T / dt)))[0]

    ref = run(0.0125 / 8)
    e1 = np.max(np.abs(run(0.05) - ref))
    e2 = np.max(np.abs(run(0.025) - ref))
    assert 3.6 < math.log2(e1 / e2) < 4.4


# ----------------------------------------------------------------------------
# full Navier-Stokes step: Taylor-Green closed form
# ----------------------------------------------------------------------------
def test_taylor_green_decay_second_order():
    nu, T = 0.1, 0.25
    errs = []
    for n in (16, 32, 64):
        dt = 0.025 * 16 / n
        p = prob(n, nu=nu, dt=dt)
        out, _ = O.rollout(I.taylor_green(n), p, int(round(T / dt)))
        errs.append(np.max(np.abs(out - I.taylor_green(n, T, nu))))
    rate = math.log2(errs[1] / errs[2])
    assert errs[2] < 2e-3
    assert 1.8 < rate < 2.3, (errs, rate)


def test_taylor_green_stays_divergence_free():
    n = 32
    p = prob(n, nu=0.01, dt=0.01)
    out, _ = O.rollout(I.taylor_green(n), p, 5)
    assert np.max(np.abs(O.divergence(out, p.dx, p.dy))) < 1e-12


# ----------------------------------------------------------------------------
# conservation of mean momentum (periodic box, flux form)
# ----------------------------------------------------------------------------
def test_decaying_mean_momentum_conserved():
    n = 32
    p = prob(n, nu=1e-3, dt=5e-3)
    U0 = I.decaying_ic(n, 2) + np.array([0.3, -0.2])[:, None, None]
    out, _ = O.rollout(U0, p, 10)
    for c in range(2):
        assert abs(out[c].sum() - U0[c].sum()) < 1e-13 * np.abs(U0[c]).sum()


def test_forced_mean_momentum_follows_drag():
    n, dt, steps = 32, 5e-3, 10
    p = prob(n, nu=1e-3, dt=dt, forcing_kind=1)
    U0 = I.kolmogorov_ic(n, 4) + np.array([0.5, 0.25])[:, None, None]
    out, _ = O.rollout(U0, p, steps)
    z = -0.1 * dt
    R = 1 + z + z * z / 2 + z**3 / 6 + z**4 / 24
    for c in range(2):
        expect = U0[c].sum() * R**steps
        assert abs(out[c].sum() - expect) < 1e-12 * np.abs(U0[c]).sum()


def test_kolmogorov_laminar_fixed_point():
    n, nu = 32, 1e-3
    p = prob(n, nu=nu, dt=0.01, forcing_kind=1)
    h = p.dy
    th = 4 * h
    dcorner = (27 * math.sin(th / 2) - math.sin(3 * th / 2)) / (12 * h)
    sigma = -dcorner * 2 * math.sin(th / 2) / h
    A = 1.0 / (-nu * sigma + 0.1)
    assert abs(A - 1 / (16 * nu + 0.1)) < 0.01 * A  # near the continuum 8.62
    (xu, yu), _ = I.face_coords(n, n)
    U = np.stack([A * np.sin(4 * yu), np.zeros((n, n))])
    out = O.rk4_step(U, p)
    assert np.max(np.abs(out - U)) < 1e-14 * A


# ----------------------------------------------------------------------------
# Burgers: Cole-Hopf closed form
# ----------------------------------------------------------------------------
def _cole_hopf_1d(x, t, nu, A, nterms=80):
    """u(x, t) for u0 = -A sin x: theta0 = exp(-a cos x), a = A / (2 nu)."""
    from scipy.special import ive

    a = A / (2 * nu)
    g = ive(0, a) * np.ones_like(x)
    gx = np.zeros_like(x)
    for m in range(1, nterms):
        c = 2 * (-1) ** m * ive(m, a) * math.exp(-nu * m * m * t)
        g = g + c * np.cos(m * x)
        gx = gx - c * m * np.sin(m * x)
    return -2 * nu * gx / g


@pytest.mark.parametrize("order", [2, 4])
def test_burgers_cole_hopf_second_order(order):
    nu, A, T = 0.05, 0.5, 0.5
    errs = []
    for n in (16, 32, 64):
        dt = 0.02 * 16 / n
        p = prob(n, nu=nu, dt=dt, flow=O.FLOW_BURGERS, deriv_order=order)
        (xu, yu), (xv, yv) = I.face_coords(n, n)
        U0 = np.stack([-A * np.sin(xu), -A * np.sin(yv)])
        out, _ = O.rollout(U0, p, int(round(T / dt)))
        exact = np.stack([_cole_hopf_1d(xu, T, nu, A), _cole_hopf_1d(yv, T, nu, A)])
        errs.append(np.max(np.abs(out - exact)))
    rate = math.log2(errs[1] / errs[2])
    assert 1.8 < rate < 2.3, (errs, rate)
    assert errs[2] < 2e-3


def test_burgers_cole_hopf_rectangular_grid():
    """Cole-Hopf on a non-power-of-two rectangular grid (48 x 40 cells): u depends on
    x only and v on y only, so each component is the 1D closed form on its own axis;
    the error lies between those of the square 32^2 and 64^2 runs (second order)."""
    nu, A, T = 0.05, 0.5, 0.5

    def err(nx, ny):
        dt = 0.02 * 16 / max(nx, ny)
        p = O.Problem(nx=nx, ny=ny, nu=nu, dt=dt, flow=O.FLOW_BURGERS, deriv_order=4)
        (xu, yu), (xv, yv) = I.face_coords(nx, ny)
        U0 = np.stack([-A * np.sin(xu), -A * np.sin(yv)])
        out, _ = O.rollout(U0, p, int(round(T / dt)))
        return (np.max(np.abs(out[0] - _cole_hopf_1d(xu, T, nu, A))),
                np.max(np.abs(out[1] - _cole_hopf_1d(yv, T, nu, A))))

    e32, e64 = max(err(32, 32)), max(err(64, 64))
    eu, ev = err(48, 40)
    assert e64 < eu < e32 and e64 < ev < e32, (eu, ev, e32, e64)
    assert ev > eu  # v lives on the coarser axis (40 cells)


@pytest.mark.parametrize("flow", [O.FLOW_BURGERS, O.FLOW_NAVIER_STOKES])
def test_axis_transposition_symmetry(flow):
    """Swapping the axes (x <-> y with u <-> v, nx <-> ny, lx <-> ly) maps a step onto
    the transposed step: u-faces and v-faces trade places and every instance keeps its
    offsets. On a rectangular non-power-of-two grid this catches any nx / ny mix-up."""
    nx, ny, lx, ly = 12, 20, 3.0, 4.0
    rng = np.random.default_rng(12)
    U = rng.standard_normal((2, ny, nx)) * 0.3
    pa = O.Problem(nx=nx, ny=ny, lx=lx, ly=ly, nu=0.02, dt=2e-3, flow=flow)
    pb = O.Problem(nx=ny, ny=nx, lx=ly, ly=lx, nu=0.02, dt=2e-3, flow=flow)
    if flow == O.FLOW_NAVIER_STOKES:
        U = O.project(U, pa)
    a = O.rk4_step(U, pa)
    b = O.rk4_step(np.stack([U[1].T, U[0].T]), pb)
    assert np.abs(np.stack([b[1].T, b[0].T]) - a).max() < 1e-13


# ----------------------------------------------------------------------------
# symmetry
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("flow", [O.FLOW_BURGERS, O.FLOW_NAVIER_STOKES])
def test_translation_equivariance(flow):
    n = 16
    p = prob(n, nu=0.01, dt=0.01, flow=flow)
    U = I.decaying_ic(n, 5)
    a = O.rk4_step(np.roll(U, (1, 2), axis=(1, 2)), p)
    b = np.roll(O.rk4_step(U, p), (1, 2), axis=(1, 2))
    assert np.max(np.abs(a - b)) < 1e-13


def test_reflection_x_plain():
    # x -> -x maps a u-face i to u-face -i and a v-face i to v-face -1-i,
    # with u -> -u
    n = 16
    p = prob(n, nu=0.01, dt=0.01)
    U = I.decaying_ic(n, 6)

    def refl(W):
        u = -np.roll(W[0][:, ::-1], 1, axis=1)
        v = W[1][:, ::-1]
        return np.stack([u, v])

    a = O.rk4_step(refl(U), p)
    b = refl(O.rk4_step(U, p))
    assert np.max(np.abs(a - b)) < 1e-13


# ----------------------------------------------------------------------------
# learnable module
# ----------------------------------------------------------------------------
def test_conv3x3_matches_brute_force_and_delta():
    rng = np.random.default_rng(3)
    ci, co, n = 3, 4, 6
    x = rng.standard_normal((ci, n, n))
    W = rng.standard_normal((co, ci, 3, 3))
    b = rng.standard_normal(co)
    out = O.conv3x3(x, W, b)
    ref = np.zeros((co, n, n))
    for o in range(co):
        for j in range(n):
            for i in range(n):
                s = b[o]
                for c in range(ci):
                    for a in range(3):
                        for e in range(3):
                            s += W[o, c, a, e] * x[c, (j + a - 1) % n, (i + e - 1) % n]
                ref[o, j, i] = s
    assert np.max(np.abs(out - ref)) < 1e-12
    # cross-correlation: a delta at (j0, i0) reproduces the kernel flipped
    d = np.zeros((1, n, n))
    d[0, 3, 3] = 1.0
    k = rng.standard_normal((1, 1, 3, 3))
    o = O.conv3x3(d, k, np.zeros(1))
    assert np.allclose(o[0, 2:5, 2:5], k[0, 0, ::-1, ::-1])


def test_gelu_and_grad():
    x = np.linspace(-4, 4, 101)
    g = O.gelu(x)
    assert abs(O.gelu(np.array([0.0]))[0]) == 0.0
    assert np.all(np.abs(g[x > 3.5] - x[x > 3.5]) < 1e-3)
    eps = 1e-6
    fd = (O.gelu(x + eps) - O.gelu(x - eps)) / (2 * eps)
    assert np.max(np.abs(fd - O.gelu_grad(x))) < 1e-8


def test_consistency_projection_moments():
    rng = np.random.default_rng(11)
    L = rng.standard_normal((5, 4, 3, 2))
    P = O.consistency_project(L)
    c = O.AXIAL[None, :, None, None]
    r = O.TRANSVERSE[:, None, None, None]
    assert np.max(np.abs(P.sum(axis=(0, 1)))) < 1e-14
    assert np.max(np.abs((P * c).sum(axis=(0, 1)))) < 1e-14
    assert np.max(np.abs((P * r).sum(axis=(0, 1)))) < 1e-14
    assert np.max(np.abs(O.consistency_project(P) - P)) < 1e-14
    # W_P + projected part still interpolates / differentiates linear data exactly
    h = 0.3
    for kind in (0, 1):
        K = O.physics_kernel(kind, 4, h)[:, :, None, None] + (P / h if kind else P)
        lin = 0.7 + 1.3 * (c * h) + 0.4 * (r * h)  # f = 0.7 + 1.3 s + 0.4 t
        val = (K * lin).sum(axis=(0, 1))
        assert np.max(np.abs(val - (0.7 if kind == 0 else 1.3))) < 1e-12


def _zero_model(n):
    st = I.random_conv_stack(0, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=0.0)
    return O.LearnedModel(W_L=np.zeros((2, 2, 5, 4)), stencil=st)


def test_learned_reduces_to_plain_bit_for_bit():
    n = 16
    p = prob(n, nu=0.01, dt=0.01)
    U = I.decaying_ic(n, 8)
    a = O.learned_step(U, p, _zero_model(n))
    b = O.rk4_step(U, p)
    assert np.array_equal(a, b)


def test_learned_translation_equivariance_and_conservation():
    n = 16
    p = prob(n, nu=0.01, dt=0.01)
    st = I.random_conv_stack(1, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=0.05)
    model = O.LearnedModel(W_L=I.random_wl(2), stencil=st)
    U = I.decaying_ic(n, 9) + np.array([0.2, 0.1])[:, None, None]
    a = O.learned_step(np.roll(U, (3, 1), axis=(1, 2)), p, model)
    out = O.learned_step(U, p, model)
    assert np.max(np.abs(a - np.roll(out, (3, 1), axis=(1, 2)))) < 1e-12
    for c in range(2):
        assert abs(out[c].sum() - U[c].sum()) < 1e-12 * np.abs(U[c]).sum()
    assert np.max(np.abs(O.divergence(out, p.dx, p.dy))) < 1e-11


def test_temporal_correction_keeps_mean_and_divergence():
    n = 16
    p = prob(n, nu=0.01, dt=0.01, forcing_kind=1)
    st = I.random_conv_stack(1, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=0.05)
    tc = I.random_conv_stack(5, 8, O.CNN_HIDDEN, 2, last_scale=0.5)
    model = O.LearnedModel(W_L=I.random_wl(2), stencil=st, tc=tc, k_c=4)
    U0 = I.kolmogorov_ic(n, 1)
    plain_model = O.LearnedModel(W_L=model.W_L, stencil=st)
    a, _ = O.rollout(U0, p, 4, model=model)
    b, _ = O.rollout(U0, p, 4, model=plain_model)
    assert np.max(np.abs(a - b)) > 1e-6  # the correction did something
    for c in range(2):
        assert abs(a[c].sum() - b[c].sum()) < 1e-12 * np.abs(b[c]).sum()
    assert np.max(np.abs(O.divergence(a, p.dx, p.dy))) < 1e-11


def test_vorticity_of_taylor_green_and_pcc():
    n = 32
    U = I.taylor_green(n)
    h = 2 * math.pi / n
    w = O.vorticity(U, h, h)
    x, y = np.meshgrid(np.arange(n) * h, np.arange(n) * h)
    # continuum vorticity of Taylor-Green: 2 sin x sin y (to O(h^2))
    assert np.max(np.abs(w - 2 * np.sin(x) * np.sin(y))) < 2e-2
    assert abs(O.pcc(w, 3 * w + 1) - 1.0) < 1e-14
    assert abs(O.pcc(w, -w) + 1.0) < 1e-14


# ----------------------------------------------------------------------------
# energy spectrum (Sec. 4, forced flow / Fig. 5): closed forms and Parseval
# ----------------------------------------------------------------------------
def test_shell_index_is_the_nearest_integer_root():
    q = np.arange(0, 200000)
    k = O.shell_index(q)
    # (k - 1/2)^2 <= q < (k + 1/2)^2 checked in exact integer arithmetic (x4)
    lo = np.maximum(2 * k - 1, 0)
    assert np.all(lo ** 2 <= 4 * q) and np.all(4 * q < (2 * k + 1) ** 2)


def test_energy_spectrum_single_modes_and_parseval():
    n = 32
    x = np.arange(n) * (2 * np.pi / n)
    X, Y = np.meshgrid(x, x)
    A = 0.7
    U = np.stack([A * np.cos(3 * X), np.zeros_like(X)])
    E = O.energy_spectrum(U, n)
    assert abs(E[3] - A * A / 4) < 1e-14 and np.abs(np.delete(E, 3)).max() < 1e-14
    # |k| = 5 from (kx, ky) = (3, 4), in v this time, shifted by half a cell
    U = np.stack([np.zeros_like(X), np.sin(3 * X + 4 * (Y + np.pi / n))])
    E = O.energy_spectrum(U, n)
    assert abs(E[5] - 0.25) < 1e-14 and np.abs(np.delete(E, 5)).max() < 1e-14
    # Parseval on a random field, and invariance under a periodic translation
    U = np.random.default_rng(5).standard_normal((2, n, n))
    E = O.energy_spectrum(U, n)
    assert abs(E.sum() - 0.5 * np.mean(U[0] ** 2 + U[1] ** 2)) < 1e-13
    Es = O.energy_spectrum(np.roll(U, (3, -5), axis=(1, 2)), n)
    assert np.abs(Es - E).max() < 1e-14
    # shells beyond kmax are dropped, the rest unchanged
    assert np.abs(O.energy_spectrum(U, 7) - E[:8]).max() == 0.0
