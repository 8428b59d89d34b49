"""Pins of the adjoint oracle (CPU): dot-product tests against a fourth-order
finite-difference Jacobian-vector product, and central differences on the
learnable parameters (epsilon = 1e-3, FP64)."""

import numpy as np
import pytest

import oracle as O
from oracle import adjoint as A
from paper_2507_01975_gb300 import inputs as I


def fd4_jvp(f, x, d, eps):
    """[-f(x+2ed) + 8 f(x+ed) - 8 f(x-ed) + f(x-2ed)] / (12 e): error O(e^4)."""
    return (-f(x + 2 * eps * d) + 8 * f(x + eps * d) - 8 * f(x - eps * d) + f(x - 2 * eps * d)) / (12 * eps)


def small_model(seed, n, last_scale=0.05):
    st = I.random_conv_stack(seed, 2, 8, O.N_COEF, last_scale=last_scale)  # narrow network keeps FD cheap
    return O.LearnedModel(W_L=I.random_wl(seed + 1, 1e-2), stencil=st)


@pytest.mark.parametrize("flow,forcing", [(O.FLOW_NAVIER_STOKES, 0), (O.FLOW_NAVIER_STOKES, 1), (O.FLOW_BURGERS, 0)])
def test_plain_step_dot_product(flow, forcing):
    n = 16
    p = O.Problem(nx=n, ny=n, nu=0.02, dt=0.02, flow=flow, forcing_kind=forcing)
    rng = np.random.default_rng(3)
    U = I.decaying_ic(n, 1) if flow == O.FLOW_NAVIER_STOKES else I.burgers_ic(n, 1)
    du = rng.standard_normal(U.shape)
    if flow == O.FLOW_NAVIER_STOKES:
        du = O.project(du, p)  # tangent directions of the divergence-free manifold
    lam = rng.standard_normal(U.shape)
    jv = fd4_jvp(lambda x: O.rk4_step(x, p), U, du, 1e-3)
    lam_in, _ = A.step_vjp(U, p, lam)
    lhs = np.sum(jv * lam)
    rhs = np.sum(du * lam_in)
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_tendency_kernel_gradient_matches_finite_differences():
    n = 8
    p = O.Problem(nx=n, ny=n, nu=0.05, dt=0.01)
    U = I.decaying_ic(n, 2)
    rng = np.random.default_rng(4)
    ks = [k[:, :, None, None] + 0.1 * rng.standard_normal((5, 4, n, n)) for k in O.plain_kernels(p)]
    Tb = rng.standard_normal(U.shape)
    _, Kbar = A.tendency_vjp(U, p, ks, Tb, want_kbar=True)
    for q, (r, c, j, i) in [(0, (2, 1, 3, 4)), (3, (0, 3, 7, 1)), (6, (4, 0, 2, 2))]:
        def L(eps, q=q, r=r, c=c, j=j, i=i):
            kk = [k.copy() for k in ks]
            kk[q][r, c, j, i] += eps
            return np.sum(O.tendency(U, p, kk) * Tb)
        fd = (L(1e-4) - L(-1e-4)) / 2e-4
        assert abs(fd - Kbar[q][r, c, j, i]) <= 1e-8 * max(1.0, abs(fd))


def test_cnn_vjp_dot_product_and_weight_gradient():
    n = 8
    layers = I.random_conv_stack(5, 2, 8, 6, last_scale=1.0)
    rng = np.random.default_rng(6)
    x = rng.standard_normal((2, n, n))
    dx = rng.standard_normal(x.shape)
    yb = rng.standard_normal((6, n, n))
    jv = fd4_jvp(lambda z: O.cnn_forward(z, layers), x, dx, 1e-3)
    xb, grads = A.cnn_vjp(x, layers, yb)
    assert abs(np.sum(jv * yb) - np.sum(dx * xb)) <= 1e-9 * np.abs(jv * yb).sum()
    for l, idx in [(0, (3, 1, 0, 2)), (2, (5, 7, 1, 1)), (5, (4, 2, 2, 0))]:
        def L(eps, l=l, idx=idx):
            ll = [(W.copy(), b.copy()) for W, b in layers]
            ll[l][0][idx] += eps
            return np.sum(O.cnn_forward(x, ll) * yb)
        fd = (L(1e-3) - L(-1e-3)) / 2e-3
        assert abs(fd - grads[l][0][idx]) <= 1e-5 * max(1.0, abs(fd))
    def Lb(eps):
        ll = [(W.copy(), b.copy()) for W, b in layers]
        ll[3][1][2] += eps
        return np.sum(O.cnn_forward(x, ll) * yb)
    fd = (Lb(1e-3) - Lb(-1e-3)) / 2e-3
    assert abs(fd - grads[3][1][2]) <= 1e-5 * max(1.0, abs(fd))


def test_learned_step_dot_product():
    n = 8
    p = O.Problem(nx=n, ny=n, nu=0.02, dt=0.02, forcing_kind=1)
    model = small_model(7, n)
    rng = np.random.default_rng(8)
    U = I.kolmogorov_ic(n, 3)
    du = O.project(rng.standard_normal(U.shape), p)
    lam = rng.standard_normal(U.shape)
    jv = fd4_jvp(lambda x: O.learned_step(x, p, model), U, du, 1e-3)
    lam_in, _ = A.step_vjp(U, p, lam, model)
    lhs, rhs = np.sum(jv * lam), np.sum(du * lam_in)
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_learned_step_parameter_gradients_central_differences():
    n = 8
    p = O.Problem(nx=n, ny=n, nu=0.02, dt=0.02)
    model = small_model(9, n)
    rng = np.random.default_rng(10)
    U = I.decaying_ic(n, 4)
    lam = rng.standard_normal(U.shape)
    _, (wlb, grads) = A.step_vjp(U, p, lam, model)

    def loss_with(mod):
        return np.sum(O.learned_step(U, p, mod) * lam)

    eps = 1e-3
    # W_L entries
    for idx in [(0, 0, 2, 1), (1, 1, 0, 3), (1, 0, 4, 2)]:
        def m(s, idx=idx):
            wl = model.W_L.copy()
            wl[idx] += s
            return O.LearnedModel(W_L=wl, stencil=model.stencil)
        fd = (loss_with(m(eps)) - loss_with(m(-eps))) / (2 * eps)
        assert abs(fd - wlb[idx]) <= 1e-5 * max(1e-3, abs(fd))
    # network weights and a bias
    for l, idx in [(0, (1, 0, 1, 1)), (3, (2, 5, 0, 2)), (5, (17, 3, 1, 1))]:
        def m(s, l=l, idx=idx):
            st = [(W.copy(), b.copy()) for W, b in model.stencil]
            st[l][0][idx] += s
            return O.LearnedModel(W_L=model.W_L, stencil=st)
        fd = (loss_with(m(eps)) - loss_with(m(-eps))) / (2 * eps)
        assert abs(fd - grads[l][0][idx]) <= 1e-5 * max(1e-3, abs(fd))


def test_adjoint_of_projection_is_projection():
    # P is symmetric: the reverse of "project" is "project"
    n = 16
    p = O.Problem(nx=n, ny=n)
    rng = np.random.default_rng(12)
    a, b = rng.standard_normal((2, 2, n, n))
    assert abs(np.sum(O.project(a, p) * b) - np.sum(a * O.project(b, p))) < 1e-12 * np.abs(a * b).sum()


@pytest.mark.parametrize("flow", [O.FLOW_NAVIER_STOKES, O.FLOW_BURGERS])
@pytest.mark.parametrize("head", ["cnn", "fno"])
def test_temporal_correction_vjp(flow, head):
    """Reverse mode of the temporal correction (CNN head and FNO): the dot product
    with a central-difference JVP in the state and every history state, and central
    differences on parameter entries."""
    from oracle.adjoint import temporal_correction_vjp
    from oracle.fno import FNOParams

    rng = np.random.default_rng(16)
    n, kc = 8, 3
    p = O.Problem(nx=n, ny=n, nu=1e-2, dt=1e-2, flow=flow)
    U = rng.standard_normal((2, n, n))
    hist = [rng.standard_normal((2, n, n)) for _ in range(kc)]
    m = O.LearnedModel(W_L=np.zeros((2, 2, 5, 4)), stencil=[], k_c=kc)
    if head == "cnn":
        m.tc = [(rng.standard_normal((4, 2 * kc, 3, 3)) * 0.3, rng.standard_normal(4) * 0.1),
                (rng.standard_normal((2, 4, 3, 3)) * 0.3, rng.standard_normal(2) * 0.1)]
    else:
        w = 3
        m.tc_fno = FNOParams(P_w=rng.standard_normal((w, 2 * kc)) * 0.4, P_b=rng.standard_normal(w) * 0.1,
                             R=[(rng.standard_normal((6, 3, w, w)) + 1j * rng.standard_normal((6, 3, w, w))) * 0.2
                                for _ in range(2)],
                             W=[rng.standard_normal((w, w)) * 0.4 for _ in range(2)],
                             Wb=[rng.standard_normal(w) * 0.1 for _ in range(2)],
                             Q_w=rng.standard_normal((2, w)) * 0.4, Q_b=rng.standard_normal(2) * 0.1)
    gbar = rng.standard_normal((2, n, n))
    Ubar, hbar, grads = temporal_correction_vjp(U, hist, p, m, gbar)
    L = lambda U_, h_: float(np.sum(gbar * O.temporal_correction(U_, h_, p, m)))
    eps = 1e-6
    dU = rng.standard_normal(U.shape)
    dh = [rng.standard_normal(h.shape) for h in hist]
    jvp = (L(U + eps * dU, [h + eps * d for h, d in zip(hist, dh)])
           - L(U - eps * dU, [h - eps * d for h, d in zip(hist, dh)])) / (2 * eps)
    vjp = np.sum(Ubar * dU) + sum(np.sum(b * d) for b, d in zip(hbar, dh))
    assert abs(jvp - vjp) < 1e-6 * max(1.0, abs(jvp))
    # parameter entries
    if head == "cnn":
        for l, idx in ((0, (1, 2, 0, 1)), (1, (0, 3, 2, 2))):
            W = m.tc[l][0]
            W[idx] += eps
            lp = L(U, hist)
            W[idx] -= 2 * eps
            lm = L(U, hist)
            W[idx] += eps
            assert abs((lp - lm) / (2 * eps) - grads[l][0][idx]) < 1e-6 * max(1.0, abs(grads[l][0][idx]))
    else:
        for arr, garr, idx in ((m.tc_fno.P_w, grads.P_w, (1, 4)), (m.tc_fno.Q_w, grads.Q_w, (0, 2)),
                               (m.tc_fno.W[1], grads.W[1], (2, 1))):
            arr[idx] += eps
            lp = L(U, hist)
            arr[idx] -= 2 * eps
            lm = L(U, hist)
            arr[idx] += eps
            assert abs((lp - lm) / (2 * eps) - garr[idx]) < 1e-6 * max(1.0, abs(garr[idx]))


def _fno_small(seed, width=3, modes=2, layers=2):
    rng = np.random.default_rng(seed)
    return O.FNOParams(P_w=rng.standard_normal((width, 2)) * 0.4, P_b=rng.standard_normal(width) * 0.1,
                       R=[(rng.standard_normal((2 * modes, modes, width, width))
                           + 1j * rng.standard_normal((2 * modes, modes, width, width))) * 0.2 for _ in range(layers)],
                       W=[rng.standard_normal((width, width)) * 0.4 for _ in range(layers)],
                       Wb=[rng.standard_normal(width) * 0.1 for _ in range(layers)],
                       Q_w=rng.standard_normal((8, width)) * 0.05, Q_b=rng.standard_normal(8) * 0.01)


@pytest.mark.parametrize("ablation,with_fno,flow", [(0, True, O.FLOW_NAVIER_STOKES), (1, False, O.FLOW_NAVIER_STOKES),
                                                    (1, True, O.FLOW_BURGERS), (2, True, O.FLOW_NAVIER_STOKES)])
def test_learned_step_vjp_with_fno_and_ablations(ablation, with_fno, flow):
    """Reverse mode of the learned step with the frequency-domain operator and the
    ablation variants: dot product with a fourth-order finite-difference JVP, and
    central differences on a W_L entry and on O_F parameters."""
    n = 8
    p = O.Problem(nx=n, ny=n, nu=0.02, dt=0.02, flow=flow, forcing_kind=1 if flow == O.FLOW_NAVIER_STOKES else 0)
    model = small_model(11, n)
    model.ablation = ablation
    model.fno = _fno_small(12) if with_fno else None
    rng = np.random.default_rng(13)
    U = I.kolmogorov_ic(n, 5) if flow == O.FLOW_NAVIER_STOKES else I.burgers_ic(n, 5)
    du = rng.standard_normal(U.shape)
    if flow == O.FLOW_NAVIER_STOKES:
        du = O.project(du, p)
    lam = rng.standard_normal(U.shape)
    jv = fd4_jvp(lambda x: O.learned_step(x, p, model), U, du, 1e-3)
    lam_in, grads = A.step_vjp(U, p, lam, model)
    lhs, rhs = np.sum(jv * lam), np.sum(du * lam_in)
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)

    def loss_with(mod):
        return np.sum(O.learned_step(U, p, mod) * lam)

    eps = 1e-4
    if ablation != 2:
        idx = (1, 0, 2, 1)
        def m(s):
            import copy
            mm = copy.copy(model)
            mm.W_L = model.W_L.copy()
            mm.W_L[idx] += s
            return mm
        fd = (loss_with(m(eps)) - loss_with(m(-eps))) / (2 * eps)
        assert abs(fd - grads[0][idx]) <= 1e-6 * max(1e-3, abs(fd))
    else:
        assert np.all(grads[0] == 0)
    if with_fno:
        fg = grads[2]
        for name, get, idx in (("Q_w", lambda f: f.Q_w, (3, 1)), ("W1", lambda f: f.W[1], (0, 2)),
                               ("P_w", lambda f: f.P_w, (2, 0)), ("R0", lambda f: f.R[0], (1, 1, 0, 2))):
            def m(s, get=get, idx=idx):
                import copy
                mm = copy.copy(model)
                f = copy.deepcopy(model.fno)
                get(f)[idx] += s
                mm.fno = f
                return mm
            fd = (loss_with(m(eps)) - loss_with(m(-eps))) / (2 * eps)
            want = get(fg)[idx]
            want = want.real if np.iscomplexobj(want) else want
            assert abs(fd - want) <= 1e-6 * max(1e-3, abs(fd)), name
