"""Pins of the oracle's frequency-domain operator O_F (Sec. 3.4; Table S3).

* a single Fourier mode through the spectral convolution has a closed form
  (a cos - b sin for the complex weight a + ib), in both row blocks;
* modes outside the kept set are removed;
* with zero spectral weights the operator is a chain of pointwise maps and
  GELUs, checked against explicit loops;
* the whole operator commutes with periodic translations;
* inside the flux block: zero output changes nothing, any output keeps the
  mean momentum (the flux form telescopes for any face values).
"""

import numpy as np

import oracle as O
from oracle.fno import FNOParams, fno_forward, spectral_conv


def random_fno(rng, width=4, modes=4, layers=2, scale=0.3):
    R = [(rng.standard_normal((2 * modes, modes, width, width)) + 1j * rng.standard_normal((2 * modes, modes, width, width)))
         * scale / width for _ in range(layers)]
    return FNOParams(P_w=rng.standard_normal((width, 2)) * scale, P_b=rng.standard_normal(width) * 0.1,
                     R=R, W=[rng.standard_normal((width, width)) * scale for _ in range(layers)],
                     Wb=[rng.standard_normal(width) * 0.1 for _ in range(layers)],
                     Q_w=rng.standard_normal((8, width)) * scale, Q_b=rng.standard_normal(8) * 0.01)


def mode(n, ky, kx):
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return 2 * np.pi * (ky * j + kx * i) / n


def test_single_mode_closed_form_both_blocks():
    n, m = 16, 4
    for ky, row in ((2, 2), (-2, 2 * m - 2)):  # ky = -2 lives in the second block
        th = mode(n, ky, 3)
        v = np.stack([np.zeros((n, n)), np.cos(th)])
        R = np.zeros((2 * m, m, 2, 3), dtype=complex)
        w = np.array([0.5 - 0.25j, -1.0 + 2.0j, 0.3j])
        R[row, 3, 1, :] = w
        out = spectral_conv(v, R)
        for o in range(3):
            ref = w[o].real * np.cos(th) - w[o].imag * np.sin(th)
            assert np.abs(out[o] - ref).max() < 1e-13


def test_modes_outside_the_kept_set_are_removed():
    n, m = 16, 4
    R = np.ones((2 * m, m, 1, 1), dtype=complex)
    for ky, kx in ((0, m), (m, 1), (-m - 1, 2), (n // 2, 0)):
        v = np.cos(mode(n, ky, kx))[None]
        assert np.abs(spectral_conv(v, R)).max() < 1e-13
    # a kept mode with unit weights passes unchanged
    v = np.cos(mode(n, -3, 2))[None]
    assert np.abs(spectral_conv(v, R) - v).max() < 1e-13


def test_zero_spectral_weights_reduce_to_pointwise_loops():
    rng = np.random.default_rng(7)
    n, width = 8, 3
    prm = random_fno(rng, width=width, modes=2, layers=2)
    prm.R = [np.zeros_like(r) for r in prm.R]
    U = rng.standard_normal((2, n, n))
    out = fno_forward(U, prm)
    ref = np.zeros((8, n, n))
    for y in range(n):
        for x in range(n):
            v = [sum(prm.P_w[o, i] * U[i, y, x] for i in range(2)) + prm.P_b[o] for o in range(width)]
            for l in range(2):
                v = [sum(prm.W[l][o, i] * v[i] for i in range(width)) + prm.Wb[l][o] for o in range(width)]
                if l == 0:
                    v = [float(O.gelu(np.array(t))) for t in v]
            for q in range(8):
                ref[q, y, x] = sum(prm.Q_w[q, i] * v[i] for i in range(width)) + prm.Q_b[q]
    assert np.abs(out - ref).max() < 1e-12


def test_translation_equivariance():
    rng = np.random.default_rng(8)
    n = 16
    prm = random_fno(rng, width=4, modes=4, layers=3)
    U = rng.standard_normal((2, n, n))
    a = fno_forward(np.roll(U, (3, -5), axis=(1, 2)), prm)
    b = np.roll(fno_forward(U, prm), (3, -5), axis=(1, 2))
    assert np.abs(a - b).max() < 1e-12


def _model(rng, fno):
    st = [(rng.standard_normal((64, 2, 3, 3)) * 0.05, np.zeros(64))]
    for _ in range(4):
        st.append((rng.standard_normal((64, 64, 3, 3)) * 0.02, np.zeros(64)))
    st.append((np.zeros((160, 64, 3, 3)), np.zeros(160)))
    return O.LearnedModel(W_L=rng.standard_normal((2, 2, 5, 4)) * 1e-3, stencil=st, fno=fno)


def test_operator_in_the_flux_block():
    rng = np.random.default_rng(9)
    n = 16
    p = O.Problem(nx=n, ny=n, nu=1e-3, dt=2e-3)
    U = O.project(rng.standard_normal((2, n, n)) * 0.3, p)
    prm = random_fno(rng, width=4, modes=4, layers=2)
    base = O.learned_step(U, p, _model(np.random.default_rng(1), None))
    zero = FNOParams(**{**prm.__dict__, "Q_w": np.zeros_like(prm.Q_w), "Q_b": np.zeros_like(prm.Q_b)})
    assert np.array_equal(O.learned_step(U, p, _model(np.random.default_rng(1), zero)), base)
    with_f = O.learned_step(U, p, _model(np.random.default_rng(1), prm))
    assert np.abs(with_f - base).max() > 1e-6
    for c in range(2):
        assert abs(with_f[c].sum() - U[c].sum()) < 1e-12 * np.abs(U[c]).sum()


def test_temporal_correction_operator():
    """The FNO temporal correction (Sec. 3.5): 2 k_c -> 2 channels. With zero
    spectral weights it is a chain of pointwise maps (brute force over the
    history channels); the corrected state keeps the mean momentum and is
    divergence-free; Q = 0 leaves a divergence-free state unchanged."""
    rng = np.random.default_rng(10)
    n, kc, width = 8, 3, 3
    prm = random_fno(rng, width=width, modes=2, layers=2)
    prm.P_w = rng.standard_normal((width, 2 * kc)) * 0.3
    prm.Q_w = rng.standard_normal((2, width)) * 0.3
    prm.Q_b = rng.standard_normal(2) * 0.01
    hist = [rng.standard_normal((2, n, n)) for _ in range(kc)]
    zero_r = FNOParams(**{**prm.__dict__, "R": [np.zeros_like(r) for r in prm.R]})
    out = fno_forward(np.concatenate(hist), zero_r)
    for y, x in ((0, 0), (3, 5), (7, 2)):
        v = [sum(prm.P_w[o, 2 * s + c] * hist[s][c, y, x] for s in range(kc) for c in range(2)) + prm.P_b[o]
             for o in range(width)]
        for l in range(2):
            v = [sum(prm.W[l][o, i] * v[i] for i in range(width)) + prm.Wb[l][o] for o in range(width)]
            if l == 0:
                v = [float(O.gelu(np.array(t))) for t in v]
        for q in range(2):
            ref = sum(prm.Q_w[q, i] * v[i] for i in range(width)) + prm.Q_b[q]
            assert abs(out[q, y, x] - ref) < 1e-12
    p = O.Problem(nx=n, ny=n, nu=1e-3, dt=2e-3)
    U = O.project(rng.standard_normal((2, n, n)), p)
    m = _model(np.random.default_rng(2), None)
    m.k_c, m.tc_fno = kc, prm
    V = O.temporal_correction(U, hist, p, m)
    assert np.abs(V.mean(axis=(1, 2)) - U.mean(axis=(1, 2))).max() < 1e-13
    assert np.abs(O.divergence(V, p.dx, p.dy)).max() < 1e-11
    assert np.abs(V - U).max() > 1e-3
    m.tc_fno = FNOParams(**{**prm.__dict__, "Q_w": np.zeros_like(prm.Q_w), "Q_b": np.zeros_like(prm.Q_b)})
    assert np.abs(O.temporal_correction(U, hist, p, m) - U).max() < 1e-13


def test_ablation_variants():
    """The ablation variants of the flux block (Sec. 4, Table 4). Without the
    physics-based convolution and with zero learned kernels the face values
    vanish, so the step is pure forcing (plus projection); with only the
    frequency-domain operator the face values are O_F(u) itself, checked
    against face values assembled by hand; both keep the mean momentum."""
    rng = np.random.default_rng(11)
    n = 16
    p = O.Problem(nx=n, ny=n, nu=1e-3, dt=2e-3, forcing_kind=0)
    U = O.project(rng.standard_normal((2, n, n)) * 0.3, p)
    zero = _model(np.random.default_rng(3), None)
    zero.W_L = np.zeros_like(zero.W_L)
    zero.ablation = 1  # the last network layer is zero: K = W_L + C = 0
    for k in O.learned_kernels(U, p, zero):
        assert np.abs(k).max() == 0.0
    assert np.array_equal(O.learned_step(U, p, zero), O.project(U, p))
    # without the physics conv the learned kernel is used as is (no projection)
    m1 = _model(np.random.default_rng(3), None)
    m1.ablation = 1
    ks = O.learned_kernels(U, p, m1)
    q = 1  # u-x derivative: W_L / h, no physics part, not projected
    ref = m1.W_L[1, 0] / p.dx
    assert np.abs(ks[q] - ref[:, :, None, None]).max() < 1e-14
    # frequency operator only: tendency from the O_F face values alone
    prm = random_fno(rng, width=4, modes=4, layers=2)
    m2 = _model(np.random.default_rng(3), prm)
    m2.ablation = 2
    H = O.tendency(U, p, O.learned_kernels(U, p, m2), O.fno_forward(U, prm))
    Uc, Gxc, Uk, Gyu, Vk, Gxv, Vc, Gyc = O.fno_forward(U, prm)
    sh = O.shifted
    Tu = (-(Uc**2 - sh(Uc**2, 0, -1)) / p.dx - (sh(Uk * Vk, 1, 0) - Uk * Vk) / p.dy
          + p.nu * ((Gxc - sh(Gxc, 0, -1)) / p.dx + (sh(Gyu, 1, 0) - Gyu) / p.dy))
    assert np.abs(H[0] - Tu).max() < 1e-12 * max(1.0, np.abs(Tu).max())
    for m in (m1, m2):
        V = O.learned_step(U, p, m)
        assert np.abs(V.mean(axis=(1, 2)) - U.mean(axis=(1, 2))).max() < 1e-13


def test_spectral_conv_vjp_dot_products():
    """spectral_conv is real-linear in v and in R: <ybar, S(v)> = <vbar, v> and
    <ybar, S_v(dR)> = Re sum conj(Rbar) dR, for M < N/2 and M = N/2."""
    from oracle.fno import spectral_conv_vjp

    rng = np.random.default_rng(14)
    for n, m in ((16, 4), (16, 8), (12, 3)):
        ci, co = 3, 2
        v = rng.standard_normal((ci, n, n))
        R = rng.standard_normal((2 * m, m, ci, co)) + 1j * rng.standard_normal((2 * m, m, ci, co))
        ybar = rng.standard_normal((co, n, n))
        vbar, Rbar = spectral_conv_vjp(v, R, ybar)
        assert abs(np.sum(ybar * spectral_conv(v, R)) - np.sum(vbar * v)) < 1e-11 * np.abs(ybar).sum()
        dR = rng.standard_normal(R.shape) + 1j * rng.standard_normal(R.shape)
        assert abs(np.sum(ybar * spectral_conv(v, dR)) - np.real(np.sum(np.conj(Rbar) * dR))) < 1e-11 * np.abs(ybar).sum()


def test_fno_vjp_against_finite_differences():
    """Every gradient of fno_vjp against central differences of fno_forward (FP64):
    the input, P, every layer's R (real and imaginary parts), W and b, and Q; a
    random direction for the input."""
    from oracle.fno import fno_vjp

    rng = np.random.default_rng(15)
    n, cin = 8, 4
    prm = random_fno(rng, width=3, modes=3, layers=3, scale=0.5)
    prm.P_w = rng.standard_normal((3, cin)) * 0.5
    prm.Q_w = rng.standard_normal((2, 3)) * 0.5
    prm.Q_b = rng.standard_normal(2) * 0.1
    U = rng.standard_normal((cin, n, n))
    gbar = rng.standard_normal((2, n, n))
    Ubar, g = fno_vjp(U, prm, gbar)
    L = lambda P, X=U: float(np.sum(gbar * fno_forward(X, P)))
    eps = 1e-6

    def fd(get, set_, idx, imag=False):
        def shifted_params(delta):
            P = FNOParams(P_w=prm.P_w.copy(), P_b=prm.P_b.copy(), R=[r.copy() for r in prm.R],
                          W=[w.copy() for w in prm.W], Wb=[b.copy() for b in prm.Wb], Q_w=prm.Q_w.copy(),
                          Q_b=prm.Q_b.copy())
            a = get(P)
            a[idx] += delta * (1j if imag else 1.0)
            return P
        return (L(shifted_params(eps)) - L(shifted_params(-eps))) / (2 * eps)

    checks = [
        (lambda P: P.P_w, (1, 2), g.P_w[1, 2]), (lambda P: P.P_b, (0,), g.P_b[0]),
        (lambda P: P.W[1], (2, 0), g.W[1][2, 0]), (lambda P: P.Wb[2], (1,), g.Wb[2][1]),
        (lambda P: P.Q_w, (1, 1), g.Q_w[1, 1]), (lambda P: P.Q_b, (0,), g.Q_b[0]),
    ]
    for get, idx, want in checks:
        got = fd(get, None, idx)
        assert abs(got - want) < 1e-6 * max(1.0, abs(want)), (idx, got, want)
    for l, idx in ((0, (0, 1, 2, 1)), (2, (5, 0, 1, 0)), (1, (2, 2, 0, 2))):
        want = g.R[l][idx]
        re = fd(lambda P, l=l: P.R[l], None, idx)
        im = fd(lambda P, l=l: P.R[l], None, idx, imag=True)
        assert abs(re - want.real) < 1e-6 * max(1.0, abs(want)) and abs(im - want.imag) < 1e-6 * max(1.0, abs(want))
    dU = rng.standard_normal(U.shape)
    jvp = (L(prm, U + eps * dU) - L(prm, U - eps * dU)) / (2 * eps)
    assert abs(jvp - np.sum(Ubar * dU)) < 1e-6 * max(1.0, abs(jvp))
