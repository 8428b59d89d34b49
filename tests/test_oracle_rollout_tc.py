"""Pins of the oracle's rollout reverse mode with the temporal correction (CPU).

u_k = P(FV(u_{k-1}) + TC(u_{k-k_c} .. u_{k-1}) - mean) at k = M k_c (Sec. 3.2,
Sec. 3.5) makes a state depend on the k_c states before it, so the reverse mode
must route each corrected state's cotangent back to its whole history window.
``rollout_vjp_full`` is held to the definition of a vector-Jacobian product:

* <J du, lam> = <du, J^T lam> with J du from a fourth-order finite difference of
  the rollout itself (CNN head and FNO correction, forced and decaying flows);
* parameter gradients (a temporal-correction weight of each network kind, a
  W_L entry, a stencil weight, an O_F weight) against central differences of
  L = sum_k <lam_k, u_k>, each read from ``flat_grads`` at the index where the
  parameter array of ``inputs.pack_params`` holds that parameter.

A planted mistake (the history cotangents dropped) breaks the first identity.
"""

import copy

import numpy as np
import pytest

import oracle as O
from oracle import adjoint as A
from oracle import train as T
from paper_2507_01975_gb300 import inputs as I

N, KC, STEPS = 12, 2, 5


def _model(kind, with_fno=False):
    st = I.random_conv_stack(81, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=0.3)
    fno = O.FNOParams(**I.random_fno(82, 4, 3, 2, out_scale=0.3)) if with_fno else None
    if kind == "cnn":
        tc = I.random_conv_stack(83, 2 * KC, O.CNN_HIDDEN, 2, last_scale=0.5)
        return O.LearnedModel(W_L=I.random_wl(84, 0.05), stencil=st, tc=tc, k_c=KC, fno=fno)
    tcf = O.FNOParams(**I.random_fno(85, 4, 3, 2, out_scale=0.5, cin=2 * KC, cout=2))
    return O.LearnedModel(W_L=I.random_wl(84, 0.05), stencil=st, tc_fno=tcf, k_c=KC, fno=fno)


def _problem(forced):
    return O.Problem(nx=N, ny=N, nu=0.02, dt=0.02, forcing_kind=1 if forced else 0)


def _traj(U, p, model):
    states, _ = T.rollout_states(U, p, STEPS, model)
    return np.stack(states[1:])


def _objective(U, p, model, lam):
    return float(np.sum(_traj(U, p, model) * lam))


def dot_product_residual(kind, forced, with_fno=False):
    p = _problem(forced)
    model = _model(kind, with_fno)
    rng = np.random.default_rng(86)
    U = O.project(I.kolmogorov_ic(N, 3) + 0.1 * rng.standard_normal((2, N, N)), p)
    du = rng.standard_normal(U.shape)
    lam = rng.standard_normal((STEPS, 2, N, N))
    eps = 1e-3
    f = lambda x: _traj(x, p, model)  # noqa: E731
    jv = (-f(U + 2 * eps * du) + 8 * f(U + eps * du) - 8 * f(U - eps * du) + f(U - 2 * eps * du)) / (12 * eps)
    lam0, _ = T.rollout_vjp_full(U, p, STEPS, lam, model)
    lhs, rhs = np.sum(jv * lam), np.sum(du * lam0)
    return abs(lhs - rhs) / abs(lhs)


@pytest.mark.parametrize("kind,forced,with_fno", [("cnn", True, False), ("cnn", False, False), ("fno", True, False),
                                                  ("fno", False, True)])
def test_rollout_vjp_with_temporal_correction_dot_product(kind, forced, with_fno):
    assert dot_product_residual(kind, forced, with_fno) < 1e-9


def _flat_index(model, mutate):
    """Index of the parameter that ``mutate`` changes in the packed parameter array."""
    m2 = copy.deepcopy(model)
    mutate(m2, 0.5)
    a = I.pack_params(model.W_L, model.stencil, _tc_pack(model), _fno_pack(model))
    b = I.pack_params(m2.W_L, m2.stencil, _tc_pack(m2), _fno_pack(m2))
    idx = np.flatnonzero(a != b)
    assert idx.size == 1
    return int(idx[0])


def _op_dict(f):
    return None if f is None else {"P_w": f.P_w, "P_b": f.P_b, "R": f.R, "W": f.W, "Wb": f.Wb, "Q_w": f.Q_w,
                                   "Q_b": f.Q_b}


def _tc_pack(m):
    return _op_dict(m.tc_fno) if m.tc_fno is not None else m.tc


def _fno_pack(m):
    return _op_dict(m.fno)


@pytest.mark.parametrize("kind", ["cnn", "fno"])
def test_rollout_parameter_gradients_against_central_differences(kind):
    p = _problem(True)
    model = _model(kind, with_fno=True)
    rng = np.random.default_rng(87)
    U = O.project(I.kolmogorov_ic(N, 4) + 0.1 * rng.standard_normal((2, N, N)), p)
    lam = rng.standard_normal((STEPS, 2, N, N))
    _, g = T.rollout_vjp_full(U, p, STEPS, lam, model)
    flat = T.flat_grads(g, model)
    assert flat.size == I.pack_params(model.W_L, model.stencil, _tc_pack(model), _fno_pack(model)).size

    def set_wl(m, d):
        m.W_L = m.W_L.copy()
        m.W_L[1, 0, 3, 2] += d

    def set_st(m, d):
        W, b = m.stencil[2]
        W = W.copy()
        W[5, 7, 1, 2] += d
        m.stencil = list(m.stencil)
        m.stencil[2] = (W, b)

    def set_fno(m, d):
        m.fno = copy.deepcopy(m.fno)
        m.fno.Q_w[3, 1] += d

    checks = [set_wl, set_st, set_fno]
    if kind == "cnn":
        def set_tc_last(m, d):
            W, b = m.tc[5]
            W = W.copy()
            W[1, 9, 0, 2] += d
            m.tc = list(m.tc)
            m.tc[5] = (W, b)

        def set_tc_first(m, d):
            W, b = m.tc[0]
            W = W.copy()
            W[11, 3, 2, 1] += d
            m.tc = list(m.tc)
            m.tc[0] = (W, b)

        def set_tc_bias(m, d):
            W, b = m.tc[3]
            b = b.copy()
            b[17] += d
            m.tc = list(m.tc)
            m.tc[3] = (W, b)

        checks += [set_tc_last, set_tc_first, set_tc_bias]
    else:
        def set_tcf_r(m, d):
            m.tc_fno = copy.deepcopy(m.tc_fno)
            m.tc_fno.R[1][4, 2, 1, 3] += d

        def set_tcf_p(m, d):
            m.tc_fno = copy.deepcopy(m.tc_fno)
            m.tc_fno.P_w[2, 3] += d

        checks += [set_tcf_r, set_tcf_p]
    eps = 1e-4
    for mutate in checks:
        idx = _flat_index(model, mutate)
        mp, mm = copy.deepcopy(model), copy.deepcopy(model)
        mutate(mp, eps)
        mutate(mm, -eps)
        fd = (_objective(U, p, mp, lam) - _objective(U, p, mm, lam)) / (2 * eps)
        assert abs(fd - flat[idx]) <= 1e-6 * max(1.0, abs(fd)), (mutate.__name__, fd, flat[idx])


def test_planted_dropped_history_cotangents_fail(monkeypatch):
    real = A.temporal_correction_vjp

    def dropped(*args, **kw):
        Ub, hb, g = real(*args, **kw)
        return Ub, [np.zeros_like(h) for h in hb], g

    monkeypatch.setattr(A, "temporal_correction_vjp", dropped)
    assert dot_product_residual("cnn", True) > 1e-3
