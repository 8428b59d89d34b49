"""GPU parity of the joint velocity-scalar reverse mode (shear flow's passive
scalar, App. C.1) on the generic-grid path against the FP64 oracle: one joint
step's VJP for the plain solver and for a model that learns the scalar (W_L,
W_Ls, the stencil network on (u, v, s)), and the checkpointed joint training
step with the velocity's temporal correction.

Grids: the shear flow's 128 x 64 grid on [0, 8] x [0, 4] and the 25^2 Burgers
preset. FP32 on the GPU, BF16-representable weights in both. Bars: cotangents
<= 1e-5 (plain) and <= 1e-4 (learned) relative L2; parameter blocks <= 1e-3;
the training step's loss <= 1e-4 and gradient blocks <= 2e-3.
"""

import numpy as np
import pytest

import oracle as O
import oracle.scalar as OS
from oracle import adjoint as A
from oracle import train as T
from paper_2507_01975_gb300 import fd
from paper_2507_01975_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_01975_gb300 import build

    build.build()
    fd.load()


def rel_l2(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float32, device="cuda")


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


CASES = {
    "shear128x64": dict(n=128, ny=64, dtype="f32", lx=8.0, ly=4.0, nu=1e-3, dt=5e-3),
    "burgers25": dict(n=25, dtype="f32", flow="burgers", lx=1.0, ly=1.0, nu=1e-2, dt=1e-3, deriv_order=2),
}


def problem(cfg):
    return O.Problem(nx=cfg.n, ny=cfg.ny or cfg.n, lx=cfg.lx, ly=cfg.ly, nu=cfg.nu, dt=cfg.dt,
                     flow=O.FLOW_BURGERS if cfg.flow == "burgers" else O.FLOW_NAVIER_STOKES,
                     deriv_order=cfg.deriv_order)


def joint_states(case, p, b):
    if case == "shear128x64":
        ics = [I.shear_scalar_ic(p.nx, p.ny, p.lx, p.ly, seed=k) for k in range(b)]
        return f32(np.stack([O.project(u, p) for u, _ in ics])), f32(np.stack([s for _, s in ics]))
    U = np.stack([I.burgers_ic(p.nx, 60 + k) for k in range(b)])
    S = np.stack([I.burgers_ic(p.nx, 70 + k)[0] + 1.0 for k in range(b)])
    return f32(U), f32(S)


def scalar_model(seed, kc=0):
    st = I.random_conv_stack(seed, 3, O.CNN_HIDDEN, OS.N_COEF_SCALAR, last_scale=0.3)
    rng = np.random.default_rng(seed + 7)
    tc = I.random_conv_stack(seed + 2, 2 * kc, O.CNN_HIDDEN, 2, last_scale=0.02) if kc else []
    return O.LearnedModel(W_L=I.random_wl(seed + 1, 1e-2), stencil=st, W_Ls=f32(rng.standard_normal((2, 2, 5, 4)) * 0.05),
                          k_c=kc, tc=tc)


def check_blocks(g, wl, wls, layers, m, tol, tc=None):
    assert rel_l2(g[:80], wl.ravel()) <= tol, ("W_L", rel_l2(g[:80], wl.ravel()))
    assert rel_l2(g[80:160], wls.ravel()) <= tol, ("W_Ls", rel_l2(g[80:160], wls.ravel()))
    o = 160
    for l, ((W, bb), (dW, db)) in enumerate(zip(m.stencil, layers)):
        assert rel_l2(g[o:o + W.size], dW.ravel()) <= tol, ("W", l, rel_l2(g[o:o + W.size], dW.ravel()))
        o += W.size
        assert rel_l2(g[o:o + bb.size], db) <= tol, ("b", l, rel_l2(g[o:o + bb.size], db))
        o += bb.size
    for l, ((W, bb), (dW, db)) in enumerate(zip(m.tc, tc or [])):
        assert rel_l2(g[o:o + W.size], dW.ravel()) <= tol, ("tc W", l, rel_l2(g[o:o + W.size], dW.ravel()))
        o += W.size
        if l == len(m.tc) - 1:
            # the last bias sees the mean-free correction cotangent: zero in exact
            # arithmetic, an FP32 residue here, bounded against its layer's weights
            assert np.abs(g[o:o + bb.size]).max() <= 1e-6 * np.linalg.norm(dW)
        else:
            assert rel_l2(g[o:o + bb.size], db) <= tol, ("tc b", l)
        o += bb.size
    assert o == g.size


@pytest.mark.parametrize("case", list(CASES))
def test_plain_joint_step_adjoint_matches_oracle(case):
    cfg = fd.Config(batch=2, path=3, **CASES[case])
    p = problem(cfg)
    U, S = joint_states(case, p, 2)
    rng = np.random.default_rng(5)
    lu, ls = rng.standard_normal(U.shape), rng.standard_normal(S.shape)
    s = fd.Solver(cfg)
    gu, gs = torch.empty_like(dev(U)), torch.empty_like(dev(S))
    D = 2e-3
    s.step_adjoint_scalar(D, dev(U), dev(S), dev(lu), dev(ls), gu, gs)
    torch.cuda.synchronize()
    refs = [A.rk4_step_scalar_vjp(U[k], S[k], p, D, lu[k], ls[k]) for k in range(2)]
    assert rel_l2(gu.double().cpu().numpy(), np.stack([r[0] for r in refs])) <= 1e-5
    assert rel_l2(gs.double().cpu().numpy(), np.stack([r[1] for r in refs])) <= 1e-5
    s.close()


@pytest.mark.parametrize("case", list(CASES))
def test_learned_joint_step_adjoint_matches_oracle(case):
    cfg = fd.Config(batch=2, learned=True, scalar_learned=True, **CASES[case])
    p = problem(cfg)
    U, S = joint_states(case, p, 2)
    m = scalar_model(9)
    s = fd.Solver(cfg)
    s.set_params(I.pack_params(m.W_L, m.stencil, W_Ls=m.W_Ls))
    rng = np.random.default_rng(6)
    lu, ls = rng.standard_normal(U.shape), rng.standard_normal(S.shape)
    lu_d, ls_d = dev(lu), dev(ls)
    dp = torch.zeros(s.param_count(), device="cuda")
    D = 2e-3
    # outputs aliasing the cotangents
    s.step_adjoint_scalar(D, dev(U), dev(S), lu_d, ls_d, lu_d, ls_d, dp)
    torch.cuda.synchronize()
    refs = [A.rk4_step_scalar_vjp(U[k], S[k], p, D, lu[k], ls[k], m) for k in range(2)]
    ru, rs = np.stack([r[0] for r in refs]), np.stack([r[1] for r in refs])
    assert rel_l2(lu_d.double().cpu().numpy(), ru) <= 1e-4
    assert rel_l2(ls_d.double().cpu().numpy(), rs) <= 1e-4
    wl = sum(r[2][0] for r in refs)
    wls = sum(r[2][1] for r in refs)
    layers = [(sum(r[2][2][l][0] for r in refs), sum(r[2][2][l][1] for r in refs)) for l in range(6)]
    check_blocks(dp.double().cpu().numpy(), wl, wls, layers, m, 1e-3)
    # the learned scalar operators change the scalar's cotangent by far more than the bar
    plain = np.stack([A.rk4_step_scalar_vjp(U[k], S[k], p, D, lu[k], ls[k])[1] for k in range(2)])
    assert rel_l2(rs, plain) > 10 * rel_l2(ls_d.double().cpu().numpy(), rs)
    s.close()


def test_joint_train_step_with_corrections_matches_oracle():
    """Four joint steps on the shear grid with a correction every two steps and
    checkpoints every two: loss and every parameter block against the oracle."""
    kc, steps, D = 2, 4, 1e-3
    cfg = fd.Config(batch=1, learned=True, scalar_learned=True, k_c=kc, **CASES["shear128x64"])
    p = problem(cfg)
    U, S = joint_states("shear128x64", p, 1)
    m = scalar_model(13, kc=kc)
    s = fd.Solver(cfg)
    s.set_params_device(dev(I.pack_params(m.W_L, m.stencil, m.tc, W_Ls=m.W_Ls)))
    states, _ = T.rollout_scalar_states(U[0], S[0], p, D, steps, m)
    rng = np.random.default_rng(9)
    tu = f32(np.stack([states[k][0] for k in range(1, steps + 1)])[:, None] + 0.05 * rng.standard_normal((steps, 1) + U.shape[1:]))
    ts = f32(np.stack([states[k][1] for k in range(1, steps + 1)])[:, None] + 0.05 * rng.standard_normal((steps, 1) + S.shape[1:]))
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    dp = torch.zeros(s.param_count(), device="cuda")
    s.train_step_scalar(D, dev(U), dev(S), dev(tu), dev(ts), steps, 2, dp, loss)
    torch.cuda.synchronize()
    pu = np.stack([states[k][0] for k in range(1, steps + 1)])
    ps = np.stack([states[k][1] for k in range(1, steps + 1)])
    total = steps * (pu[0].size + ps[0].size)
    lref = (np.sum((pu - tu[:, 0]) ** 2) + np.sum((ps - ts[:, 0]) ** 2)) / total
    assert abs(float(loss.item()) - lref) <= 1e-4 * lref
    _, _, g = T.rollout_scalar_vjp(U[0], S[0], p, D, steps, 2 * (pu - tu[:, 0]) / total, 2 * (ps - ts[:, 0]) / total, m)
    check_blocks(dp.double().cpu().numpy(), g["W_L"], g["W_Ls"], g["stencil"], m, 2e-3, tc=g["tc"])
    s.close()


def test_joint_reverse_mode_refusals():
    u = torch.zeros((1, 2, 64, 128), device="cuda")
    sc = torch.zeros((1, 64, 128), device="cuda")
    # a velocity-only learned model does not read the scalar
    s = fd.Solver(fd.Config(batch=1, learned=True, **CASES["shear128x64"]))
    with pytest.raises(fd.FdError) as e:
        s.step_adjoint_scalar(1e-3, u, sc, u, sc, torch.empty_like(u), torch.empty_like(sc))
    assert e.value.status == fd.FD_EUNSUPPORTED
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(fd.FdError) as e:
        s.train_step_scalar(1e-3, u, sc, u[None], sc[None], 1, 1, torch.zeros(8, device="cuda"), loss)
    assert e.value.status == fd.FD_EUNSUPPORTED
    s.close()
    # a plain context takes no parameter gradient; a negative diffusivity is invalid
    s = fd.Solver(fd.Config(batch=1, **CASES["shear128x64"]))
    with pytest.raises(fd.FdError) as e:
        s.step_adjoint_scalar(1e-3, u, sc, u, sc, torch.empty_like(u), torch.empty_like(sc),
                              torch.zeros(8, device="cuda"))
    assert e.value.status == fd.FD_EINVAL
    with pytest.raises(fd.FdError) as e:
        s.step_adjoint_scalar(-1.0, u, sc, u, sc, torch.empty_like(u), torch.empty_like(sc))
    assert e.value.status == fd.FD_EINVAL
    s.close()
