"""GPU parity of the learned passive scalar (shear flow, App. C.1) on the
generic-grid path against the FP64 oracle: the stencil network on (u, v, s)
with 240 output channels, the scalar's four operator instances with per-face
kernels W_P + proj(W_Ls + C_s) / h^deriv, the scalar's flux-form stage fused
into the velocity's, and the velocity's temporal correction.

Grids: the shear flow's 128 x 64 grid on [0, 8] x [0, 4] (Table S2) and the
25^2 Burgers preset on [0, 1]^2. FP32 network with BF16-representable weights
(the oracle takes the same weights in FP64). Bars: network outputs <= 1e-4
relative L2; one joint step <= 1e-5 on the states and <= 2e-4 on their
increments over the step; a 4-step rollout with two corrections <= 1e-4; the
total scalar conserved to FP32 round-off; a zero module equal to the plain
joint step to 1e-6.
"""

import numpy as np
import pytest

import oracle as O
import oracle.scalar as OS
from paper_2507_01975_gb300 import fd
from paper_2507_01975_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NX, NY, LX, LY = 128, 64, 8.0, 4.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_01975_gb300 import build

    build.build()
    fd.load()


def rel_l2(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def scalar_model(seed, last_scale=0.3, ws_std=0.05, kc=0, zero=False):
    st = I.random_conv_stack(seed, 3, O.CNN_HIDDEN, OS.N_COEF_SCALAR, last_scale=0.0 if zero else last_scale)
    rng = np.random.default_rng(seed + 7)
    W_Ls = np.zeros((2, 2, 5, 4)) if zero else f32(rng.standard_normal((2, 2, 5, 4)) * ws_std)
    W_L = np.zeros((2, 2, 5, 4)) if zero else I.random_wl(seed + 1, 1e-2)
    tc = I.random_conv_stack(seed + 2, 2 * kc, O.CNN_HIDDEN, 2, last_scale=0.02) if kc else []
    return O.LearnedModel(W_L=W_L, stencil=st, W_Ls=W_Ls, k_c=kc, tc=tc)


def shear_cfg(batch=2, dt=5e-3, kc=0, **kw):
    return fd.Config(n=NX, ny=NY, batch=batch, dtype="f32", nu=1e-3, dt=dt, lx=LX, ly=LY, learned=True, k_c=kc,
                     scalar_learned=True, **kw)


def problem(cfg):
    return O.Problem(nx=cfg.n, ny=cfg.ny or cfg.n, lx=cfg.lx, ly=cfg.ly, nu=cfg.nu, dt=cfg.dt,
                     flow=O.FLOW_BURGERS if cfg.flow == "burgers" else O.FLOW_NAVIER_STOKES,
                     deriv_order=cfg.deriv_order)


def shear_states(p, b):
    ics = [I.shear_scalar_ic(p.nx, p.ny, p.lx, p.ly, seed=k) for k in range(b)]
    U0 = f32(np.stack([O.project(u, p) for u, _ in ics]))
    S0 = f32(np.stack([s for _, s in ics]))
    return U0, S0


def solver(cfg, model):
    s = fd.Solver(cfg)
    s.set_params(I.pack_params(model.W_L, model.stencil, model.tc, W_Ls=model.W_Ls))
    return s


def gpu_joint(s, U0, S0, steps, D):
    u = torch.tensor(U0, dtype=torch.float32, device="cuda")
    sc = torch.tensor(S0, dtype=torch.float32, device="cuda")
    uo, so = torch.empty_like(u), torch.empty_like(sc)
    s.rollout_scalar(u, sc, uo, so, steps, D)
    torch.cuda.synchronize()
    return uo.double().cpu().numpy(), so.double().cpu().numpy()


def test_parameter_count_and_network_on_u_v_s():
    cfg = shear_cfg()
    model = scalar_model(3, last_scale=1.0)
    s = solver(cfg, model)
    # W_L, W_Ls, the stencil network 3 -> 64 x 5 -> 240
    assert s.param_count() == 160 + (64 * 3 * 9 + 64) + 4 * (64 * 64 * 9 + 64) + (240 * 64 * 9 + 240)
    p = problem(cfg)
    U0, S0 = shear_states(p, 2)
    x = np.concatenate([U0, S0[:, None]], axis=1)
    coef = torch.empty((2, OS.N_COEF_SCALAR, NY, NX), dtype=torch.float32, device="cuda")
    s.network_forward(torch.tensor(x, dtype=torch.float32, device="cuda"), coef)
    torch.cuda.synchronize()
    g = coef.double().cpu().numpy()
    for b in range(2):
        assert rel_l2(g[b], O.cnn_forward(x[b], model.stencil)) <= 1e-4
    s.close()


@pytest.mark.parametrize("case", ["shear128x64", "burgers25"])
def test_learned_joint_step_matches_oracle(case):
    if case == "shear128x64":
        cfg, D = shear_cfg(), 2e-3
        p = problem(cfg)
        U0, S0 = shear_states(p, 2)
    else:
        cfg = fd.Config(n=25, batch=2, dtype="f32", flow="burgers", lx=1.0, ly=1.0, nu=1e-2, dt=1e-3, learned=True,
                        scalar_learned=True, deriv_order=2)
        D = 1e-3
        p = problem(cfg)
        U0 = f32(np.stack([I.burgers_ic(25, 40 + k) for k in range(2)]))
        S0 = f32(np.stack([I.burgers_ic(25, 50 + k)[0] + 1.0 for k in range(2)]))
    model = scalar_model(5)
    s = solver(cfg, model)
    gu, gs = gpu_joint(s, U0, S0, 1, D)
    ref = [OS.rk4_step_scalar(U0[k], S0[k], p, D, model) for k in range(2)]
    plain = [OS.rk4_step_scalar(U0[k], S0[k], p, D) for k in range(2)]
    ru, rs = np.stack([r[0] for r in ref]), np.stack([r[1] for r in ref])
    pu, ps = np.stack([r[0] for r in plain]), np.stack([r[1] for r in plain])
    assert rel_l2(gu, ru) <= 1e-5 and rel_l2(gs, rs) <= 1e-5
    err_u, err_s = rel_l2(gu - U0, ru - U0), rel_l2(gs - S0, rs - S0)
    assert err_u <= 2e-4 and err_s <= 2e-4, (err_u, err_s)
    # the learned module changed both increments by much more than the tolerance
    assert rel_l2(rs - S0, ps - S0) > 10 * err_s
    assert rel_l2(ru - U0, pu - U0) > 10 * err_u
    # the flux form keeps the total scalar
    assert abs(gs.sum() - S0.sum()) <= 1e-5 * np.abs(S0).sum()
    assert s.lib.fd_last_launch_count(s.h) == 4 * (6 + 2 + (5 if cfg.flow == "ns" else 0))
    s.close()


def test_learned_joint_rollout_with_correction_matches_oracle():
    cfg = shear_cfg(kc=2)
    model = scalar_model(11, kc=2)
    s = solver(cfg, model)
    p = problem(cfg)
    U0, S0 = shear_states(p, 2)
    for D in (1e-3, 2e-3):  # the second diffusivity replaces the captured graph
        gu, gs = gpu_joint(s, U0, S0, 4, D)
        ref = [OS.rollout_scalar(U0[k], S0[k], p, D, 4, model=model) for k in range(2)]
        ru, rs = np.stack([r[0] for r in ref]), np.stack([r[1] for r in ref])
        assert rel_l2(gu, ru) <= 1e-4 and rel_l2(gs, rs) <= 1e-4
        assert rel_l2(gs - S0, rs - S0) <= 1e-3
        assert abs(gs.sum() - S0.sum()) <= 1e-5 * np.abs(S0).sum()
    # without the correction the velocity differs by much more than the tolerance
    no_tc = O.LearnedModel(W_L=model.W_L, stencil=model.stencil, W_Ls=model.W_Ls)
    ru0 = np.stack([OS.rollout_scalar(U0[k], S0[k], p, 2e-3, 4, model=no_tc)[0] for k in range(2)])
    assert rel_l2(ru, ru0) > 10 * rel_l2(gu, ru)
    # replaying the graph again gives the same result bit for bit; the odd step
    # count runs one group from the graph and the last step directly
    gu2, gs2 = gpu_joint(s, U0, S0, 4, 2e-3)
    assert np.array_equal(gu2, gu) and np.array_equal(gs2, gs)
    gu3, gs3 = gpu_joint(s, U0, S0, 3, 2e-3)
    ref3 = [OS.rollout_scalar(U0[k], S0[k], p, 2e-3, 3, model=model) for k in range(2)]
    assert rel_l2(gu3, np.stack([r[0] for r in ref3])) <= 1e-4
    assert rel_l2(gs3, np.stack([r[1] for r in ref3])) <= 1e-4
    s.close()


def test_zero_module_gives_the_plain_joint_step():
    cfg = shear_cfg(dt=1e-2)
    p = problem(cfg)
    U0, S0 = shear_states(p, 2)
    s = solver(cfg, scalar_model(17, zero=True))
    gu, gs = gpu_joint(s, U0, S0, 3, 2e-3)
    s.close()
    plain = fd.Solver(fd.Config(n=NX, ny=NY, batch=2, dtype="f32", nu=1e-3, dt=1e-2, lx=LX, ly=LY))
    pu, ps = gpu_joint(plain, U0, S0, 3, 2e-3)
    plain.close()
    assert rel_l2(gu, pu) <= 1e-6 and rel_l2(gs, ps) <= 1e-6


def test_scalar_model_refuses_velocity_only_calls():
    cfg = shear_cfg(batch=1)
    model = scalar_model(19)
    s = fd.Solver(cfg)
    u = torch.zeros((1, 2, NY, NX), device="cuda")
    sc = torch.zeros((1, NY, NX), device="cuda")
    with pytest.raises(fd.FdError) as e:  # parameters not set
        s.rollout_scalar(u, sc, torch.empty_like(u), torch.empty_like(sc), 1, 1e-3)
    assert e.value.status == fd.FD_EINVAL
    s.set_params(I.pack_params(model.W_L, model.stencil, W_Ls=model.W_Ls))
    with pytest.raises(fd.FdError) as e:
        s.step(u, torch.empty_like(u))
    assert e.value.status == fd.FD_EUNSUPPORTED
    s.close()
    # a velocity-only learned model does not read the scalar
    v = fd.Solver(fd.Config(n=NX, ny=NY, batch=1, dtype="f32", nu=1e-3, dt=1e-2, lx=LX, ly=LY, learned=True))
    with pytest.raises(fd.FdError) as e:
        v.rollout_scalar(u, sc, torch.empty_like(u), torch.empty_like(sc), 1, 1e-3)
    assert e.value.status == fd.FD_EUNSUPPORTED
    v.close()


def test_joint_step_at_the_timed_batch_matches_oracle_on_sampled_trajectories():
    """The configuration the bench times (128 x 64, batch 16: the network's
    two-pixels-per-thread convolution variant): one joint step, the first and the
    last trajectory against the oracle."""
    b = 16
    cfg = shear_cfg(batch=b, dt=1e-2)
    p = problem(cfg)
    U0, S0 = shear_states(p, b)
    model = scalar_model(29)
    s = solver(cfg, model)
    gu, gs = gpu_joint(s, U0, S0, 1, 2e-3)
    for k in (0, b - 1):
        ru, rs = OS.rk4_step_scalar(U0[k], S0[k], p, 2e-3, model)
        assert rel_l2(gu[k], ru) <= 1e-5 and rel_l2(gs[k], rs) <= 1e-5
        assert rel_l2(gs[k] - S0[k], rs - S0[k]) <= 2e-4
    s.close()
