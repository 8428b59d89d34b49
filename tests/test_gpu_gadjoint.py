"""GPU parity of the reverse mode on the generic-grid path (FP32, CUDA cores)
against the FP64 oracle's hand-derived VJPs.

Grids: the 25^2 Burgers preset on [0, 1]^2 (App. C.1), a ragged 40 x 24 Burgers
grid with unequal spacings, and the 128 x 64 Navier-Stokes grid on [0, 8] x
[0, 4] (the shear-flow grid of Table S2). Plain and learned steps (the full
operator and the variant without the physics convolution), the temporal
correction, and a checkpointed training step with corrections. The network
weights are BF16-representable (the oracle takes the same weights in FP64);
activations and every reverse product are FP32. Bars: state cotangents
<= 1e-5 (plain) and <= 1e-4 (learned) relative L2; parameter gradients per
block (W_L, each layer's weights and biases) <= 1e-3.
"""

import numpy as np
import pytest

import oracle as O
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
    "burgers25": dict(n=25, dtype="f32", flow="burgers", lx=1.0, ly=1.0, nu=1e-2, dt=1e-3),
    "burgers40x24": dict(n=40, ny=24, dtype="f32", flow="burgers", lx=1.0, ly=0.6, nu=1e-2, dt=1e-3, deriv_order=2),
    "ns128x64": dict(n=128, ny=64, dtype="f32", lx=8.0, ly=4.0, nu=1e-3, dt=5e-3),
}


def problem(cfg):
    return O.Problem(nx=cfg.n, ny=cfg.ny or cfg.n, lx=cfg.lx, ly=cfg.ly, nu=cfg.nu, dt=cfg.dt,
                     flow=O.FLOW_BURGERS if cfg.flow == "burgers" else O.FLOW_NAVIER_STOKES,
                     forcing_kind=1 if cfg.forcing == "kolmogorov" else 0, amp=cfg.amp, kf=cfg.kf, drag=cfg.drag,
                     deriv_order=cfg.deriv_order)


def smooth(nx, ny, seed):
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.arange(ny) / ny, np.arange(nx) / nx, indexing="ij")
    U = np.zeros((2, ny, nx))
    for c in range(2):
        for _ in range(4):
            kx, ky = rng.integers(-3, 4, size=2)
            U[c] += rng.standard_normal() * np.sin(2 * np.pi * (kx * x + ky * y) + rng.uniform(0, 2 * np.pi))
    return U


def states(cfg, b, seed):
    p = problem(cfg)
    U = np.stack([smooth(p.nx, p.ny, seed + k) for k in range(b)])
    if p.flow == O.FLOW_NAVIER_STOKES:
        U = np.stack([O.project(U[k], p) for k in range(b)])
    return f32(U)


def model(seed, kc=0, ablation=0, last_scale=0.05):
    st = I.random_conv_stack(seed, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=last_scale)
    tc = I.random_conv_stack(seed + 1, 2 * kc, O.CNN_HIDDEN, 2, last_scale=0.02) if kc else []
    return O.LearnedModel(W_L=I.random_wl(seed + 2, 1e-2), stencil=st, tc=tc, k_c=kc, ablation=ablation)


def check_grads(g, wl_ref, layers_ref, m, tol=1e-3, tc_ref=None):
    assert rel_l2(g[:80], wl_ref.ravel()) <= tol, ("W_L", rel_l2(g[:80], wl_ref.ravel()))
    o = 80
    for l, ((W, bb), (dW, db)) in enumerate(zip(m.stencil, layers_ref)):
        assert rel_l2(g[o:o + W.size], dW.ravel()) <= tol, ("W", l, rel_l2(g[o:o + W.size], dW.ravel()))
        o += W.size
        assert rel_l2(g[o:o + bb.size], db) <= tol, ("b", l, rel_l2(g[o:o + bb.size], db))
        o += bb.size
    for l, ((W, bb), (dW, db)) in enumerate(zip(m.tc, tc_ref or [])):
        assert rel_l2(g[o:o + W.size], dW.ravel()) <= tol, ("tc W", l, rel_l2(g[o:o + W.size], dW.ravel()))
        o += W.size
        check_bias(g[o:o + bb.size], db, dW, tol, last=l == len(m.tc) - 1)
        o += bb.size


def check_bias(got, ref, dW, tol, last):
    """The correction network's last bias sees the mean-free cotangent c_bar, so its
    gradient (a sum of c_bar over the pixels) is zero in exact arithmetic: there
    only the FP32 rounding residue of that sum remains, bounded against the
    layer's weight gradient."""
    if last:
        assert np.abs(ref).max() <= 1e-9 * np.linalg.norm(dW)
        assert np.abs(got).max() <= 1e-6 * np.linalg.norm(dW), (got, np.linalg.norm(dW))
    else:
        assert rel_l2(got, ref) <= tol, ("tc b", rel_l2(got, ref))


@pytest.mark.parametrize("case", list(CASES))
def test_plain_step_adjoint_matches_oracle(case):
    cfg = fd.Config(batch=2, path=3, **CASES[case])
    s = fd.Solver(cfg)
    U = states(cfg, 2, 3)
    lam = np.random.default_rng(4).standard_normal(U.shape)
    li = torch.empty_like(dev(U))
    s.step_adjoint(dev(U), dev(lam), li)
    torch.cuda.synchronize()
    p = problem(cfg)
    ref = np.stack([A.step_vjp(U[k], p, lam[k])[0] for k in range(2)])
    assert rel_l2(li.double().cpu().numpy(), ref) <= 1e-5
    s.close()


@pytest.mark.parametrize("case,ablation", [("burgers25", 0), ("burgers25", 1), ("burgers40x24", 0), ("ns128x64", 0)])
def test_learned_step_adjoint_matches_oracle(case, ablation):
    cfg = fd.Config(batch=2, learned=True, ablation=ablation, **CASES[case])
    m = model(7, ablation=ablation)
    s = fd.Solver(cfg)
    s.set_params(I.pack_params(m.W_L, m.stencil))
    U = states(cfg, 2, 5)
    lam = np.random.default_rng(6).standard_normal(U.shape)
    li = torch.empty_like(dev(U))
    dp = torch.zeros(s.param_count(), device="cuda")
    lam_d = dev(lam)
    s.step_adjoint(dev(U), lam_d, li, dp)
    torch.cuda.synchronize()
    p = problem(cfg)
    refs = [A.step_vjp(U[k], p, lam[k], m) for k in range(2)]
    ref = np.stack([r[0] for r in refs])
    assert rel_l2(li.double().cpu().numpy(), ref) <= 1e-4
    wl = sum(r[1][0] for r in refs)
    layers = [(sum(r[1][1][l][0] for r in refs), sum(r[1][1][l][1] for r in refs)) for l in range(6)]
    check_grads(dp.double().cpu().numpy(), wl, layers, m)
    # the learned module's cotangent differs from the plain step's by far more than the bar
    plain = np.stack([A.step_vjp(U[k], p, lam[k])[0] for k in range(2)])
    assert rel_l2(ref, plain) > 10 * rel_l2(li.double().cpu().numpy(), ref)
    # lam_in may alias lam_out; a second call accumulates the same gradient again
    s.step_adjoint(dev(U), lam_d, lam_d, dp)
    torch.cuda.synchronize()
    assert rel_l2(lam_d.double().cpu().numpy(), ref) <= 1e-4
    check_grads(dp.double().cpu().numpy(), 2 * wl, [(2 * a, 2 * b) for a, b in layers], m)
    s.close()


def test_temporal_correction_adjoint_on_the_shear_grid_matches_oracle():
    kc = 2
    cfg = fd.Config(batch=2, learned=True, k_c=kc, **CASES["ns128x64"])
    m = model(11, kc=kc)
    s = fd.Solver(cfg)
    s.set_params(I.pack_params(m.W_L, m.stencil, m.tc))
    p = problem(cfg)
    hist = np.stack([states(cfg, 2, 20 + 3 * q) for q in range(kc)])  # [kc, b, 2, ny, nx]
    lam = np.random.default_rng(8).standard_normal(hist.shape[1:])
    hb = torch.empty_like(dev(hist))
    vb = torch.empty_like(dev(lam))
    dp = torch.zeros(s.param_count(), device="cuda")
    s.tc_adjoint(dev(hist), dev(lam), hb, vb, dp)
    torch.cuda.synchronize()
    refs = [A.temporal_correction_vjp(np.zeros_like(lam[k]), [hist[q, k] for q in range(kc)], p, m, lam[k])
            for k in range(2)]
    assert rel_l2(vb.double().cpu().numpy(), np.stack([r[0] for r in refs])) <= 1e-5
    href = np.stack([np.stack(r[1]) for r in refs], axis=1)
    assert rel_l2(hb.double().cpu().numpy(), href) <= 1e-4
    g = dp.double().cpu().numpy()
    n_st = 80 + sum(W.size + b.size for W, b in m.stencil)
    assert not g[:n_st].any()
    o = n_st
    for l, (W, bb) in enumerate(m.tc):
        dW = sum(r[2][l][0] for r in refs)
        db = sum(r[2][l][1] for r in refs)
        assert rel_l2(g[o:o + W.size], dW.ravel()) <= 1e-3, ("tc W", l)
        o += W.size
        check_bias(g[o:o + bb.size], db, dW, 1e-3, last=l == len(m.tc) - 1)
        o += bb.size
    s.close()


@pytest.mark.parametrize("case", ["burgers25", "ns128x64"])
def test_train_step_with_corrections_matches_oracle(case):
    """MSE of a 4-step rollout with a correction every 2 steps, checkpoints every 2
    steps: the loss and every parameter block against the oracle's rollout VJP."""
    kc, steps = 2, 4
    cfg = fd.Config(batch=1, learned=True, k_c=kc, **CASES[case])
    m = model(13, kc=kc)
    s = fd.Solver(cfg)
    s.set_params_device(dev(I.pack_params(m.W_L, m.stencil, m.tc)))
    p = problem(cfg)
    U0 = states(cfg, 1, 30)
    states_ref, _ = T.rollout_states(U0[0], p, steps, m)
    tgt = np.stack(states_ref[1:])[:, None] + 0.05 * np.random.default_rng(9).standard_normal((steps,) + U0.shape)
    tgt = f32(tgt)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    dp = torch.zeros(s.param_count(), device="cuda")
    s.train_step(dev(U0), dev(tgt), steps, 2, dp, loss)
    torch.cuda.synchronize()
    traj = np.stack(states_ref[1:])
    lref, gref = T.mse_loss(traj, tgt[:, 0])
    assert abs(float(loss.item()) - lref) <= 1e-4 * lref
    _, g = T.rollout_vjp_full(U0[0], p, steps, gref, m)
    flat = T.flat_grads(g, m)
    got = dp.double().cpu().numpy()
    assert got.shape == flat.shape
    check_grads(got, g["W_L"], g["stencil"], m, tol=2e-3, tc_ref=g["tc"])
    s.close()


def test_reverse_mode_refusals():
    cfg = fd.Config(batch=1, learned=True, **CASES["burgers25"])
    s = fd.Solver(cfg)
    u = torch.zeros((1, 2, 25, 25), device="cuda")
    with pytest.raises(fd.FdError) as e:  # parameters not set
        s.step_adjoint(u, u, torch.empty_like(u))
    assert e.value.status == fd.FD_EINVAL
    s.close()
    # FP64 generic-grid contexts have no reverse mode
    s = fd.Solver(fd.Config(batch=1, **dict(CASES["burgers25"], dtype="f64")))
    ud = torch.zeros((1, 2, 25, 25), dtype=torch.float64, device="cuda")
    with pytest.raises(fd.FdError) as e:
        s.step_adjoint(ud, ud, torch.empty_like(ud))
    assert e.value.status == fd.FD_EUNSUPPORTED
    s.close()
    # a plain context takes no parameter gradient
    s = fd.Solver(fd.Config(batch=1, **CASES["burgers25"]))
    with pytest.raises(fd.FdError) as e:
        s.step_adjoint(u, u, torch.empty_like(u), torch.zeros(8, device="cuda"))
    assert e.value.status == fd.FD_EINVAL
    s.close()
