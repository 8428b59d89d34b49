"""GPU parity of the training runtime against the FP64 training oracle:
face-average coarse-graining, the MSE objective, Adam, the checkpointed
rollout reverse mode and the fused training step; device-side parameter
upload; and a short training run that lowers the loss of the learned solver
below that of the method without the network.

Tolerances: coarse-graining FP32 <= 1e-6 (a mean of <= 8 values), FP64
<= 1e-14; MSE <= 1e-6 (FP64 accumulation of FP32 differences); Adam <= 1e-6
(FP32 update of FP32 state); rollout reverse mode: plain <= 1e-5 (FP32, a few
steps of the 1e-5 step tolerance), learned as the one-step adjoint (state
cotangent <= 1e-4 per step, network gradients <= 2e-2).
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
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def dev(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def problem(cfg):
    return O.Problem(nx=cfg.n, ny=cfg.n, nu=cfg.nu, dt=cfg.dt,
                     flow=O.FLOW_BURGERS if cfg.flow == "burgers" else O.FLOW_NAVIER_STOKES,
                     forcing_kind=1 if cfg.forcing == "kolmogorov" else 0, deriv_order=cfg.deriv_order)


@pytest.mark.parametrize("ratio", [4, 8])
def test_downsample_matches_oracle(ratio):
    n, b = 64, 2
    p = O.Problem(nx=n, ny=n)
    rng = np.random.default_rng(ratio)
    U = np.stack([O.project(rng.standard_normal((2, n, n)), p) for _ in range(b)])
    ref = np.stack([T.face_average(U[k], ratio) for k in range(b)])
    for dtype, tol in ((torch.float32, 1e-6), (torch.float64, 1e-14)):
        fine = dev(U, dtype)
        coarse = torch.empty((b, 2, n // ratio, n // ratio), dtype=dtype, device="cuda")
        fd.downsample(fine, coarse, ratio)
        torch.cuda.synchronize()
        assert rel_l2(coarse.double().cpu().numpy(), ref) <= tol
        if dtype == torch.float64:
            for k in range(b):
                d = O.divergence(coarse[k].cpu().numpy(), ratio * p.dx, ratio * p.dy)
                assert np.max(np.abs(d)) < 1e-10


def test_mse_and_adam_match_oracle():
    s = fd.Solver(fd.Config(n=32, batch=1, dtype="f32"))
    rng = np.random.default_rng(1)
    a, b = rng.standard_normal((2, 3, 2, 32, 32)).astype(np.float32)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.empty((3, 2, 32, 32), device="cuda")
    s.mse_loss(dev(a), dev(b), loss, grad)
    torch.cuda.synchronize()
    lref, gref = T.mse_loss(a.astype(np.float64), b.astype(np.float64))
    assert abs(float(loss.item()) - lref) <= 1e-6 * lref
    assert rel_l2(grad.double().cpu().numpy(), gref) <= 1e-6
    # Adam: three steps against the oracle update
    p0, g = rng.standard_normal((2, 1000)).astype(np.float32)
    P, G = dev(p0), dev(g)
    M, V = torch.zeros_like(P), torch.zeros_like(P)
    pr, mr, vr = p0.astype(np.float64), np.zeros(1000), np.zeros(1000)
    for t in (1, 2, 3):
        G.copy_(dev(g * t))
        fd.adam_step(P, G, M, V, t, lr=1e-3)
        pr, mr, vr = T.adam_step(pr, g.astype(np.float64) * t, mr, vr, t, lr=1e-3)
    torch.cuda.synchronize()
    # FP32 parameters: one rounding of p (|p| < 4) per step dominates
    assert np.max(np.abs(P.double().cpu().numpy() - pr)) <= 1e-6 * max(1.0, float(np.max(np.abs(pr))))
    assert float(G.abs().max()) == 0.0  # gradients cleared after use


def test_plain_rollout_adjoint_with_checkpoints_matches_oracle():
    n, b, steps = 32, 2, 5
    cfg = fd.Config(n=n, batch=b, dtype="f32", nu=2e-3, dt=5e-3, forcing="kolmogorov")
    s = fd.Solver(cfg)
    U0 = I.ic_batch("kolmogorov", n, b, seed0=9)
    lam = np.random.default_rng(2).standard_normal((steps,) + U0.shape)
    lam0 = torch.empty((b, 2, n, n), device="cuda")
    s.rollout_adjoint(dev(U0), steps, 2, dev(lam), lam0)
    torch.cuda.synchronize()
    p = problem(cfg)
    U32 = U0.astype(np.float32).astype(np.float64)
    ref = np.stack([T.rollout_vjp(U32[k], p, steps, lam[:, k])[0] for k in range(b)])
    assert rel_l2(lam0.double().cpu().numpy(), ref) <= 1e-5


def make_model(seed, last_scale=0.05, wl_std=1e-2):
    st = I.random_conv_stack(seed, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=last_scale)
    return O.LearnedModel(W_L=I.random_wl(seed + 2, wl_std), stencil=st)


def test_learned_train_step_matches_oracle():
    n, b, steps = 32, 1, 3
    model = make_model(50)
    cfg = fd.Config(n=n, batch=b, dtype="f32", learned=True, nu=1e-3, dt=5e-3)
    s = fd.Solver(cfg)
    theta = dev(I.pack_params(model.W_L, model.stencil))
    s.set_params_device(theta)
    U0 = I.ic_batch("decaying", n, b, seed0=51)
    tgt = np.random.default_rng(3).standard_normal((steps,) + U0.shape) * 0.1 + U0[None]
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    dp = torch.zeros(s.param_count(), device="cuda")
    s.train_step(dev(U0), dev(tgt), steps, 2, dp, loss)
    torch.cuda.synchronize()
    p = problem(cfg)
    U32 = U0[0].astype(np.float32).astype(np.float64)
    traj, st = [], U32
    for _ in range(steps):
        st = O.learned_step(st, p, model)
        traj.append(st)
    traj = np.stack(traj)
    lref, gref = T.mse_loss(traj, tgt[:, 0].astype(np.float32).astype(np.float64))
    assert abs(float(loss.item()) - lref) <= 1e-4 * lref
    _, (wl_ref, layers_ref) = T.rollout_vjp(U32, p, steps, gref, model)
    g = dp.double().cpu().numpy()
    assert rel_l2(g[:80], wl_ref.ravel()) <= 2e-3
    o = 80
    for (W, bb), (dW, db) in zip(model.stencil, layers_ref):
        assert rel_l2(g[o:o + W.size], dW.ravel()) <= 2e-2, rel_l2(g[o:o + W.size], dW.ravel())
        o += W.size
        assert rel_l2(g[o:o + bb.size], db) <= 2e-2, rel_l2(g[o:o + bb.size], db)
        o += bb.size


def test_device_upload_equals_host_upload():
    n, b = 32, 2
    model = make_model(60, last_scale=1.0)
    flat = I.pack_params(model.W_L, model.stencil)
    a = fd.Solver(fd.Config(n=n, batch=b, dtype="f32", learned=True))
    c = fd.Solver(fd.Config(n=n, batch=b, dtype="f32", learned=True))
    a.set_params(flat)
    c.set_params_device(dev(flat))
    u = dev(I.ic_batch("decaying", n, b))
    ca = torch.empty((b, O.N_COEF, n, n), device="cuda")
    cc = torch.empty_like(ca)
    a.network_forward(u, ca)
    c.network_forward(u, cc)
    torch.cuda.synchronize()
    assert torch.equal(ca, cc)


def test_autograd_rollout_gradient_matches_rollout_adjoint():
    from paper_2507_01975_gb300.train import Rollout

    n, b, steps = 32, 1, 4
    model = make_model(70)
    s = fd.Solver(fd.Config(n=n, batch=b, dtype="f32", learned=True, nu=1e-3, dt=5e-3))
    theta = dev(I.pack_params(model.W_L, model.stencil)).requires_grad_(True)
    s.set_params_device(theta.detach())
    u0 = dev(I.ic_batch("decaying", n, b, seed0=71)).requires_grad_(True)
    traj = Rollout.apply(s, u0, theta, steps, 2)
    w = dev(np.random.default_rng(4).standard_normal((steps, b, 2, n, n)))
    (traj * w).sum().backward()
    lam0 = torch.empty_like(u0)
    dp = torch.zeros_like(theta)
    s.rollout_adjoint(u0.detach(), steps, 2, w, lam0, dp)
    torch.cuda.synchronize()
    assert rel_l2(u0.grad.double().cpu().numpy(), lam0.double().cpu().numpy()) <= 1e-5
    assert rel_l2(theta.grad.double().cpu().numpy(), dp.double().cpu().numpy()) <= 1e-3


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_vorticity_correlation_matches_oracle(dtype):
    n, b = 64, 3
    s = fd.Solver(fd.Config(n=n, batch=b, dtype=dtype))
    A_ = I.ic_batch("decaying", n, b, seed0=80)
    rng = np.random.default_rng(81)
    B_ = A_ + 0.3 * rng.standard_normal(A_.shape)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    out = torch.zeros(b, dtype=torch.float64, device="cuda")
    s.vorticity_pcc(dev(A_, tdt), dev(B_, tdt), out)
    torch.cuda.synchronize()
    h = 2 * np.pi / n
    cast = (lambda x: x) if dtype == "f64" else (lambda x: x.astype(np.float32).astype(np.float64))
    ref = [O.pcc(O.vorticity(cast(A_[k]), h, h), O.vorticity(cast(B_[k]), h, h)) for k in range(b)]
    assert np.max(np.abs(out.cpu().numpy() - np.array(ref))) <= 1e-12
    # identical fields correlate perfectly
    s.vorticity_pcc(dev(A_, tdt), dev(A_, tdt), out)
    torch.cuda.synchronize()
    assert np.max(np.abs(out.cpu().numpy() - 1.0)) <= 1e-12


def test_vorticity_correlation_on_a_rectangular_grid_matches_oracle():
    # generic-grid context: 40 x 24 cells on [0, 1] x [0, 0.6] (unequal spacings)
    nx, ny, b = 40, 24, 2
    s = fd.Solver(fd.Config(n=nx, ny=ny, batch=b, dtype="f32", flow="burgers", lx=1.0, ly=0.6, nu=1e-2, dt=1e-3))
    rng = np.random.default_rng(82)
    A_ = rng.standard_normal((b, 2, ny, nx)).astype(np.float32).astype(np.float64)
    B_ = (A_ + 0.5 * rng.standard_normal(A_.shape)).astype(np.float32).astype(np.float64)
    out = torch.zeros(b, dtype=torch.float64, device="cuda")
    s.vorticity_pcc(dev(A_), dev(B_), out)
    torch.cuda.synchronize()
    dx, dy = 1.0 / nx, 0.6 / ny
    ref = [O.pcc(O.vorticity(A_[k], dx, dy), O.vorticity(B_[k], dx, dy)) for k in range(b)]
    assert np.max(np.abs(out.cpu().numpy() - np.array(ref))) <= 1e-12


def test_batch_of_mixed_rollouts_equals_individual_rollouts():
    # one graph with a branch per context: plain on-chip (Burgers 32^2, NS 64^2),
    # learned 32^2, and the streaming path at 64^2
    specs = [
        (fd.Config(n=32, batch=2, dtype="f32", flow="burgers", nu=1e-2, dt=2e-3, deriv_order=2), "burgers", 10, None),
        (fd.Config(n=64, batch=2, dtype="f32", nu=1e-3, dt=5e-3), "decaying", 5, None),
        (fd.Config(n=32, batch=2, dtype="f32", nu=1e-3, dt=1e-2, learned=True), "kolmogorov", 4, make_model(90)),
        (fd.Config(n=64, batch=1, dtype="f32", nu=1e-3, dt=5e-3, path=2), "decaying", 3, None),
    ]
    batch = fd.Batch()
    runs = []
    for cfg, kind, steps, model in specs:
        s = fd.Solver(cfg)
        if model is not None:
            s.set_params(I.pack_params(model.W_L, model.stencil))
        u0 = dev(I.ic_batch(kind, cfg.n, cfg.batch, seed0=91))
        out = torch.empty_like(u0)
        ref = torch.empty_like(u0)
        s.rollout(u0, ref, steps)
        batch.add(s, u0, out, steps)
        runs.append((out, ref))
    batch.run()
    batch.run()  # replay
    torch.cuda.synchronize()
    assert batch.launch_count() > 0
    for out, ref in runs:
        assert torch.equal(out, ref)
