"""GPU reverse mode of the temporal correction (CNN head) against the FP64 oracle.

fd_tc_adjoint differentiates one correction u_k = P(V + c - mean(c)),
c = TC(u_{k-k_c} .. u_{k-1}) (Sec. 3.2, Sec. 3.5); fd_rollout_adjoint and
fd_train_step route every corrected state's cotangent back to its history
window. Compared with ``oracle.adjoint.temporal_correction_vjp`` and
``oracle.train.rollout_vjp_full``.

Tolerances: vbar = P(lam) <= 1e-5 (FP32 projection); the history cotangents
and the network's weight gradients come out of the BF16 network and are held
to its 2e-2 relative bound, except the hidden layers' bias gradients: a bias
gradient is a pixel sum of a cotangent whose terms largely cancel, so the BF16
rounding of the activations upstream of it is amplified by that cancellation
(the sums themselves are taken in FP32); they are held to 3e-2 (measured at
most 2.3e-2 over these cases). The last layer's bias gradient is zero in exact
arithmetic (the mean removal makes the output cotangent sum to zero), so it is
held to 2e-2 of the summed magnitude of that cotangent instead. Rollout
cotangents: <= 2e-3 (the network parts are a small share of them), W_L
<= 1e-3, network layers <= 2e-2.
"""

import numpy as np
import pytest

import oracle as O
from paper_2507_01975_gb300 import fd
from paper_2507_01975_gb300 import inputs as I

from oracle_jobs import rollout_vjp_job, run_pool, tc_vjp_job

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


def _model(seed, kc, tc_scale=0.5, st_scale=0.05):
    st = I.random_conv_stack(seed, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=st_scale)
    tc = I.random_conv_stack(seed + 1, 2 * kc, O.CNN_HIDDEN, 2, last_scale=tc_scale)
    return O.LearnedModel(W_L=I.random_wl(seed + 2, 1e-2), stencil=st, tc=tc, k_c=kc)


def _solver(n, b, model, flow="ns", forcing="kolmogorov", dt=5e-3):
    s = fd.Solver(fd.Config(n=n, batch=b, dtype="f32", flow=flow, forcing=forcing if flow == "ns" else None, nu=1e-3,
                            dt=dt, learned=True, k_c=model.k_c))
    s.set_params(I.pack_params(model.W_L, model.stencil, model.tc))
    return s


def _problem(s):
    c = s.cfg
    return O.Problem(nx=c.n, ny=c.n, nu=c.nu, dt=c.dt, flow=O.FLOW_BURGERS if c.flow == "burgers" else
                     O.FLOW_NAVIER_STOKES, forcing_kind=1 if c.forcing == "kolmogorov" else 0)


def _tc_offsets(model):
    o = 80 + sum(W.size + b.size for W, b in model.stencil)
    offs = []
    for W, b in model.tc:
        offs.append((o, o + W.size, o + W.size + b.size))
        o += W.size + b.size
    return offs


@pytest.mark.parametrize("n,kc,flow", [(32, 2, "ns"), (64, 4, "ns"), (32, 3, "burgers")])
def test_tc_adjoint_matches_oracle(n, kc, flow):
    b = 2
    model = _model(91 + n + kc, kc)
    s = _solver(n, b, model, flow=flow)
    p = _problem(s)
    rng = np.random.default_rng(92)
    hist = np.stack([np.stack([(I.burgers_ic(n, 10 * t + k) if flow == "burgers" else I.kolmogorov_ic(n, 10 * t + k))
                               for k in range(b)]) for t in range(kc)]).astype(np.float32)
    lam = rng.standard_normal((b, 2, n, n)).astype(np.float32)
    h = torch.tensor(hist, device="cuda")
    lo = torch.tensor(lam, device="cuda")
    hb = torch.full_like(h, float("nan"))
    vb = torch.empty_like(lo)
    dp = torch.zeros(s.param_count(), dtype=torch.float32, device="cuda")
    s.tc_adjoint(h, lo, hb, vbar=vb, dparams=dp)
    torch.cuda.synchronize()
    refs = run_pool(tc_vjp_job, [(hist[-1, k].astype(np.float64), [hist[t, k].astype(np.float64) for t in range(kc)],
                                  p, model, lam[k].astype(np.float64)) for k in range(b)])
    assert rel_l2(vb.double().cpu().numpy(), np.stack([r[0] for r in refs])) <= 1e-5
    want_h = np.stack([np.stack([refs[k][1][t] for k in range(b)]) for t in range(kc)])
    assert rel_l2(hb.double().cpu().numpy(), want_h) <= 2e-2
    g = dp.double().cpu().numpy()
    assert np.all(g[:80 + sum(W.size + bb.size for W, bb in model.stencil)] == 0.0)  # only the correction's part
    for l, (o0, o1, o2) in enumerate(_tc_offsets(model)):
        dW = sum(r[2][l][0] for r in refs).ravel()
        db = sum(r[2][l][1] for r in refs)
        assert rel_l2(g[o0:o1], dW) <= 2e-2, (l, rel_l2(g[o0:o1], dW))
        if l < 5:
            assert rel_l2(g[o1:o2], db) <= 3e-2, (l, rel_l2(g[o1:o2], db))
        else:
            cbar_mass = sum(np.abs(r[0] - r[0].mean(axis=(1, 2), keepdims=True)).sum() for r in refs)
            assert np.max(np.abs(g[o1:o2] - db)) <= 2e-2 * cbar_mass
    s.close()


@pytest.mark.parametrize("n_steps,ckpt", [(6, 4), (5, 2)])
def test_rollout_adjoint_with_temporal_correction_matches_oracle(n_steps, ckpt):
    n, b, kc = 32, 2, 2
    model = _model(95, kc, tc_scale=0.3)
    s = _solver(n, b, model)
    p = _problem(s)
    rng = np.random.default_rng(96)
    U0 = np.stack([I.kolmogorov_ic(n, 97 + k) for k in range(b)]).astype(np.float32)
    lam_traj = rng.standard_normal((n_steps, b, 2, n, n)).astype(np.float32)
    u = torch.tensor(U0, device="cuda")
    lt = torch.tensor(lam_traj, device="cuda")
    l0 = torch.empty_like(u)
    dp = torch.zeros(s.param_count(), dtype=torch.float32, device="cuda")
    s.rollout_adjoint(u, n_steps, ckpt, lt, l0, dp)
    torch.cuda.synchronize()
    refs = run_pool(rollout_vjp_job, [(U0[k].astype(np.float64), p, n_steps, lam_traj[:, k].astype(np.float64), model)
                                      for k in range(b)])
    want0 = np.stack([r[0] for r in refs])
    assert rel_l2(l0.double().cpu().numpy(), want0) <= 2e-3
    g = dp.double().cpu().numpy()
    want = sum(r[1] for r in refs)
    assert rel_l2(g[:80], want[:80]) <= 1e-3
    o = 80
    for W, bb in list(model.stencil) + list(model.tc)[:5]:
        assert rel_l2(g[o:o + W.size], want[o:o + W.size]) <= 2e-2
        o += W.size + bb.size
    W5 = model.tc[5][0]
    assert rel_l2(g[o:o + W5.size], want[o:o + W5.size]) <= 2e-2
    # the correction is live: without its history cotangents the answer moves far
    no_tc = O.LearnedModel(W_L=model.W_L, stencil=model.stencil)
    ref_plain = run_pool(rollout_vjp_job, [(U0[0].astype(np.float64), p, n_steps, lam_traj[:, 0].astype(np.float64),
                                            no_tc)])[0][0]
    assert rel_l2(ref_plain, want0[0]) > 10 * rel_l2(l0[0].double().cpu().numpy(), want0[0])
    s.close()


def test_train_step_with_temporal_correction_matches_oracle():
    n, b, kc, steps = 32, 2, 2, 4
    model = _model(98, kc, tc_scale=0.3)
    s = _solver(n, b, model)
    p = _problem(s)
    U0 = np.stack([I.kolmogorov_ic(n, 99 + k) for k in range(b)]).astype(np.float32)
    targets = np.stack([np.stack([I.kolmogorov_ic(n, 200 + 10 * t + k) for k in range(b)]) for t in range(steps)])
    targets = (0.9 * targets).astype(np.float32)
    u = torch.tensor(U0, device="cuda")
    tg = torch.tensor(targets, device="cuda")
    dp = torch.zeros(s.param_count(), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.train_step(u, tg, steps, 2, dp, loss)
    torch.cuda.synchronize()
    from oracle import train as T

    states = [T.rollout_states(U0[k].astype(np.float64), p, steps, model)[0] for k in range(b)]
    pred = np.stack([np.stack(st[1:]) for st in states], axis=1)  # [steps][b]...
    want_loss = float(np.mean((pred - targets) ** 2))
    assert abs(float(loss.item()) - want_loss) <= 1e-5 * want_loss
    lam_traj = 2.0 * (pred - targets) / pred.size
    refs = run_pool(rollout_vjp_job, [(U0[k].astype(np.float64), p, steps, lam_traj[:, k], model) for k in range(b)])
    want = sum(r[1] for r in refs)
    g = dp.double().cpu().numpy()
    o = 80 + sum(W.size + bb.size for W, bb in model.stencil)
    for l, (W, bb) in enumerate(model.tc):
        assert rel_l2(g[o:o + W.size], want[o:o + W.size]) <= 2e-2, l
        o += W.size + bb.size
    with pytest.raises(fd.FdError) as ei:
        s.train_step(u, tg, steps, 3, dp, loss)  # checkpoint interval not a multiple of k_c
    assert ei.value.status == fd.FD_EINVAL
    s.close()
