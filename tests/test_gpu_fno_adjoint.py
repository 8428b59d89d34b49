"""GPU reverse mode of the Fourier operators and of the ablation variants
against the FP64 oracle.

The frequency-domain operator O_F (Sec. 3.4) is differentiated inside the
learned step: its output cotangent is the face-value cotangent of the flux-block
reverse kernel, its input cotangent joins the state cotangent, and its
parameters (lift, every layer's complex mode matrices, channel maps, biases,
projection) get their gradients. The FNO temporal correction (Sec. 3.5) is the
same operator on the stacked history. Compared with ``oracle.adjoint.step_vjp``,
``temporal_correction_vjp`` and ``oracle.train.rollout_vjp_full`` through
``flat_grads`` (the parameter-array layout).

Tolerances: state cotangents <= 1e-4 (FP32 operators; the BF16 stencil network
only touches the learned part of the kernels); W_L <= 1e-3; stencil network
layers <= 2e-2 (BF16); O_F parameters <= 2e-3 per block (FP32 operators fed by
face-value cotangents that carry the BF16 network's share, ~1e-4, amplified in
the bias gradients by the cancellation of their pixel sums); the FNO correction
alone (no network upstream) <= 1e-5 for the history cotangents and its
parameters, in a training step <= 2e-3. The correction's last-layer bias and
projection-bias gradients are zero in exact arithmetic (the mean removal makes
its output cotangent sum to zero over the pixels), so they are held to 1e-5 of
that cotangent's summed magnitude instead of a relative bound.
"""

import numpy as np
import pytest

import oracle as O
from oracle import train as T
from paper_2507_01975_gb300 import fd
from paper_2507_01975_gb300 import inputs as I

from oracle_jobs import rollout_vjp_job, run_pool, step_vjp_job, tc_vjp_job

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


def _fno_blocks(prm):
    """(name, size) of the flat blocks of one operator, in the parameter layout."""
    out = [("P_w", prm.P_w.size), ("P_b", prm.P_b.size)]
    for l in range(prm.layers):
        out += [(f"R{l}", prm.R[l].size * 2), (f"W{l}", prm.W[l].size), (f"b{l}", prm.Wb[l].size)]
    return out + [("Q_w", prm.Q_w.size), ("Q_b", prm.Q_b.size)]


def _check_operator(g, want, o, prm, tol, what, zero_sum_mass=None):
    """Block-wise comparison of one operator's gradients. With zero_sum_mass (the
    summed magnitude of an output cotangent that sums to zero), the last layer's
    bias and the projection bias are zero in exact arithmetic and are held to
    1e-5 of that mass."""
    zero = {f"b{prm.layers - 1}", "Q_b"} if zero_sum_mass is not None else set()
    for name, size in _fno_blocks(prm):
        if name in zero:
            scale = zero_sum_mass * max(1.0, float(np.abs(prm.Q_w).max()))
            assert np.max(np.abs(g[o:o + size] - want[o:o + size])) <= 1e-5 * scale, (what, name)
        else:
            err = rel_l2(g[o:o + size], want[o:o + size])
            assert err <= tol, (what, name, err)
        o += size
    return o


def _model(seed, n, width, modes, layers, ablation=0, kc=0, tc_fno=None):
    st = I.random_conv_stack(seed, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=0.05)
    fno = I.random_fno(seed + 3, width, modes, layers, out_scale=0.3) if layers else None
    m = O.LearnedModel(W_L=I.random_wl(seed + 2, 1e-2), stencil=st, fno=None if fno is None else O.FNOParams(**fno),
                       ablation=ablation, k_c=kc, tc_fno=None if tc_fno is None else O.FNOParams(**tc_fno))
    return m, fno


def _solver(n, b, m, fno, tc_fno=None, forcing="kolmogorov", flow="ns", dt=5e-3):
    cfg = fd.Config(n=n, batch=b, dtype="f32", nu=1e-3, dt=dt, forcing=forcing if flow == "ns" else None, flow=flow,
                    learned=True, ablation=m.ablation, k_c=m.k_c,
                    fno_layers=0 if fno is None else len(fno["R"]), fno_modes=0 if fno is None else fno["R"][0].shape[1],
                    fno_width=0 if fno is None else fno["P_w"].shape[0],
                    tc_fno_layers=0 if tc_fno is None else len(tc_fno["R"]),
                    tc_fno_modes=0 if tc_fno is None else tc_fno["R"][0].shape[1],
                    tc_fno_width=0 if tc_fno is None else tc_fno["P_w"].shape[0])
    s = fd.Solver(cfg)
    s.set_params(I.pack_params(m.W_L, m.stencil, tc_fno, fno))
    return s


def _problem(s):
    c = s.cfg
    return O.Problem(nx=c.n, ny=c.n, nu=c.nu, dt=c.dt, flow=O.FLOW_BURGERS if c.flow == "burgers" else
                     O.FLOW_NAVIER_STOKES, forcing_kind=1 if c.forcing == "kolmogorov" else 0)


def _flat_step(ref, m):
    g = {"W_L": ref[1][0], "stencil": ref[1][1], "fno": ref[1][2] if len(ref[1]) > 2 else None, "tc": None}
    return T.flat_grads(g, m)


@pytest.mark.parametrize("n,width,modes,layers,ablation,flow", [
    (32, 8, 8, 2, 0, "ns"), (64, 16, 16, 4, 0, "ns"), (32, 8, 8, 2, 1, "ns"), (32, 8, 8, 2, 2, "ns"),
    (32, 8, 8, 3, 0, "burgers"), (32, 0, 0, 0, 1, "burgers")])
def test_step_adjoint_with_frequency_operator_and_ablations(n, width, modes, layers, ablation, flow):
    b = 2
    m, fno = _model(111 + n + ablation, n, width, modes, layers, ablation=ablation)
    s = _solver(n, b, m, fno, flow=flow)
    p = _problem(s)
    U0 = I.ic_batch("burgers" if flow == "burgers" else "kolmogorov", n, b, seed0=112).astype(np.float32)
    lam = np.random.default_rng(113).standard_normal(U0.shape).astype(np.float32)
    u = torch.tensor(U0, device="cuda")
    lo = torch.tensor(lam, device="cuda")
    li = torch.empty_like(u)
    dp = torch.zeros(s.param_count(), dtype=torch.float32, device="cuda")
    s.step_adjoint(u, lo, li, dp)
    torch.cuda.synchronize()
    refs = run_pool(step_vjp_job, [(U0[k].astype(np.float64), p, lam[k].astype(np.float64), m) for k in range(b)])
    assert rel_l2(li.double().cpu().numpy(), np.stack([r[0] for r in refs])) <= 1e-4
    g = dp.double().cpu().numpy()
    want = sum(_flat_step(r, m) for r in refs)
    assert g.size == want.size
    if ablation != 2:
        assert rel_l2(g[:80], want[:80]) <= 1e-3
        o = 80
        for W, bb in m.stencil:
            assert rel_l2(g[o:o + W.size], want[o:o + W.size]) <= 2e-2
            assert rel_l2(g[o + W.size:o + W.size + bb.size], want[o + W.size:o + W.size + bb.size]) <= 2e-2
            o += W.size + bb.size
    else:
        o = 80 + sum(W.size + bb.size for W, bb in m.stencil)
        assert np.all(g[:o] == 0.0)  # no kernels: no W_L or network gradient
    if m.fno is not None:
        _check_operator(g, want, o, m.fno, 2e-3, "O_F")
    s.close()


@pytest.mark.parametrize("n,kc,width,modes,layers", [(32, 2, 8, 8, 2), (64, 4, 8, 32, 4)])
def test_fno_temporal_correction_adjoint(n, kc, width, modes, layers):
    b = 2
    tcf = I.random_fno(121 + n, width, modes, layers, out_scale=0.5, cin=2 * kc, cout=2)
    m, _ = _model(122, n, 0, 0, 0, kc=kc, tc_fno=tcf)
    s = _solver(n, b, m, None, tc_fno=tcf)
    p = _problem(s)
    hist = np.stack([np.stack([I.kolmogorov_ic(n, 10 * t + k) for k in range(b)]) for t in range(kc)]).astype(np.float32)
    lam = np.random.default_rng(123).standard_normal((b, 2, n, n)).astype(np.float32)
    h = torch.tensor(hist, device="cuda")
    lo = torch.tensor(lam, device="cuda")
    hb = torch.full_like(h, float("nan"))
    vb = torch.empty_like(lo)
    dp = torch.zeros(s.param_count(), dtype=torch.float32, device="cuda")
    s.tc_adjoint(h, lo, hb, vbar=vb, dparams=dp)
    torch.cuda.synchronize()
    refs = run_pool(tc_vjp_job, [(hist[-1, k].astype(np.float64), [hist[t, k].astype(np.float64) for t in range(kc)],
                                  p, m, lam[k].astype(np.float64)) for k in range(b)])
    assert rel_l2(vb.double().cpu().numpy(), np.stack([r[0] for r in refs])) <= 1e-5
    want_h = np.stack([np.stack([refs[k][1][t] for k in range(b)]) for t in range(kc)])
    assert rel_l2(hb.double().cpu().numpy(), want_h) <= 1e-5
    g = dp.double().cpu().numpy()
    o = 80 + sum(W.size + bb.size for W, bb in m.stencil)
    assert np.all(g[:o] == 0.0)
    want = T.flat_grads({"W_L": None, "stencil": None, "fno": None,
                         "tc": A_sum([r[2] for r in refs])}, m)
    mass = sum(np.abs(r[0] - r[0].mean(axis=(1, 2), keepdims=True)).sum() for r in refs)
    _check_operator(g, want, o, m.tc_fno, 1e-5, "FNO correction", zero_sum_mass=mass)
    s.close()


def A_sum(gs):
    from oracle import adjoint as A

    acc = gs[0]
    for x in gs[1:]:
        acc = A._fno_sum(acc, x)
    return acc


def test_train_step_of_the_full_model_matches_oracle():
    # stencil network + O_F + FNO temporal correction (the paper's forced-flow
    # learnable module, small): the fused training step's loss and gradient
    n, b, kc, steps = 32, 2, 2, 4
    tcf = I.random_fno(131, 8, 8, 2, out_scale=0.3, cin=2 * kc, cout=2)
    m, fno = _model(132, n, 8, 8, 2, kc=kc, tc_fno=tcf)
    s = _solver(n, b, m, fno, tc_fno=tcf)
    p = _problem(s)
    U0 = np.stack([I.kolmogorov_ic(n, 133 + k) for k in range(b)]).astype(np.float32)
    targets = (0.9 * np.stack([np.stack([I.kolmogorov_ic(n, 300 + 10 * t + k) for k in range(b)])
                               for t in range(steps)])).astype(np.float32)
    u = torch.tensor(U0, device="cuda")
    tg = torch.tensor(targets, device="cuda")
    dp = torch.zeros(s.param_count(), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.train_step(u, tg, steps, 2, dp, loss)
    torch.cuda.synchronize()
    states = [T.rollout_states(U0[k].astype(np.float64), p, steps, m)[0] for k in range(b)]
    pred = np.stack([np.stack(st_[1:]) for st_ in states], axis=1)
    want_loss = float(np.mean((pred - targets) ** 2))
    assert abs(float(loss.item()) - want_loss) <= 1e-5 * want_loss
    lam_traj = 2.0 * (pred - targets) / pred.size
    refs = run_pool(rollout_vjp_job, [(U0[k].astype(np.float64), p, steps, lam_traj[:, k], m) for k in range(b)])
    want = sum(r[1] for r in refs)
    g = dp.double().cpu().numpy()
    assert g.size == want.size
    assert rel_l2(g[:80], want[:80]) <= 1e-3
    o = 80
    for W, bb in m.stencil:
        assert rel_l2(g[o:o + W.size], want[o:o + W.size]) <= 2e-2
        o += W.size + bb.size
    # the correction's zero-sum blocks: scale by the largest state cotangent mass
    mass = float(np.abs(lam_traj).sum())
    o = _check_operator(g, want, o, m.tc_fno, 2e-3, "FNO correction", zero_sum_mass=mass)
    _check_operator(g, want, o, m.fno, 2e-3, "O_F")
    s.close()
