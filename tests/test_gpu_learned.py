"""GPU parity of the learnable module (tensor-core network, learned flux block,
consistency projection, temporal correction) against the FP64 oracle.

Tolerances: BF16 network outputs <= 2e-2 relative L2 (the network runs in BF16
with FP32 accumulation; the oracle uses the same BF16-rounded weights in FP64);
a learned FP32 step <= 1e-4 (the BF16 network perturbs the small learned part of
the kernels only); reduction to the plain solver <= 1e-6.
"""

import numpy as np
import pytest

import oracle as O
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


def make_model(seed, last_scale, kc=0, wl_std=1e-3, tc_scale=0.02):
    st = I.random_conv_stack(seed, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=last_scale)
    tc = I.random_conv_stack(seed + 1, 2 * kc, O.CNN_HIDDEN, 2, last_scale=tc_scale) if kc else []
    return O.LearnedModel(W_L=I.random_wl(seed + 2, wl_std), stencil=st, tc=tc, k_c=kc)


def solver(n, batch, model, **kw):
    cfg = fd.Config(n=n, batch=batch, dtype="f32", learned=True, k_c=model.k_c, **kw)
    s = fd.Solver(cfg)
    s.set_params(I.pack_params(model.W_L, model.stencil, model.tc))
    return s


def oracle_problem(s: fd.Solver) -> O.Problem:
    c = s.cfg
    return O.Problem(nx=c.n, ny=c.n, nu=c.nu, dt=c.dt,
                     flow=O.FLOW_BURGERS if c.flow == "burgers" else O.FLOW_NAVIER_STOKES,
                     forcing_kind=1 if c.forcing == "kolmogorov" else 0, deriv_order=c.deriv_order)


@pytest.mark.parametrize("n", [32, 64])
def test_network_forward_matches_oracle_bf16(n):
    model = make_model(1, last_scale=1.0)
    s = solver(n, 3, model)
    assert s.param_count() == 241_248 + 80
    U0 = np.stack([I.decaying_ic(n, k) for k in range(3)])
    u = torch.tensor(U0, dtype=torch.float32, device="cuda")
    coef = torch.empty((3, O.N_COEF, n, n), dtype=torch.float32, device="cuda")
    s.network_forward(u, coef)
    torch.cuda.synchronize()
    assert s.check_finite(u)  # raises on a timed-out device wait (FD_ETIMEOUT)
    g = coef.double().cpu().numpy()
    for b in range(3):
        ref = O.cnn_forward(U0[b].astype(np.float32).astype(np.float64), model.stencil)
        assert rel_l2(g[b], ref) <= 2e-2


def test_learned_step_matches_oracle():
    n, b = 64, 2
    model = make_model(3, last_scale=0.05, wl_std=1e-2)
    s = solver(n, b, model, nu=1e-3, dt=7e-3, forcing="kolmogorov")
    U0 = np.stack([I.kolmogorov_ic(n, k) for k in range(b)])
    u = torch.tensor(U0, dtype=torch.float32, device="cuda")
    out = torch.empty_like(u)
    s.step(u, out)
    torch.cuda.synchronize()
    assert s.check_finite(out)  # raises on a timed-out device wait (FD_ETIMEOUT)
    g = out.double().cpu().numpy()
    p = oracle_problem(s)
    ref = np.stack([O.learned_step(U0[k], p, model) for k in range(b)])
    plain = np.stack([O.rk4_step(U0[k], p) for k in range(b)])
    assert rel_l2(g, ref) <= 1e-4
    # the network changed the step by much more than the tolerance
    assert rel_l2(ref, plain) > 10 * rel_l2(g, ref)
    for k in range(b):
        assert np.max(np.abs(O.divergence(g[k], p.dx, p.dy))) <= 1e-5 * np.max(np.abs(g[k])) / p.dx


def test_learned_reduces_to_plain_on_gpu():
    n, b = 64, 2
    model = O.LearnedModel(W_L=np.zeros((2, 2, 5, 4)),
                           stencil=I.random_conv_stack(5, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=0.0))
    s = solver(n, b, model, nu=1e-3, dt=5e-3)
    plain = fd.Solver(fd.Config(n=n, batch=b, dtype="f32", nu=1e-3, dt=5e-3))
    U0 = np.stack([I.decaying_ic(n, k) for k in range(b)])
    u = torch.tensor(U0, dtype=torch.float32, device="cuda")
    a, c = torch.empty_like(u), torch.empty_like(u)
    s.rollout(u, a, 3)
    plain.rollout(u, c, 3)
    torch.cuda.synchronize()
    assert rel_l2(a.double().cpu().numpy(), c.double().cpu().numpy()) <= 1e-6


def test_learned_conserves_mean_momentum():
    n, b = 32, 2
    model = make_model(7, last_scale=0.05, wl_std=1e-2)
    s = solver(n, b, model, nu=1e-3, dt=1e-2)
    U0 = np.stack([I.decaying_ic(n, k) + 0.25 for k in range(b)])
    u = torch.tensor(U0, dtype=torch.float32, device="cuda")
    out = torch.empty_like(u)
    s.rollout(u, out, 10)
    torch.cuda.synchronize()
    g = out.double().cpu().numpy()
    for k in range(b):
        for c in range(2):
            assert abs(g[k, c].sum() - U0[k, c].sum()) <= 1e-5 * np.abs(U0[k, c]).sum()


def test_temporal_correction_rollout_matches_oracle():
    n, b, kc = 32, 2, 4
    model = make_model(11, last_scale=0.05, kc=kc, wl_std=1e-2)
    s = solver(n, b, model, nu=1e-3, dt=1e-2, forcing="kolmogorov")
    U0 = np.stack([I.kolmogorov_ic(n, k) for k in range(b)])
    u = torch.tensor(U0, dtype=torch.float32, device="cuda")
    out = torch.empty_like(u)
    s.rollout(u, out, 9)  # two corrections (after steps 4 and 8) and one plain step
    torch.cuda.synchronize()
    g = out.double().cpu().numpy()
    p = oracle_problem(s)
    ref = np.stack([O.rollout(U0[k], p, 9, model=model)[0] for k in range(b)])
    no_tc = O.LearnedModel(W_L=model.W_L, stencil=model.stencil)
    ref_plain = np.stack([O.rollout(U0[k], p, 9, model=no_tc)[0] for k in range(b)])
    assert rel_l2(g, ref) <= 2e-3
    assert rel_l2(ref, ref_plain) > 5 * rel_l2(g, ref)
    for k in range(b):
        assert np.max(np.abs(O.divergence(g[k], p.dx, p.dy))) <= 1e-5 * np.max(np.abs(g[k])) / p.dx


def test_graph_replay_equals_direct_launches():
    n, b, kc = 32, 2, 4
    model = make_model(13, last_scale=0.05, kc=kc, wl_std=1e-2)
    s = solver(n, b, model, nu=1e-3, dt=1e-2, forcing="kolmogorov")
    U0 = np.stack([I.kolmogorov_ic(n, k) for k in range(b)])
    u = torch.tensor(U0, dtype=torch.float32, device="cuda")
    a = torch.empty_like(u)
    s.rollout(u, a, 8)  # graph path (no snapshots)
    traj = torch.empty((8,) + tuple(u.shape), device="cuda")
    c = torch.empty_like(u)
    s.rollout(u, c, 8, traj=traj, save_every=1)  # direct launches
    torch.cuda.synchronize()
    assert torch.equal(a, c)
    assert torch.equal(traj[-1], c)
    assert s.check_finite(c)
