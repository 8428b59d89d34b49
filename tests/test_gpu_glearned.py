"""GPU parity of the learnable module on the generic-grid path (CUDA-core
network, learned face kernels with wrap on any grid, the rectangular spectral
projection, the temporal-correction head) against the FP64 oracle.

Grids: the 25^2 Burgers preset on [0, 1]^2 (App. C.1), a ragged 40 x 24 Burgers
grid, the 128 x 64 Navier-Stokes grid on [0, 8] x [0, 4] (the shear-flow grid
of Table S2), 128^2 Kolmogorov flow, and 64^2 through path 3 beside the
tensor-core path. The network runs in FP32 with BF16-representable weights (the
oracle uses the same weights in FP64): network outputs <= 1e-4 relative L2,
one learned FP32 step <= 1e-5, a 4-step rollout with two corrections <= 1e-4.
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
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def make_model(seed, last_scale=0.05, kc=0, wl_std=1e-2, ablation=0):
    st = I.random_conv_stack(seed, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=last_scale)
    tc = I.random_conv_stack(seed + 1, 2 * kc, O.CNN_HIDDEN, 2, last_scale=0.02) if kc else []
    return O.LearnedModel(W_L=I.random_wl(seed + 2, wl_std), stencil=st, tc=tc, k_c=kc, ablation=ablation)


def problem(cfg: fd.Config) -> O.Problem:
    return O.Problem(nx=cfg.n, ny=cfg.ny or cfg.n, lx=cfg.lx, ly=cfg.ly, nu=cfg.nu, dt=cfg.dt,
                     flow=O.FLOW_BURGERS if cfg.flow == "burgers" else O.FLOW_NAVIER_STOKES,
                     forcing_kind=1 if cfg.forcing == "kolmogorov" else 0, amp=cfg.amp, kf=cfg.kf, drag=cfg.drag,
                     deriv_order=cfg.deriv_order, poisson_symbol=cfg.poisson_symbol)


def smooth_field(nx, ny, seed, modes=4):
    """A smooth periodic velocity field [2, ny, nx] of a few low modes."""
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.arange(ny) / ny, np.arange(nx) / nx, indexing="ij")
    U = np.zeros((2, ny, nx))
    for c in range(2):
        for _ in range(modes):
            kx, ky = rng.integers(-3, 4, size=2)
            U[c] += rng.standard_normal() * np.sin(2 * np.pi * (kx * x + ky * y) + rng.uniform(0, 2 * np.pi))
    return U


def initial(cfg: fd.Config, b: int, seed: int):
    nx, ny = cfg.n, cfg.ny or cfg.n
    p = problem(cfg)
    U0 = np.stack([smooth_field(nx, ny, seed + k) for k in range(b)])
    if cfg.flow != "burgers":
        U0 = np.stack([O.project(U0[k], p) for k in range(b)])
    return U0.astype(np.float32).astype(np.float64)


def solver(cfg, model):
    s = fd.Solver(cfg)
    s.set_params(I.pack_params(model.W_L, model.stencil, model.tc))
    return s


def test_network_on_a_ragged_rectangular_grid_matches_oracle():
    cfg = fd.Config(n=40, ny=24, batch=2, dtype="f32", flow="burgers", lx=1.0, ly=0.6, nu=1e-2, dt=1e-3, learned=True)
    model = make_model(3, last_scale=1.0)
    s = solver(cfg, model)
    assert s.param_count() == 241_248 + 80
    U0 = initial(cfg, 2, 10)
    u = torch.tensor(U0, dtype=torch.float32, device="cuda")
    coef = torch.empty((2, O.N_COEF, 24, 40), dtype=torch.float32, device="cuda")
    s.network_forward(u, coef)
    torch.cuda.synchronize()
    g = coef.double().cpu().numpy()
    for b in range(2):
        assert rel_l2(g[b], O.cnn_forward(U0[b], model.stencil)) <= 1e-4


@pytest.mark.parametrize("case", ["burgers25", "burgers40x24", "ns128x64", "kolmogorov128", "ablation1_25"])
def test_learned_step_matches_oracle(case):
    if case == "burgers25":
        cfg = fd.Config(n=25, batch=2, dtype="f32", flow="burgers", lx=1.0, ly=1.0, nu=1e-2, dt=1e-3, learned=True)
    elif case == "burgers40x24":
        cfg = fd.Config(n=40, ny=24, batch=2, dtype="f32", flow="burgers", lx=1.0, ly=0.6, nu=1e-2, dt=1e-3,
                        learned=True, deriv_order=2)
    elif case == "ns128x64":
        cfg = fd.Config(n=128, ny=64, batch=2, dtype="f32", lx=8.0, ly=4.0, nu=1e-3, dt=5e-3, learned=True)
    elif case == "kolmogorov128":
        cfg = fd.Config(n=128, batch=2, dtype="f32", nu=1e-3, dt=3e-3, forcing="kolmogorov", learned=True)
    else:
        cfg = fd.Config(n=25, batch=2, dtype="f32", flow="burgers", lx=1.0, ly=1.0, nu=1e-2, dt=1e-3, learned=True,
                        ablation=1)
    model = make_model(7, ablation=1 if case == "ablation1_25" else 0)
    s = solver(cfg, model)
    U0 = initial(cfg, 2, 20)
    u = torch.tensor(U0, dtype=torch.float32, device="cuda")
    out = torch.empty_like(u)
    s.step(u, out)
    torch.cuda.synchronize()
    g = out.double().cpu().numpy()
    p = problem(cfg)
    ref = np.stack([O.learned_step(U0[k], p, model) for k in range(2)])
    plain = np.stack([O.rk4_step(U0[k], p) for k in range(2)])
    assert rel_l2(g, ref) <= 1e-5
    # the learned module changed the step by much more than the tolerance
    assert rel_l2(ref, plain) > 10 * rel_l2(g, ref)
    if cfg.flow != "burgers":
        for k in range(2):
            assert np.max(np.abs(O.divergence(g[k], p.dx, p.dy))) <= 1e-5 * np.max(np.abs(g[k])) / min(p.dx, p.dy)


def test_rollout_with_temporal_correction_on_the_shear_grid_matches_oracle():
    cfg = fd.Config(n=128, ny=64, batch=2, dtype="f32", lx=8.0, ly=4.0, nu=1e-3, dt=5e-3, learned=True, k_c=2)
    model = make_model(11, kc=2)
    s = solver(cfg, model)
    U0 = initial(cfg, 2, 30)
    u = torch.tensor(U0, dtype=torch.float32, device="cuda")
    out = torch.empty_like(u)
    traj = torch.empty((4,) + tuple(u.shape), dtype=torch.float32, device="cuda")
    s.rollout(u, out, 4, traj=traj, save_every=1)
    torch.cuda.synchronize()
    p = problem(cfg)
    ref = np.stack([O.rollout(U0[k], p, 4, model=model)[0] for k in range(2)])
    no_tc = O.LearnedModel(W_L=model.W_L, stencil=model.stencil)
    ref_plain = np.stack([O.rollout(U0[k], p, 4, model=no_tc)[0] for k in range(2)])
    g = out.double().cpu().numpy()
    assert rel_l2(g, ref) <= 1e-4
    assert rel_l2(ref, ref_plain) > 10 * rel_l2(g, ref)
    assert torch.equal(traj[-1], out)
    assert s.check_finite(out)


def test_generic_path_at_64_agrees_with_the_tensor_core_path():
    base = dict(n=64, batch=2, dtype="f32", nu=1e-3, dt=7e-3, forcing="kolmogorov", learned=True)
    model = make_model(13)
    tc = solver(fd.Config(**base), model)
    gen = solver(fd.Config(**base, path=3), model)
    U0 = np.stack([I.kolmogorov_ic(64, k) for k in range(2)]).astype(np.float32).astype(np.float64)
    u = torch.tensor(U0, dtype=torch.float32, device="cuda")
    a, b = torch.empty_like(u), torch.empty_like(u)
    tc.rollout(u, a, 3)
    gen.rollout(u, b, 3)
    torch.cuda.synchronize()
    p = problem(fd.Config(**base))
    ref = np.stack([O.rollout(U0[k], p, 3, model=model)[0] for k in range(2)])
    ga, gb = a.double().cpu().numpy(), b.double().cpu().numpy()
    assert rel_l2(gb, ref) <= 1e-5  # FP32 activations
    assert rel_l2(ga, ref) <= 5e-4  # BF16 activations on the tensor cores
    assert tc.plan()["path"] != gen.plan()["path"]


def test_zero_module_reduces_to_the_plain_generic_solver():
    cfg = fd.Config(n=25, batch=2, dtype="f32", flow="burgers", lx=1.0, ly=1.0, nu=1e-2, dt=1e-3, learned=True)
    model = O.LearnedModel(W_L=np.zeros((2, 2, 5, 4)),
                           stencil=I.random_conv_stack(5, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=0.0))
    s = solver(cfg, model)
    plain = fd.Solver(fd.Config(n=25, batch=2, dtype="f32", flow="burgers", lx=1.0, ly=1.0, nu=1e-2, dt=1e-3))
    U0 = initial(cfg, 2, 40)
    u = torch.tensor(U0, dtype=torch.float32, device="cuda")
    a, c = torch.empty_like(u), torch.empty_like(u)
    s.rollout(u, a, 5)
    plain.rollout(u, c, 5)
    torch.cuda.synchronize()
    assert rel_l2(a.double().cpu().numpy(), c.double().cpu().numpy()) <= 1e-6


def test_graph_replay_equals_direct_launches():
    # a rollout without snapshots replays one captured group of k_c steps; with
    # snapshots every launch is direct: the same arithmetic in the same order
    cfg = fd.Config(n=25, batch=2, dtype="f32", flow="burgers", lx=1.0, ly=1.0, nu=1e-2, dt=1e-3, learned=True, k_c=3)
    model = make_model(17, kc=3)
    s = solver(cfg, model)
    U0 = initial(cfg, 2, 50)
    u = torch.tensor(U0, dtype=torch.float32, device="cuda")
    a, c = torch.empty_like(u), torch.empty_like(u)
    s.rollout(u, a, 8)  # two replayed groups and two direct steps
    traj = torch.empty((8,) + tuple(u.shape), dtype=torch.float32, device="cuda")
    s.rollout(u, c, 8, traj=traj, save_every=1)
    torch.cuda.synchronize()
    assert torch.equal(a, c)
    assert torch.equal(traj[-1], c)
    p = problem(cfg)
    ref = np.stack([O.rollout(U0[k], p, 8, model=model)[0] for k in range(2)])
    assert rel_l2(a.double().cpu().numpy(), ref) <= 1e-4
