"""GPU (sm_103a) vs FP64 oracle parity of the plain FV step, through the C ABI.

Tolerances (relative L2 over the whole state):
  * FP32 one step                       <= 1e-6
  * FP32 100 steps, non-chaotic flows   <= 1e-3
  * FP64 (any number of steps here)     <= 1e-12
  * chaotic flows: corner-vorticity PCC >= 0.999 over the compared horizon
"""

import math

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


def run_gpu(cfg: fd.Config, U0: np.ndarray, n_steps: int, save_every: int = 0):
    s = fd.Solver(cfg)
    dt = s.torch_dtype
    u = torch.tensor(U0, dtype=dt, device="cuda")
    out = torch.empty_like(u)
    traj = None
    if save_every:
        traj = torch.empty((n_steps // save_every,) + tuple(u.shape), dtype=dt, device="cuda")
    s.rollout(u, out, n_steps, traj=traj, save_every=save_every)
    torch.cuda.synchronize()
    res = out.double().cpu().numpy()
    tr = traj.double().cpu().numpy() if traj is not None else None
    s.close()
    return res, tr


def oracle_problem(cfg: fd.Config) -> O.Problem:
    return O.Problem(nx=cfg.n, ny=cfg.n, lx=cfg.lx, ly=cfg.ly, nu=cfg.nu, dt=cfg.dt,
                     flow=O.FLOW_BURGERS if cfg.flow == "burgers" else O.FLOW_NAVIER_STOKES,
                     forcing_kind=1 if cfg.forcing == "kolmogorov" else 0, amp=cfg.amp, kf=cfg.kf,
                     drag=cfg.drag, deriv_order=cfg.deriv_order, poisson_symbol=cfg.poisson_symbol)


def oracle_rollout(cfg, U0, n_steps):
    p = oracle_problem(cfg)
    return np.stack([O.rollout(U0[b], p, n_steps)[0] for b in range(U0.shape[0])])


# ----------------------------------------------------------------------------
# Burgers, 32^2, FP64, 2nd-order operators, nu = 0.01, dt = 1e-3, 200 steps
# ----------------------------------------------------------------------------
def test_burgers_32_fp64_200_steps():
    cfg = fd.Config(n=32, batch=1, dtype="f64", flow="burgers", nu=0.01, dt=1e-3, deriv_order=2)
    U0 = I.burgers_ic(32, 0)[None]
    g, _ = run_gpu(cfg, U0, 200)
    o = oracle_rollout(cfg, U0, 200)
    assert rel_l2(g, o) <= 1e-12


@pytest.mark.parametrize("order", [2, 4])
def test_burgers_fp32_one_step_and_100_steps(order):
    cfg = fd.Config(n=32, batch=3, dtype="f32", flow="burgers", nu=0.01, dt=1e-3, deriv_order=order)
    U0 = np.stack([I.burgers_ic(32, s) for s in range(3)])
    g1, _ = run_gpu(cfg, U0, 1)
    assert rel_l2(g1, oracle_rollout(cfg, U0, 1)) <= 1e-6
    g100, _ = run_gpu(cfg, U0, 100)
    assert rel_l2(g100, oracle_rollout(cfg, U0, 100)) <= 1e-3


# ----------------------------------------------------------------------------
# Navier-Stokes: every built grid size, both types, ragged batches
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n", [8, 16, 32, 64, 128, 256])
def test_ns_decaying_fp32_one_step(n):
    b = 3 if n <= 128 else 2
    cfg = fd.Config(n=n, batch=b, dtype="f32", nu=1e-3, dt=1.75e-3 * 256 / n / 4)
    U0 = np.stack([I.decaying_ic(n, s) for s in range(b)])
    g, _ = run_gpu(cfg, U0, 1)
    o = oracle_rollout(cfg, U0, 1)
    assert rel_l2(g, o) <= 1e-6
    p = oracle_problem(cfg)
    for k in range(b):
        d = O.divergence(g[k], p.dx, p.dy)
        assert np.max(np.abs(d)) <= 1e-5 * np.max(np.abs(g[k])) / p.dx


@pytest.mark.parametrize("n", [8, 16, 32, 64, 128])
def test_ns_fp64_matches_oracle_to_roundoff(n):
    cfg = fd.Config(n=n, batch=2, dtype="f64", nu=1e-3, dt=2e-3, forcing="kolmogorov")
    U0 = np.stack([I.kolmogorov_ic(n, s) for s in range(2)])
    steps = 5 if n >= 128 else 20
    g, _ = run_gpu(cfg, U0, steps)
    assert rel_l2(g, oracle_rollout(cfg, U0, steps)) <= 1e-12


def test_taylor_green_fp32_100_steps():
    n = 64
    cfg = fd.Config(n=n, batch=1, dtype="f32", nu=0.01, dt=5e-3)
    U0 = I.taylor_green(n)[None]
    g, _ = run_gpu(cfg, U0, 100)
    o = oracle_rollout(cfg, U0, 100)
    assert rel_l2(g, o) <= 1e-3
    # and the closed form, to the scheme's own O(h^2) accuracy
    exact = I.taylor_green(n, 100 * 5e-3, 0.01)
    assert np.max(np.abs(g[0] - exact)) < 5e-3


def test_kolmogorov_laminar_state_is_fixed_on_gpu():
    n, nu = 64, 1e-3
    cfg = fd.Config(n=n, batch=1, dtype="f64", nu=nu, dt=0.01, forcing="kolmogorov")
    h = 2 * math.pi / n
    th = 4 * h
    dcorner = (27 * math.sin(th / 2) - math.sin(3 * th / 2)) / (12 * h)
    A = 1.0 / (nu * dcorner * 2 * math.sin(th / 2) / h + 0.1)
    (xu, yu), _ = I.face_coords(n, n)
    U = np.stack([A * np.sin(4 * yu), np.zeros((n, n))])[None]
    g, _ = run_gpu(cfg, U, 10)
    assert np.max(np.abs(g - U)) < 1e-12 * A


def test_forced_fp32_100_steps_mean_momentum():
    n = 64
    cfg = fd.Config(n=n, batch=2, dtype="f32", nu=1e-3, dt=7e-3, forcing="kolmogorov")
    U0 = np.stack([I.kolmogorov_ic(n, s) + 0.3 for s in range(2)])
    g, _ = run_gpu(cfg, U0, 100)
    z = -0.1 * cfg.dt
    R = 1 + z + z * z / 2 + z**3 / 6 + z**4 / 24
    for b in range(2):
        for c in range(2):
            expect = U0[b, c].sum() * R**100
            assert abs(g[b, c].sum() - expect) <= 1e-4 * np.abs(U0[b, c]).sum()


def test_chaotic_decaying_256_vorticity_correlation():
    n = 256
    cfg = fd.Config(n=n, batch=1, dtype="f32", nu=1e-3, dt=1.75e-3)
    U0 = I.decaying_ic(n, 0)[None]
    g, _ = run_gpu(cfg, U0, 20)
    o = oracle_rollout(cfg, U0, 20)
    p = oracle_problem(cfg)
    assert rel_l2(g, o) <= 1e-4
    assert O.pcc(O.vorticity(g[0], p.dx, p.dy), O.vorticity(o[0], p.dx, p.dy)) >= 0.999


def test_chaotic_decaying_128_200_steps_pcc():
    n = 128
    cfg = fd.Config(n=n, batch=1, dtype="f32", nu=1e-3, dt=3.5e-3)
    U0 = I.decaying_ic(n, 1)[None]
    g, _ = run_gpu(cfg, U0, 200)
    o = oracle_rollout(cfg, U0, 200)
    p = oracle_problem(cfg)
    assert O.pcc(O.vorticity(g[0], p.dx, p.dy), O.vorticity(o[0], p.dx, p.dy)) >= 0.999


# ----------------------------------------------------------------------------
# API behaviour: snapshots, aliasing, host path, zero steps, finite check
# ----------------------------------------------------------------------------
def test_snapshots_match_separate_rollouts():
    n = 32
    cfg = fd.Config(n=n, batch=2, dtype="f64", nu=1e-3, dt=5e-3)
    U0 = np.stack([I.decaying_ic(n, s) for s in range(2)])
    final, traj = run_gpu(cfg, U0, 12, save_every=4)
    assert traj.shape[0] == 3
    for s in range(3):
        ref, _ = run_gpu(cfg, U0, 4 * (s + 1))
        assert np.array_equal(traj[s], ref)
    assert np.array_equal(traj[-1], final)


def test_step_in_place_and_zero_steps():
    n = 64
    cfg = fd.Config(n=n, batch=2, dtype="f32", nu=1e-3, dt=5e-3)
    s = fd.Solver(cfg)
    U0 = np.stack([I.decaying_ic(n, k) for k in range(2)])
    u = torch.tensor(U0, dtype=torch.float32, device="cuda")
    ref = torch.empty_like(u)
    s.step(u, ref)
    s.step(u, u)  # aliasing in and out
    torch.cuda.synchronize()
    assert torch.equal(u, ref)
    z = torch.empty_like(u)
    s.rollout(ref, z, 0)
    torch.cuda.synchronize()
    assert torch.equal(z, ref)
    assert s.last_launch_count() == 1


def test_rollout_host_matches_device_rollout():
    n = 64
    cfg = fd.Config(n=n, batch=2, dtype="f32", nu=1e-3, dt=5e-3)
    U0 = np.stack([I.decaying_ic(n, k) for k in range(2)]).astype(np.float32)
    dev, _ = run_gpu(cfg, U0, 10)
    s = fd.Solver(cfg)
    hin = torch.tensor(U0).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    s.rollout_host(hin, hout, 10)
    assert np.array_equal(hout.double().numpy(), dev)


def test_check_finite_flags_nan():
    n = 16
    cfg = fd.Config(n=n, batch=1, dtype="f32")
    s = fd.Solver(cfg)
    u = torch.zeros((1, 2, n, n), device="cuda")
    assert s.check_finite(u)
    u[0, 1, 3, 5] = float("nan")
    assert not s.check_finite(u)


def test_translation_equivariance_full_size_c2():
    # full decaying-turbulence size: 256^2, batch 16, launch as in the bench
    n, b = 256, 16
    cfg = fd.Config(n=n, batch=b, dtype="f32", nu=1e-3, dt=1.75e-3)
    U0 = np.stack([I.decaying_ic(n, s) for s in range(b)])
    g, _ = run_gpu(cfg, U0, 10)
    sh, _ = run_gpu(cfg, np.roll(U0, (37, 5), axis=(2, 3)), 10)
    assert rel_l2(np.roll(g, (37, 5), axis=(2, 3)), sh) <= 1e-5
    p = oracle_problem(cfg)
    for k in (0, b - 1):
        assert np.max(np.abs(O.divergence(g[k], p.dx, p.dy))) <= 1e-5 * np.max(np.abs(g[k])) / p.dx
        for c in range(2):
            assert abs(g[k, c].sum() - U0[k, c].sum()) <= 1e-5 * np.abs(U0[k, c]).sum()
    # sampled trajectories against the oracle
    for k in (0, 7, b - 1):
        o = oracle_rollout(cfg, U0[k:k + 1], 10)
        assert rel_l2(g[k:k + 1], o) <= 1e-5
