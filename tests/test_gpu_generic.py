"""Burgers on the generic-grid path (non-power-of-two and rectangular grids) on
sm_103a vs the FP64 oracle, through the C ABI: the paper's Burgers case
(App. C.1: [0, 1]^2, nu = 0.002, dt = 1e-3, 100^2 data grid, 25^2 model grid),
rectangular grids with ragged strips, forcing, both derivative orders, the
on-chip path on a power-of-two grid, snapshots, coarse-graining 100^2 -> 25^2.
Tolerances as for the other plain paths: FP64 <= 1e-12 and FP32 <= 1e-6 per step
(relative L2), FP32 <= 1e-4 after 100 steps."""

import numpy as np
import pytest

import oracle as O
from oracle.train import face_average
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


def gpu_rollout(cfg, U0, steps, save_every=0):
    s = fd.Solver(cfg)
    dt = torch.float64 if cfg.dtype == "f64" else torch.float32
    u = torch.tensor(U0, dtype=dt, device="cuda")
    out = torch.empty_like(u)
    traj = None
    if save_every:
        traj = torch.empty((steps // save_every,) + tuple(u.shape), dtype=dt, device="cuda")
        s.rollout(u, out, steps, traj=traj, save_every=save_every)
    else:
        s.rollout(u, out, steps)
    torch.cuda.synchronize()
    res = (out.double().cpu().numpy(), None if traj is None else traj.double().cpu().numpy(),
           s.lib.fd_last_launch_count(s.h))
    s.close()
    return res


def oracle_rollout(p, U0, steps):
    return np.stack([O.rollout(U0[b], p, steps)[0] for b in range(U0.shape[0])])


@pytest.mark.parametrize("dtype,tol1,tol100", [("f64", 1e-12, 1e-11), ("f32", 1e-6, 1e-4)])
def test_paper_burgers_case_25(dtype, tol1, tol100):
    """The paper's Burgers setting on its 25^2 model grid."""
    n, b = 25, 3
    U0 = np.stack([I.burgers_ic(n, 40 + k, lx=1.0) for k in range(b)])
    if dtype == "f32":
        U0 = U0.astype(np.float32).astype(np.float64)
    cfg = fd.Config(n=n, batch=b, dtype=dtype, flow="burgers", nu=0.002, dt=1e-3, lx=1.0, ly=1.0)
    p = O.Problem(nx=n, ny=n, lx=1.0, ly=1.0, nu=0.002, dt=1e-3, flow=O.FLOW_BURGERS)
    for steps, tol in ((1, tol1), (100, tol100)):
        g, _, launches = gpu_rollout(cfg, U0, steps)
        err = rel_l2(g, oracle_rollout(p, U0, steps))
        assert err <= tol, (steps, err)
        assert launches == 4 * steps


@pytest.mark.parametrize("nx,ny,dord,forced", [(48, 40, 4, False), (30, 17, 2, True), (7, 5, 4, False)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_rectangular_grids(nx, ny, dord, forced, dtype):
    """Rectangular grids with a ragged last strip (4 does not divide 30 or 7),
    unequal spacings, Kolmogorov forcing on ny rows, both derivative orders."""
    b, lx, ly = 2, 3.0, 2.0
    U0 = np.stack([I.burgers_ic(nx, 50 + k, lx=lx, ny=ny, ly=ly) for k in range(b)]) * 0.5
    if dtype == "f32":
        U0 = U0.astype(np.float32).astype(np.float64)
    cfg = fd.Config(n=nx, ny=ny, batch=b, dtype=dtype, flow="burgers", nu=0.01, dt=2e-3, lx=lx, ly=ly,
                    deriv_order=dord, forcing="kolmogorov" if forced else None)
    p = O.Problem(nx=nx, ny=ny, lx=lx, ly=ly, nu=0.01, dt=2e-3, flow=O.FLOW_BURGERS, deriv_order=dord,
                  forcing_kind=1 if forced else 0)
    g, _, _ = gpu_rollout(cfg, U0, 5)
    err = rel_l2(g, oracle_rollout(p, U0, 5))
    assert err <= (1e-12 if dtype == "f64" else 1e-6), err


def test_generic_path_matches_on_chip_path_and_snapshots():
    """On a power-of-two square grid path 3 computes the on-chip path's step;
    snapshots hold every save_every-th state."""
    n, b = 64, 2
    U0 = np.stack([I.burgers_ic(n, 60 + k) for k in range(b)]).astype(np.float32)
    base = dict(n=n, batch=b, dtype="f32", flow="burgers", nu=0.01, dt=2e-3)
    on_chip, _, _ = gpu_rollout(fd.Config(**base), U0, 20)
    gen, traj, _ = gpu_rollout(fd.Config(**base, path=3), U0, 20, save_every=5)
    assert rel_l2(gen, on_chip) <= 1e-6
    assert traj.shape[0] == 4 and np.array_equal(traj[-1], gen)
    mid, _, _ = gpu_rollout(fd.Config(**base, path=3), U0, 10)
    assert np.array_equal(traj[1], mid)


def test_paper_burgers_data_pipeline_100_to_25():
    """The paper's data recipe for Burgers: a 100^2 run (dt = 1e-3) coarse-grained by
    face averages to 25^2, against the oracle's run and face average."""
    n, b, steps = 100, 2, 20
    U0 = np.stack([I.burgers_ic(n, 70 + k, lx=1.0) for k in range(b)]).astype(np.float32).astype(np.float64)
    cfg = fd.Config(n=n, batch=b, dtype="f32", flow="burgers", nu=0.002, dt=1e-3, lx=1.0, ly=1.0)
    g, _, _ = gpu_rollout(cfg, U0, steps)
    p = O.Problem(nx=n, ny=n, lx=1.0, ly=1.0, nu=0.002, dt=1e-3, flow=O.FLOW_BURGERS)
    ref = oracle_rollout(p, U0, steps)
    assert rel_l2(g, ref) <= 1e-5
    fine = torch.tensor(g, dtype=torch.float32, device="cuda")
    coarse = torch.empty((b, 2, 25, 25), dtype=torch.float32, device="cuda")
    fd.downsample(fine, coarse, 4)
    torch.cuda.synchronize()
    want = np.stack([face_average(ref[k], 4) for k in range(b)])
    assert rel_l2(coarse.double().cpu().numpy(), want) <= 1e-5


def test_generic_path_refusals():
    s = fd.Solver(fd.Config(n=25, batch=1, dtype="f32", flow="burgers", nu=0.002, dt=1e-3, lx=1.0, ly=1.0))
    u = torch.zeros((1, 2, 25, 25), device="cuda")
    with pytest.raises(fd.FdError) as e:
        s.energy_spectrum(u, torch.empty((1, 5), dtype=torch.float64, device="cuda"))
    assert e.value.status == fd.FD_EUNSUPPORTED
    assert s.plan()["path"] == 4 and s.plan()["n_stream"] == 1
    s.close()


def ns_ic(nx, ny, lx, ly, seed, b):
    """Divergence-free smooth fields on a rectangular grid: random Fourier sums
    projected by the oracle."""
    p = O.Problem(nx=nx, ny=ny, lx=lx, ly=ly)
    return np.stack([O.project(I.burgers_ic(nx, seed + k, lx=lx, ny=ny, ly=ly), p) for k in range(b)])


@pytest.mark.parametrize("nx,ny,lx,ly,forced,dord,sym", [
    (128, 64, 8.0, 4.0, False, 4, 0),   # the shear-flow model grid of Table 4
    (64, 32, 6.283185307179586, 3.141592653589793, True, 2, 0),
    (32, 64, 3.0, 5.0, False, 4, 1),
])
def test_navier_stokes_rectangular(nx, ny, lx, ly, forced, dord, sym):
    """Navier-Stokes on rectangular power-of-two grids (generic-grid path with its
    own FFT projection), FP32, against the oracle; the result is divergence-free."""
    b = 2
    U0 = ns_ic(nx, ny, lx, ly, 80, b).astype(np.float32).astype(np.float64)
    kw = dict(nu=1e-3, dt=2e-3, lx=lx, ly=ly)
    cfg = fd.Config(n=nx, ny=ny, batch=b, dtype="f32", deriv_order=dord, poisson_symbol=sym,
                    forcing="kolmogorov" if forced else None, **kw)
    p = O.Problem(nx=nx, ny=ny, flow=O.FLOW_NAVIER_STOKES, deriv_order=dord, poisson_symbol=sym,
                  forcing_kind=1 if forced else 0, **kw)
    for steps, tol in ((1, 1e-6), (20, 1e-4)):
        g, _, launches = gpu_rollout(cfg, U0, steps)
        ref = oracle_rollout(p, U0, steps)
        err = rel_l2(g, ref)
        assert err <= tol, (steps, err)
        assert launches == 20 * steps
    if sym == 0:  # the discrete symbol makes the projection exact (not the continuous one)
        div = np.stack([O.divergence(g[k], p.dx, p.dy) for k in range(b)])
        grad_scale = np.abs(g).max() / min(p.dx, p.dy)
        assert np.abs(div).max() <= 1e-5 * grad_scale


@pytest.mark.parametrize("nx,ny", [(1024, 512), (2048, 1024)])
def test_navier_stokes_shear_dns_grids(nx, ny):
    """The shear-flow DNS grids (1024 x 512 in Table 4, 2048 x 1024 in Table S2):
    one step against the oracle (2048-point transforms use the opt-in shared memory)."""
    lx, ly = 8.0, 4.0
    U0 = ns_ic(nx, ny, lx, ly, 90, 1).astype(np.float32).astype(np.float64)
    cfg = fd.Config(n=nx, ny=ny, batch=1, dtype="f32", nu=1e-3, dt=3.125e-4, lx=lx, ly=ly)
    p = O.Problem(nx=nx, ny=ny, lx=lx, ly=ly, nu=1e-3, dt=3.125e-4)
    g, _, _ = gpu_rollout(cfg, U0, 1)
    assert rel_l2(g, oracle_rollout(p, U0, 1)) <= 1e-6


def test_navier_stokes_generic_path_matches_on_chip_path():
    n, b = 64, 2
    U0 = np.stack([I.decaying_ic(n, 100 + k) for k in range(b)]).astype(np.float32)
    base = dict(n=n, batch=b, dtype="f32", nu=1e-3, dt=5e-3)
    on_chip, _, _ = gpu_rollout(fd.Config(**base), U0, 20)
    gen, _, _ = gpu_rollout(fd.Config(**base, path=3), U0, 20)
    assert rel_l2(gen, on_chip) <= 1e-5


def gpu_scalar_rollout(cfg, U0, S0, steps, D):
    s = fd.Solver(cfg)
    dt = torch.float64 if cfg.dtype == "f64" else torch.float32
    u = torch.tensor(U0, dtype=dt, device="cuda")
    sc = torch.tensor(S0, dtype=dt, device="cuda")
    uo, so = torch.empty_like(u), torch.empty_like(sc)
    s.rollout_scalar(u, sc, uo, so, steps, D)
    torch.cuda.synchronize()
    res = uo.double().cpu().numpy(), so.double().cpu().numpy(), s.lib.fd_last_launch_count(s.h)
    s.close()
    return res


@pytest.mark.parametrize("D", [1e-3, 2e-3])
def test_shear_flow_with_passive_scalar(D):
    """The shear flow (App. C.1: [0, 8] x [0, 4], Re = 1000, D in {1e-3, 2e-3}) on its
    128 x 64 model grid at the coarse step 1e-2, FP32: velocity and scalar against
    the oracle after 1 and 20 steps."""
    from oracle.scalar import rollout_scalar

    nx, ny, lx, ly, b = 128, 64, 8.0, 4.0, 2
    p = O.Problem(nx=nx, ny=ny, lx=lx, ly=ly, nu=1e-3, dt=1e-2)
    ics = [I.shear_scalar_ic(nx, ny, lx, ly, seed=k) for k in range(b)]
    U0 = np.stack([O.project(u, p) for u, _ in ics]).astype(np.float32).astype(np.float64)
    S0 = np.stack([s for _, s in ics]).astype(np.float32).astype(np.float64)
    cfg = fd.Config(n=nx, ny=ny, batch=b, dtype="f32", nu=1e-3, dt=1e-2, lx=lx, ly=ly)
    for steps, tol in ((1, 1e-6), (20, 1e-4)):
        gu, gs, launches = gpu_scalar_rollout(cfg, U0, S0, steps, D)
        ref = [rollout_scalar(U0[k], S0[k], p, D, steps) for k in range(b)]
        assert rel_l2(gu, np.stack([r[0] for r in ref])) <= tol
        assert rel_l2(gs, np.stack([r[1] for r in ref])) <= tol, (steps, rel_l2(gs, np.stack([r[1] for r in ref])))
        assert launches == 20 * steps
    # the velocity is not affected by the scalar
    gu_only, _, _ = gpu_rollout(cfg, U0, 20)
    assert np.array_equal(gu_only, gu)


def test_passive_scalar_fp64_burgers_conservation():
    """FP64, Burgers velocity on a ragged 25 x 18 grid: scalar against the oracle to
    1e-12, total scalar conserved to round-off; zero velocity and zero diffusivity
    leave the scalar unchanged."""
    from oracle.scalar import rollout_scalar

    nx, ny, lx, ly, D = 25, 18, 1.0, 0.8, 2e-3
    p = O.Problem(nx=nx, ny=ny, lx=lx, ly=ly, nu=0.002, dt=1e-3, flow=O.FLOW_BURGERS)
    U0 = I.burgers_ic(nx, 3, lx=lx, ny=ny, ly=ly)[None]
    S0 = I.burgers_ic(nx, 4, lx=lx, ny=ny, ly=ly)[0][None] + 2.0
    cfg = fd.Config(n=nx, ny=ny, batch=1, dtype="f64", flow="burgers", nu=0.002, dt=1e-3, lx=lx, ly=ly)
    gu, gs, _ = gpu_scalar_rollout(cfg, U0, S0, 10, D)
    ru, rs = rollout_scalar(U0[0], S0[0], p, D, 10)
    assert rel_l2(gs[0], rs) <= 1e-12 and rel_l2(gu[0], ru) <= 1e-12
    assert abs(gs.sum() - S0.sum()) <= 1e-12 * np.abs(S0).sum()
    _, gs0, _ = gpu_scalar_rollout(cfg, np.zeros_like(U0), S0, 5, 0.0)
    assert np.array_equal(gs0, S0)


def test_passive_scalar_graph_follows_the_diffusivity():
    """One context, rollouts at D = 1e-3, 2e-3, 1e-3 (the captured step is replaced
    each time): bit-identical to fresh contexts at each diffusivity."""
    nx, ny, lx, ly = 128, 64, 8.0, 4.0
    p = O.Problem(nx=nx, ny=ny, lx=lx, ly=ly, nu=1e-3, dt=1e-2)
    u, sc = I.shear_scalar_ic(nx, ny, lx, ly, seed=3)
    U0 = O.project(u, p)[None].astype(np.float32)
    S0 = sc[None].astype(np.float32)
    cfg = fd.Config(n=nx, ny=ny, batch=1, dtype="f32", nu=1e-3, dt=1e-2, lx=lx, ly=ly)
    fresh = {D: gpu_scalar_rollout(cfg, U0, S0, 5, D)[1] for D in (1e-3, 2e-3)}
    s = fd.Solver(cfg)
    u = torch.tensor(U0, device="cuda")
    sc = torch.tensor(S0, device="cuda")
    for D in (1e-3, 2e-3, 1e-3):
        uo, so = torch.empty_like(u), torch.empty_like(sc)
        s.rollout_scalar(u, sc, uo, so, 5, D)
        torch.cuda.synchronize()
        assert np.array_equal(so.double().cpu().numpy(), fresh[D])
    assert not np.array_equal(fresh[1e-3], fresh[2e-3])
    s.close()


def test_passive_scalar_refusals():
    s = fd.Solver(fd.Config(n=64, batch=1, dtype="f32", nu=1e-3, dt=1e-3))  # on-chip path
    u = torch.zeros((1, 2, 64, 64), device="cuda")
    sc = torch.zeros((1, 64, 64), device="cuda")
    with pytest.raises(fd.FdError) as e:
        s.rollout_scalar(u, sc, torch.empty_like(u), torch.empty_like(sc), 1, 1e-3)
    assert e.value.status == fd.FD_EUNSUPPORTED
    s.close()
    s = fd.Solver(fd.Config(n=64, ny=32, batch=1, dtype="f32", nu=1e-3, dt=1e-3))
    u = torch.zeros((1, 2, 32, 64), device="cuda")
    sc = torch.zeros((1, 32, 64), device="cuda")
    with pytest.raises(fd.FdError) as e:
        s.rollout_scalar(u, sc, torch.empty_like(u), torch.empty_like(sc), 1, -1.0)
    assert e.value.status == fd.FD_EINVAL
    s.close()
