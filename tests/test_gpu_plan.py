"""Launch plans of plain contexts (cluster shapes, on-chip / streaming split,
the autotuner) on sm_103a, through the C ABI.

Every plan computes the same step, so each is held to the FP64 oracle at the
per-step tolerance of the plain path (relative L2 <= 1e-6 for FP32 after one
step, <= 1e-3 after 100 non-chaotic steps, <= 1e-12 for FP64) and to the
default plan at a tolerance a few FP32 roundings wide.
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
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def oracle_problem(cfg: fd.Config) -> O.Problem:
    return O.Problem(nx=cfg.n, ny=cfg.n, lx=cfg.lx, ly=cfg.ly, nu=cfg.nu, dt=cfg.dt,
                     flow=O.FLOW_BURGERS if cfg.flow == "burgers" else O.FLOW_NAVIER_STOKES,
                     forcing_kind=1 if cfg.forcing == "kolmogorov" else 0, amp=cfg.amp, kf=cfg.kf,
                     drag=cfg.drag, deriv_order=cfg.deriv_order, poisson_symbol=cfg.poisson_symbol)


def ic(cfg, b):
    if cfg.flow == "burgers":
        return np.stack([I.burgers_ic(cfg.n, s) for s in range(b)])
    return np.stack([I.decaying_ic(cfg.n, s) for s in range(b)])


def rollout(s, U0, n_steps, save_every=0):
    u = torch.tensor(U0, dtype=s.torch_dtype, device="cuda")
    out = torch.empty_like(u)
    traj = None
    if save_every:
        traj = torch.full((n_steps // save_every,) + tuple(u.shape), float("nan"), dtype=s.torch_dtype, device="cuda")
    s.rollout(u, out, n_steps, traj=traj, save_every=save_every)
    torch.cuda.synchronize()
    return out.double().cpu().numpy(), (traj.double().cpu().numpy() if traj is not None else None)


def clusters_of(n, dtype):
    return {("f32", 32): [1, 2, 4], ("f32", 64): [1, 2, 4], ("f32", 128): [2, 4, 8], ("f32", 256): [8],
            ("f64", 32): [1, 2, 4]}[(dtype, n)]


@pytest.mark.parametrize("n", [32, 64, 128, 256])
@pytest.mark.parametrize("flow", ["ns", "burgers"])
def test_cluster_shapes_match_oracle_one_step(n, flow):
    cfg = fd.Config(n=n, batch=2, dtype="f32", flow=flow, nu=1e-3 if flow != "burgers" else 0.01,
                    dt=1e-3)
    U0 = ic(cfg, 2)
    p = oracle_problem(cfg)
    ref = np.stack([O.rollout(U0[b], p, 1)[0] for b in range(2)])
    s = fd.Solver(cfg)
    outs = {}
    for cl in clusters_of(n, "f32"):
        s.set_plan(cl, 2, 0)
        assert s.plan()["cluster"] == cl
        outs[cl], _ = rollout(s, U0.astype(np.float32), 1)
        assert rel_l2(outs[cl], ref) <= 1e-6, (cl, rel_l2(outs[cl], ref))
    base = outs[clusters_of(n, "f32")[0]]
    for cl, o in outs.items():
        assert rel_l2(o, base) <= 1e-6
    s.close()


@pytest.mark.parametrize("n", [32, 64, 128])
def test_cluster_shapes_100_steps_burgers(n):
    cfg = fd.Config(n=n, batch=1, dtype="f32", flow="burgers", nu=0.01, dt=1e-3)
    U0 = ic(cfg, 1)
    ref = O.rollout(U0[0], oracle_problem(cfg), 100)[0][None]
    s = fd.Solver(cfg)
    for cl in clusters_of(n, "f32"):
        s.set_plan(cl, 1, 0)
        out, _ = rollout(s, U0.astype(np.float32), 100)
        assert rel_l2(out, ref) <= 1e-3, (cl, rel_l2(out, ref))
    s.close()


def test_fp64_cluster_shapes_burgers_32():
    cfg = fd.Config(n=32, batch=1, dtype="f64", flow="burgers", nu=0.01, dt=1e-3, deriv_order=2)
    U0 = I.burgers_ic(32, 0)[None]
    ref = O.rollout(U0[0], oracle_problem(cfg), 50)[0][None]
    s = fd.Solver(cfg)
    for cl in clusters_of(32, "f64"):
        s.set_plan(cl, 1, 0)
        out, _ = rollout(s, U0, 50)
        assert rel_l2(out, ref) <= 1e-12, (cl, rel_l2(out, ref))
    s.close()


@pytest.mark.parametrize("n_onchip", [0, 3, 5])
def test_split_plan_matches_single_plan_with_snapshots(n_onchip):
    cfg = fd.Config(n=64, batch=5, dtype="f32", nu=1e-3, dt=1e-3)
    U0 = ic(cfg, 5).astype(np.float32)
    s = fd.Solver(cfg)
    base, base_tr = rollout(s, U0, 12, save_every=4)
    s.set_plan(1 if n_onchip else 0, n_onchip, 5 - n_onchip)
    pl = s.plan()
    assert (pl["n_onchip"], pl["n_stream"]) == (n_onchip, 5 - n_onchip)
    out, tr = rollout(s, U0, 12, save_every=4)
    assert np.isfinite(tr).all()  # every snapshot slot of every trajectory written
    assert rel_l2(out, base) <= 1e-5
    for k in range(3):
        assert rel_l2(tr[k], base_tr[k]) <= 1e-5
    np.testing.assert_array_equal(tr[-1], out)
    # against the oracle: one step of the split plan
    ref = np.stack([O.rollout(U0[b].astype(np.float64), oracle_problem(cfg), 1)[0] for b in range(5)])
    one, _ = rollout(s, U0, 1)
    assert rel_l2(one, ref) <= 1e-6
    s.close()


def test_split_plan_in_place_and_in_a_batch():
    cfg = fd.Config(n=32, batch=4, dtype="f32", nu=1e-3, dt=1e-3)
    U0 = ic(cfg, 4).astype(np.float32)
    ref_s = fd.Solver(cfg)
    ref, _ = rollout(ref_s, U0, 6)
    s = fd.Solver(cfg)
    s.set_plan(1, 2, 2)
    u = torch.tensor(U0, device="cuda")
    s.rollout(u, u, 6)  # u0 and u_final alias
    torch.cuda.synchronize()
    assert rel_l2(u.double().cpu().numpy(), ref) <= 1e-5
    # the split context inside a batch graph (captured fork and join)
    other = fd.Solver(fd.Config(n=64, batch=2, dtype="f32", nu=1e-3, dt=1e-3))
    U1 = np.stack([I.decaying_ic(64, s_) for s_ in range(2)]).astype(np.float32)
    o_ref, _ = rollout(other, U1, 6)
    a0 = torch.tensor(U0, device="cuda")
    a1 = torch.empty_like(a0)
    b0 = torch.tensor(U1, device="cuda")
    b1 = torch.empty_like(b0)
    bt = fd.Batch()
    bt.add(s, a0, a1, 6)
    bt.add(other, b0, b1, 6)
    for _ in range(2):
        bt.run()
        torch.cuda.synchronize()
        assert rel_l2(a1.double().cpu().numpy(), ref) <= 1e-5
        assert rel_l2(b1.double().cpu().numpy(), o_ref) <= 1e-6
    bt.close()
    for x in (ref_s, s, other):
        x.close()


def test_autotune_keeps_the_fastest_and_stays_correct():
    cfg = fd.Config(n=64, batch=6, dtype="f32", nu=1e-3, dt=1e-3)
    U0 = ic(cfg, 6).astype(np.float32)
    s = fd.Solver(cfg)
    base, _ = rollout(s, U0, 10)
    cands = s.autotune(probe_steps=8)
    shapes = {c["cluster"] for c in cands if c["n_onchip"] > 0}
    assert shapes == set(clusters_of(64, "f32"))
    assert any(c["n_onchip"] == 0 and c["n_stream"] == 6 for c in cands)
    assert all(c["us_per_step"] > 0 for c in cands)
    best = min(cands, key=lambda c: c["us_per_step"])
    pl = s.plan()
    assert (pl["cluster"], pl["n_onchip"], pl["n_stream"]) == (best["cluster"], best["n_onchip"], best["n_stream"])
    assert pl["us_per_step"] == pytest.approx(best["us_per_step"])
    out, _ = rollout(s, U0, 10)
    assert rel_l2(out, base) <= 1e-5
    s.close()


def test_autotune_headline_batch_offers_the_remainder_split():
    # 256^2, batch 16: one more trajectory than one wave of 8-CTA clusters
    # holds on a 152-SM GB300; the split candidate puts the rest on the
    # streaming kernels
    cfg = fd.Config(n=256, batch=16, dtype="f32", nu=1e-3, dt=1.75e-3)
    s = fd.Solver(cfg)
    cands = s.autotune(probe_steps=8)
    res = cands[0]["resident"]
    assert res > 0
    if 16 % res:
        assert any(c["n_onchip"] == 16 - 16 % res and c["n_stream"] == 16 % res for c in cands)
    U0 = ic(cfg, 16).astype(np.float32)
    out, _ = rollout(s, U0, 4)
    s.set_plan(8, 16, 0)
    ref, _ = rollout(s, U0, 4)
    assert rel_l2(out, ref) <= 1e-5
    s.close()


def test_plan_errors():
    s = fd.Solver(fd.Config(n=64, batch=4, dtype="f32", nu=1e-3, dt=1e-3))
    with pytest.raises(fd.FdError) as e:
        s.set_plan(3, 4, 0)  # no 3-CTA shape
    assert e.value.status == fd.FD_EUNSUPPORTED
    with pytest.raises(fd.FdError) as e:
        s.set_plan(1, 3, 0)  # does not add up to the batch
    assert e.value.status == fd.FD_EINVAL
    s.close()
    s = fd.Solver(fd.Config(n=32, batch=1, dtype="f64", flow="burgers", nu=0.01, dt=1e-3))
    with pytest.raises(fd.FdError) as e:
        s.set_plan(1, 0, 1)  # no FP64 streaming path
    assert e.value.status == fd.FD_EUNSUPPORTED
    assert len(s.autotune(probe_steps=4)) == 3  # three FP64 cluster shapes, no streaming candidate
    s.close()
    s = fd.Solver(fd.Config(n=512, batch=1, dtype="f32", nu=1e-3, dt=1e-3))
    assert s.plan()["path"] == 2
    c = s.autotune(probe_steps=2)
    assert len(c) == 1 and c[0]["n_stream"] == 1 and c[0]["us_per_step"] > 0
    s.close()


def test_batch_recaptures_after_a_member_plan_change():
    # a plan change can replace the member's streaming sub-context; the batch
    # must not replay a graph that still launches on the old buffers
    cfg = fd.Config(n=32, batch=4, dtype="f32", nu=1e-3, dt=1e-3)
    U0 = ic(cfg, 4).astype(np.float32)
    p = oracle_problem(cfg)
    ref = np.stack([O.rollout(U0[k].astype(np.float64), p, 5)[0] for k in range(4)])
    s = fd.Solver(cfg)
    other = fd.Solver(fd.Config(n=64, batch=1, dtype="f32", nu=1e-3, dt=1e-3))
    U1 = I.decaying_ic(64, 3)[None].astype(np.float32)
    o_ref, _ = rollout(other, U1, 5)
    a0 = torch.tensor(U0, device="cuda")
    a1 = torch.empty_like(a0)
    b0 = torch.tensor(U1, device="cuda")
    b1 = torch.empty_like(b0)
    bt = fd.Batch()
    bt.add(s, a0, a1, 5)
    bt.add(other, b0, b1, 5)
    for plan in [None, (1, 2, 2), (2, 1, 3), (1, 4, 0), (4, 3, 1)]:
        if plan is not None:
            s.set_plan(*plan)
        a1.fill_(float("nan"))
        bt.run()
        torch.cuda.synchronize()
        assert rel_l2(a1.double().cpu().numpy(), ref) <= 1e-5, plan
        assert rel_l2(b1.double().cpu().numpy(), o_ref) <= 1e-6
        assert s.plan()["n_stream"] == (0 if plan is None else plan[2])
    bt.close()
    s.close()
    other.close()


def test_persistent_launch_runs_the_small_plain_trajectories_bit_identically():
    # the plain FP32 members with N <= 64 (mixed sizes, flows, forcing, derivative
    # orders) go into one persistent launch per derivative order; the 128^2
    # member stays a branch of the graph. Every output equals the member's own
    # rollout bit for bit, with the persistent launch on and off, on replay too.
    specs = [
        (fd.Config(n=16, batch=3, dtype="f32", flow="burgers", nu=1e-2, dt=4e-3), "burgers", 9),
        (fd.Config(n=32, batch=5, dtype="f32", nu=1e-3, dt=4e-3), "decaying", 7),
        (fd.Config(n=64, batch=2, dtype="f32", nu=1e-3, dt=2e-3, forcing="kolmogorov"), "kolmogorov", 5),
        (fd.Config(n=64, batch=3, dtype="f32", nu=1e-3, dt=2e-3, deriv_order=2), "decaying", 6),
        (fd.Config(n=32, batch=2, dtype="f32", flow="burgers", nu=1e-2, dt=2e-3, deriv_order=2), "burgers", 8),
        (fd.Config(n=128, batch=2, dtype="f32", nu=1e-3, dt=1e-3), "decaying", 3),
    ]
    bt = fd.Batch()
    runs = []
    for cfg, kind, steps in specs:
        s = fd.Solver(cfg)
        u0 = torch.tensor(I.ic_batch(kind, cfg.n, cfg.batch, seed0=77).astype(np.float32), device="cuda")
        ref = torch.empty_like(u0)
        s.rollout(u0, ref, steps)
        out = torch.full_like(u0, float("nan"))
        bt.add(s, u0, out, steps)
        runs.append((s, out, ref))
    torch.cuda.synchronize()
    for persistent in (True, False, True):
        bt.set_persistent(persistent)
        for _ in range(2):
            for _, out, _ in runs:
                out.fill_(float("nan"))
            bt.run()
            torch.cuda.synchronize()
            for s, out, ref in runs:
                assert torch.equal(out, ref), (s.cfg.n, s.cfg.flow, persistent)
        assert bt.persistent_count() == (3 + 5 + 2 + 3 + 2 if persistent else 0)
    bt.close()
    for s, _, _ in runs:
        s.close()
