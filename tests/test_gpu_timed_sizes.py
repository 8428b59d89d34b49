"""GPU parity at the sizes and launch configurations the bench times.

Small-batch tests launch the small-batch variants of some kernels; these cases
run the variants the timed workloads use and compare them with the FP64 oracle:

* the learned 64^2 Kolmogorov step at batch 128 (8-row flux bands, four
  stages of the tensor-core network over 128 trajectories), with and without
  the frequency-domain operator, on sampled trajectories (first, middle, last);
* the learned step's reverse mode at 64^2, batch 32 on the shear flow (every
  weight-gradient CTA accumulates three or more work items in tensor memory),
  against the sum of the oracle's per-trajectory reverse modes;
* one streaming-path step on the 2048^2 fine grid, element by element.

Tolerances: learned step <= 1e-4 relative L2 (the BF16 network perturbs only
the learned part of the kernels); state cotangent <= 1e-4, W_L gradient
<= 1e-3, network weight and bias gradients <= 2e-2 (the BF16 output bound);
plain FP32 step <= 1e-6.
"""

import numpy as np
import pytest

import oracle as O
from paper_2507_01975_gb300 import fd
from paper_2507_01975_gb300 import inputs as I

from oracle_jobs import learned_step_job, run_pool, step_vjp_job

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


def problem(cfg):
    return O.Problem(nx=cfg.n, ny=cfg.n, nu=cfg.nu, dt=cfg.dt,
                     flow=O.FLOW_BURGERS if cfg.flow == "burgers" else O.FLOW_NAVIER_STOKES,
                     forcing_kind=1 if cfg.forcing == "kolmogorov" else 0, deriv_order=cfg.deriv_order)


@pytest.mark.parametrize("with_fno", [False, True])
def test_learned_step_batch128_sampled(with_fno):
    n, b = 64, 128
    st = I.random_conv_stack(31, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=0.05)
    fno = I.random_fno(33, 16, 32, 6, out_scale=0.5) if with_fno else None
    model = O.LearnedModel(W_L=I.random_wl(32, 1e-2), stencil=st, fno=None if fno is None else O.FNOParams(**fno))
    cfg = fd.Config(n=n, batch=b, dtype="f32", nu=1e-3, dt=1.75e-3, forcing="kolmogorov", learned=True,
                    fno_layers=6 if with_fno else 0, fno_modes=32 if with_fno else 0, fno_width=16 if with_fno else 0)
    s = fd.Solver(cfg)
    s.set_params(I.pack_params(model.W_L, model.stencil, None, fno))
    U0 = I.ic_batch("kolmogorov", n, b).astype(np.float32)
    u = torch.tensor(U0, device="cuda")
    out = torch.empty_like(u)
    s.step(u, out)
    torch.cuda.synchronize()
    g = out.double().cpu().numpy()
    p = problem(cfg)
    picks = [0, b // 2, b - 1]
    refs = run_pool(learned_step_job, [(U0[k].astype(np.float64), p, model) for k in picks])
    plain = O.rk4_step(U0[0].astype(np.float64), p)
    for k, ref in zip(picks, refs):
        err = rel_l2(g[k], ref)
        assert err <= 1e-4, (k, err)
    assert rel_l2(refs[0], plain) > 10 * rel_l2(g[0], refs[0])
    # the other trajectories: finite, divergence-free and momentum-conserving (forced: drag only)
    h = p.dx
    for k in range(b):
        assert np.max(np.abs(O.divergence(g[k], h, h))) <= 1e-5 * np.max(np.abs(g[k])) / h
    s.close()


def split_grads(flat, model):
    o = 80
    wl = flat[:80].reshape(2, 2, 5, 4)
    layers = []
    for W, bb in model.stencil:
        dW = flat[o:o + W.size].reshape(W.shape)
        o += W.size
        db = flat[o:o + bb.size]
        o += bb.size
        layers.append((dW, db))
    return wl, layers


def test_learned_step_adjoint_batch32_every_trajectory():
    n, b = 64, 32
    st = I.random_conv_stack(41, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=0.05)
    model = O.LearnedModel(W_L=I.random_wl(42, 1e-2), stencil=st)
    cfg = fd.Config(n=n, batch=b, dtype="f32", learned=True, nu=1e-3, dt=7e-3)
    s = fd.Solver(cfg)
    s.set_params(I.pack_params(model.W_L, model.stencil))
    rng = np.random.default_rng(43)
    U0 = np.stack([I.shear_ic(n) + 0.05 * rng.standard_normal((2, n, n)) for _ in range(b)])
    U0 = np.stack([O.project(U0[k], problem(cfg)) for k in range(b)]).astype(np.float32)
    lam = rng.standard_normal(U0.shape).astype(np.float32)
    u = torch.tensor(U0, device="cuda")
    lo = torch.tensor(lam, device="cuda")
    li = torch.empty_like(u)
    dp = torch.zeros(s.param_count(), dtype=torch.float32, device="cuda")
    s.step_adjoint(u, lo, li, dp)
    torch.cuda.synchronize()
    assert s.check_finite(li)
    p = problem(cfg)
    refs = run_pool(step_vjp_job, [(U0[k].astype(np.float64), p, lam[k].astype(np.float64), model)
                                   for k in range(b)])
    ref_lam = np.stack([r[0] for r in refs])
    assert rel_l2(li.double().cpu().numpy(), ref_lam) <= 1e-4
    wl_g, layers_g = split_grads(dp.double().cpu().numpy(), model)
    assert rel_l2(wl_g, sum(r[1][0] for r in refs)) <= 1e-3
    for l in range(6):
        dW_ref = sum(r[1][1][l][0] for r in refs)
        db_ref = sum(r[1][1][l][1] for r in refs)
        assert rel_l2(layers_g[l][0], dW_ref) <= 2e-2, (l, rel_l2(layers_g[l][0], dW_ref))
        assert rel_l2(layers_g[l][1], db_ref) <= 2e-2, (l, rel_l2(layers_g[l][1], db_ref))
    s.close()


def test_streaming_step_2048_matches_oracle():
    n = 2048
    cfg = fd.Config(n=n, batch=1, dtype="f32", nu=1e-3, dt=2.19e-4, forcing="kolmogorov")
    U0 = I.kolmogorov_ic(n, 2)[None].astype(np.float32)
    s = fd.Solver(cfg)
    u = torch.tensor(U0, device="cuda")
    out = torch.empty_like(u)
    s.rollout(u, out, 1)
    torch.cuda.synchronize()
    assert s.last_launch_count() == 17
    ref = O.rk4_step(U0[0].astype(np.float64), problem(cfg))
    assert rel_l2(out[0].double().cpu().numpy(), ref) <= 1e-6
    s.close()
