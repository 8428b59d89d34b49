"""GPU parity of the reverse mode of one step (fd_step_adjoint) against the FP64
adjoint oracle (oracle/adjoint.py, itself pinned by dot-product and finite-
difference tests).

Tolerances: plain FP32 step adjoint <= 1e-5 relative L2 (FP32 arithmetic, four
stages and five projections); learned step: state cotangent <= 1e-4 (the BF16
network only touches the small learned part), W_L gradient <= 1e-3 (FP32 sums
over all faces of terms that include the BF16 network output), network weight
and bias gradients <= 2e-2 per layer (BF16 activations and cotangents, ~2^-9
relative rounding per operand, FP32 accumulation over up to 2 x 64^2 x 64 x 9
terms).
"""

import numpy as np
import pytest

import oracle as O
from oracle import adjoint as A
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


def oracle_problem(cfg: fd.Config) -> O.Problem:
    return O.Problem(nx=cfg.n, ny=cfg.n, nu=cfg.nu, dt=cfg.dt,
                     flow=O.FLOW_BURGERS if cfg.flow == "burgers" else O.FLOW_NAVIER_STOKES,
                     forcing_kind=1 if cfg.forcing == "kolmogorov" else 0, deriv_order=cfg.deriv_order)


def to_dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("flow,forcing,n", [("ns", None, 32), ("ns", "kolmogorov", 64), ("burgers", None, 32)])
def test_plain_step_adjoint_matches_oracle(flow, forcing, n):
    b = 2
    cfg = fd.Config(n=n, batch=b, dtype="f32", flow=flow, forcing=forcing, nu=2e-3, dt=5e-3)
    s = fd.Solver(cfg)
    U0 = I.ic_batch("burgers" if flow == "burgers" else "decaying", n, b, seed0=3)
    rng = np.random.default_rng(4)
    lam = rng.standard_normal(U0.shape)
    u, lo = to_dev(U0), to_dev(lam)
    li = torch.empty_like(u)
    s.step_adjoint(u, lo, li)
    torch.cuda.synchronize()
    assert s.last_launch_count() > 0
    g = li.double().cpu().numpy()
    p = oracle_problem(cfg)
    ref = np.stack([A.step_vjp(U0[k].astype(np.float32).astype(np.float64), p, lam[k])[0] for k in range(b)])
    assert rel_l2(g, ref) <= 1e-5


def test_adjoint_output_may_alias_cotangent():
    n, b = 32, 2
    cfg = fd.Config(n=n, batch=b, dtype="f32", nu=2e-3, dt=5e-3)
    s = fd.Solver(cfg)
    U0 = I.ic_batch("decaying", n, b)
    lam = np.random.default_rng(5).standard_normal(U0.shape)
    u = to_dev(U0)
    sep = torch.empty_like(u)
    s.step_adjoint(u, to_dev(lam), sep)
    inplace = to_dev(lam)
    s.step_adjoint(u, inplace, inplace)
    torch.cuda.synchronize()
    # equal up to the order of the shared-memory atomic sums of the scatter
    assert torch.allclose(sep, inplace, rtol=1e-6, atol=1e-6 * float(sep.abs().max()))


def make_model(seed, last_scale=0.05, wl_std=1e-2):
    st = I.random_conv_stack(seed, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=last_scale)
    return O.LearnedModel(W_L=I.random_wl(seed + 2, wl_std), stencil=st)


def split_grads(flat, model):
    """Split a flat fd_set_params-layout gradient into (W_L, [(dW, db)])."""
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


@pytest.mark.parametrize("n,b,forcing", [(32, 2, "kolmogorov"), (64, 1, None)])
def test_learned_step_adjoint_matches_oracle(n, b, forcing):
    model = make_model(21 + n)
    cfg = fd.Config(n=n, batch=b, dtype="f32", learned=True, nu=1e-3, dt=5e-3, forcing=forcing)
    s = fd.Solver(cfg)
    s.set_params(I.pack_params(model.W_L, model.stencil))
    U0 = np.stack([I.kolmogorov_ic(n, 30 + k) for k in range(b)])
    lam = np.random.default_rng(6).standard_normal(U0.shape)
    u, lo = to_dev(U0), to_dev(lam)
    li = torch.empty_like(u)
    dp = torch.zeros(s.param_count(), dtype=torch.float32, device="cuda")
    s.step_adjoint(u, lo, li, dp)
    torch.cuda.synchronize()
    assert s.check_finite(li)
    g = li.double().cpu().numpy()
    p = oracle_problem(cfg)
    refs = [A.step_vjp(U0[k].astype(np.float32).astype(np.float64), p, lam[k], model) for k in range(b)]
    ref_lam = np.stack([r[0] for r in refs])
    assert rel_l2(g, ref_lam) <= 1e-4
    # the learned module changes the cotangent by much more than the tolerance
    ref_plain = np.stack([A.step_vjp(U0[k].astype(np.float32).astype(np.float64), p, lam[k])[0] for k in range(b)])
    assert rel_l2(ref_plain, ref_lam) > 10 * rel_l2(g, ref_lam)
    wl_g, layers_g = split_grads(dp.double().cpu().numpy(), model)
    wl_ref = sum(r[1][0] for r in refs)
    assert rel_l2(wl_g, wl_ref) <= 1e-3
    for l in range(6):
        dW_ref = sum(r[1][1][l][0] for r in refs)
        db_ref = sum(r[1][1][l][1] for r in refs)
        assert rel_l2(layers_g[l][0], dW_ref) <= 2e-2, (l, rel_l2(layers_g[l][0], dW_ref))
        assert rel_l2(layers_g[l][1], db_ref) <= 2e-2, (l, rel_l2(layers_g[l][1], db_ref))


def test_parameter_gradients_accumulate():
    n, b = 32, 1
    model = make_model(40)
    cfg = fd.Config(n=n, batch=b, dtype="f32", learned=True, nu=1e-3, dt=5e-3)
    s = fd.Solver(cfg)
    s.set_params(I.pack_params(model.W_L, model.stencil))
    U0 = np.stack([I.decaying_ic(n, 41)])
    lam = np.random.default_rng(7).standard_normal(U0.shape)
    u, lo = to_dev(U0), to_dev(lam)
    li = torch.empty_like(u)
    once = torch.zeros(s.param_count(), dtype=torch.float32, device="cuda")
    s.step_adjoint(u, lo, li, once)
    twice = torch.zeros_like(once)
    s.step_adjoint(u, lo, li, twice)
    s.step_adjoint(u, lo, li, twice)
    torch.cuda.synchronize()
    # calls agree up to the order of the FP32 atomic sums of the face scatter,
    # which can move a BF16 rounding of the network cotangent by one unit
    a, b1 = twice.double().cpu().numpy(), once.double().cpu().numpy()
    assert rel_l2(a, 2 * b1) <= 1e-3
    again = torch.zeros_like(once)
    s.step_adjoint(u, lo, li, again)
    torch.cuda.synchronize()
    assert rel_l2(again.double().cpu().numpy(), b1) <= 1e-3


def test_adjoint_rejects_unsupported_contexts():
    u = torch.zeros((1, 2, 128, 128), device="cuda")
    s = fd.Solver(fd.Config(n=128, batch=1, dtype="f32"))
    with pytest.raises(fd.FdError) as ei:
        s.step_adjoint(u, u, u)
    assert ei.value.status == fd.FD_EUNSUPPORTED
    s2 = fd.Solver(fd.Config(n=32, batch=1, dtype="f32"))
    v = torch.zeros((1, 2, 32, 32), device="cuda")
    dp = torch.zeros(8, device="cuda")
    with pytest.raises(fd.FdError) as ei:
        s2.step_adjoint(v, v, v, dp)
    assert ei.value.status == fd.FD_EINVAL
