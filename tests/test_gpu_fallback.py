"""Plain-FV fallback of the learned solver (fd_rollout_guarded).

A learned trajectory whose chunk produces a NaN or Inf switches to the plain
FV step (the learned module with its learnable parts removed, Sec. 3.4) from
the start of that chunk on; the others stay learned. Checked without the
oracle where the answer is another call of this library (bit-identical
learned and plain rollouts), and against the oracle for the learned
trajectories.

The failing trajectory is made on the host: a temporal-correction network with
zero biases and a last layer of BF16 weights near the format's maximum turns
every non-zero history into an overflow (Inf/NaN) at the first correction,
while an all-zero trajectory stays exactly zero through it (GELU(0) = 0). A
NaN injected into one trajectory's initial state shows the other limit: that
trajectory falls back at step 0 and cannot be rescued.
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


N, KC, NU, DT = 32, 2, 1e-3, 5e-3


def _exploding_tc():
    tc = I.random_conv_stack(71, 2 * KC, O.CNN_HIDDEN, 2, last_scale=1.0)
    tc = [(W, np.zeros_like(b)) for W, b in tc]
    W, b = tc[-1]
    tc[-1] = (I.round_bf16(np.sign(W) * 3.0e38), b)
    return tc


def _solvers(batch, tc):
    st = I.random_conv_stack(72, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=0.05)
    wl = I.random_wl(73, 1e-2)
    s = fd.Solver(fd.Config(n=N, batch=batch, dtype="f32", nu=NU, dt=DT, learned=True, k_c=KC))
    s.set_params(I.pack_params(wl, st, tc))
    plain = fd.Solver(fd.Config(n=N, batch=batch, dtype="f32", nu=NU, dt=DT))
    return s, plain, O.LearnedModel(W_L=wl, stencil=st, tc=tc, k_c=KC)


def test_exploding_trajectory_falls_back_to_the_plain_solver():
    b, steps = 3, 8
    s, plain, _ = _solvers(b, _exploding_tc())
    U0 = np.stack([np.zeros((2, N, N)), I.decaying_ic(N, 74), I.decaying_ic(N, 75)]).astype(np.float32)
    u = torch.tensor(U0, device="cuda")
    out = torch.empty_like(u)
    fell = torch.empty(b, dtype=torch.int32, device="cuda")
    s.rollout_guarded(u, out, steps, fell)
    ref_l = torch.empty_like(u)
    s.rollout(u, ref_l, steps)
    ref_p = torch.empty_like(u)
    plain.rollout(u, ref_p, steps)
    torch.cuda.synchronize()
    assert fell.tolist() == [-1, 0, 0]
    # the unguarded learned rollout really blows up for the non-zero trajectories
    assert not torch.isfinite(ref_l[1:]).all()
    assert torch.equal(out[0], ref_l[0]) and float(out[0].abs().max()) == 0.0
    assert torch.equal(out[1:], ref_p[1:])
    assert bool(torch.isfinite(out).all())
    s.close()
    plain.close()


def test_guarded_equals_unguarded_when_nothing_fails_and_matches_oracle():
    b, steps = 4, 6
    tc = I.random_conv_stack(76, 2 * KC, O.CNN_HIDDEN, 2, last_scale=0.02)
    s, plain, model = _solvers(b, tc)
    U0 = np.stack([I.decaying_ic(N, 77 + k) for k in range(b)]).astype(np.float32)
    u = torch.tensor(U0, device="cuda")
    out = torch.empty_like(u)
    fell = torch.zeros(b, dtype=torch.int32, device="cuda")
    s.rollout_guarded(u, out, steps, fell, chunk=2 * KC)
    ref = torch.empty_like(u)
    s.rollout(u, ref, steps)
    torch.cuda.synchronize()
    assert fell.tolist() == [-1] * b
    assert torch.equal(out, ref)
    p = O.Problem(nx=N, ny=N, nu=NU, dt=DT)
    want = np.stack([O.rollout(U0[k].astype(np.float64), p, steps, model=model)[0] for k in range(b)])
    assert rel_l2(out.double().cpu().numpy(), want) <= 2e-3
    s.close()
    plain.close()


def test_nan_in_the_input_falls_back_at_step_zero_and_stays_non_finite():
    b, steps = 3, 4
    tc = I.random_conv_stack(78, 2 * KC, O.CNN_HIDDEN, 2, last_scale=0.02)
    s, plain, _ = _solvers(b, tc)
    U0 = np.stack([I.decaying_ic(N, 79 + k) for k in range(b)]).astype(np.float32)
    U0[1, 0, 5, 7] = np.nan
    u = torch.tensor(U0, device="cuda")
    out = torch.empty_like(u)
    fell = torch.empty(b, dtype=torch.int32, device="cuda")
    s.rollout_guarded(u, out, steps, fell)
    ref = torch.empty_like(u)
    s.rollout(u, ref, steps)
    torch.cuda.synchronize()
    assert fell.tolist() == [-1, 0, -1]
    assert not bool(torch.isfinite(out[1]).all())
    assert torch.equal(out[0], ref[0]) and torch.equal(out[2], ref[2])
    with pytest.raises(fd.FdError) as ei:
        s.rollout_guarded(u, out, steps, fell, chunk=3)  # not a multiple of k_c
    assert ei.value.status == fd.FD_EINVAL
    with pytest.raises(fd.FdError) as ei:
        plain.rollout_guarded(u, out, steps, fell)
    assert ei.value.status == fd.FD_EUNSUPPORTED
    s.close()
    plain.close()
