"""Give-up path of the bounded waits of the tensor-core kernels.

Every mbarrier wait in the convolution and weight-gradient kernels tries at
most fd_options.spin_limit times. A context built with a limit of one try
makes those waits run out during an ordinary learned step and its reverse
mode; the kernels must then record the timeout in the context's error word
(fd_check_finite returns FD_ETIMEOUT, once), drain their own copies and MMAs,
free their tensor memory and return, leaving the device usable: a context with
the default limit, created afterwards, still matches the FP64 oracle. No wait
is left unbounded and nothing faults; only the outputs of the timed-out calls
are undefined.
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


def _model(seed):
    st = I.random_conv_stack(seed, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=0.05)
    return O.LearnedModel(W_L=I.random_wl(seed + 2, 1e-2), stencil=st)


def _solver(model, n, b, spin_limit):
    s = fd.Solver(fd.Config(n=n, batch=b, dtype="f32", learned=True, nu=1e-3, dt=5e-3, spin_limit=spin_limit))
    s.set_params(I.pack_params(model.W_L, model.stencil))
    return s


def _timed_out(s, finite_state):
    try:
        s.check_finite(finite_state)
    except fd.FdError as e:
        assert e.status == fd.FD_ETIMEOUT, e
        return True
    return False


def test_waits_give_up_report_timeout_and_leave_the_device_usable():
    n, b = 32, 2
    model = _model(61)
    U0 = np.stack([I.decaying_ic(n, 62 + k) for k in range(b)]).astype(np.float32)
    u = torch.tensor(U0, device="cuda")
    out = torch.empty_like(u)
    tiny = _solver(model, n, b, spin_limit=1)
    seen = False
    for _ in range(4):
        tiny.step(u, out)
        torch.cuda.synchronize()
        seen = _timed_out(tiny, u) or seen
    assert seen, "no wait ran out with a one-try limit"
    # reported once, then cleared
    assert tiny.check_finite(u)
    # the reverse mode's weight-gradient kernels give up the same way
    lam = torch.tensor(np.random.default_rng(63).standard_normal(U0.shape).astype(np.float32), device="cuda")
    li = torch.empty_like(u)
    dp = torch.zeros(tiny.param_count(), dtype=torch.float32, device="cuda")
    seen = False
    for _ in range(4):
        tiny.step_adjoint(u, lam, li, dp)
        torch.cuda.synchronize()
        seen = _timed_out(tiny, u) or seen
    assert seen
    tiny.close()
    # a context with the default limit on the same device is unaffected
    s = _solver(model, n, b, spin_limit=0)
    s.step(u, out)
    torch.cuda.synchronize()
    assert s.check_finite(out)
    p = O.Problem(nx=n, ny=n, nu=1e-3, dt=5e-3)
    ref = np.stack([O.learned_step(U0[k].astype(np.float64), p, model) for k in range(b)])
    assert rel_l2(out.double().cpu().numpy(), ref) <= 1e-4
    s.close()
