"""Kinetic-energy spectrum on sm_103a vs the FP64 oracle, through the C ABI.

The GPU transforms in FP32 and sums the shells in FP64; each shell is compared
relative to the largest shell (<= 1e-5), the total against Parseval (<= 1e-6).
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


def spectrum(s, U, kmax):
    u = torch.tensor(U.astype(np.float32), device="cuda")
    out = torch.full((U.shape[0], kmax + 1), float("nan"), dtype=torch.float64, device="cuda")
    s.energy_spectrum(u, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("n", [32, 64, 256, 2048])
def test_spectrum_matches_oracle(n):
    b = 2 if n < 2048 else 1
    s = fd.Solver(fd.Config(n=n, batch=b, dtype="f32", nu=1e-3, dt=1e-3))
    U = np.stack([I.decaying_ic(n, k) for k in range(b)]).astype(np.float32).astype(np.float64)
    kmax = n // 2 if n < 2048 else 512
    g = spectrum(s, U, kmax)
    for k in range(b):
        ref = O.energy_spectrum(U[k], kmax)
        assert np.abs(g[k] - ref).max() <= 1e-5 * ref.max(), n
    if n < 2048:
        # every shell (kmax = N covers the corners k = N / sqrt 2): Parseval
        full = spectrum(s, U, n)
        for k in range(b):
            half_mean = 0.5 * np.mean(U[k, 0] ** 2 + U[k, 1] ** 2)
            assert abs(full[k].sum() - half_mean) <= 1e-6 * half_mean
    s.close()


def test_spectrum_single_mode_and_errors():
    n = 64
    s = fd.Solver(fd.Config(n=n, batch=1, dtype="f32", nu=1e-3, dt=1e-3))
    x = np.arange(n) * (2 * np.pi / n)
    X, Y = np.meshgrid(x, x)
    U = np.stack([0.5 * np.cos(3 * X + 4 * Y), 0.25 * np.sin(5 * Y)])[None]
    g = spectrum(s, U, 8)[0]
    # |k| = 5 from both modes: 0.5^2 / 4 + 0.25^2 / 4
    assert abs(g[5] - (0.0625 + 0.015625)) <= 1e-6 * g[5]
    assert np.abs(np.delete(g, 5)).max() <= 1e-9
    out = torch.empty((1, n + 2), dtype=torch.float64, device="cuda")
    with pytest.raises(fd.FdError) as e:
        s.energy_spectrum(torch.zeros((1, 2, n, n), device="cuda"), out)  # kmax = N + 1
    assert e.value.status == fd.FD_EINVAL
    s.close()
    s = fd.Solver(fd.Config(n=32, batch=1, dtype="f64", flow="burgers", nu=0.01, dt=1e-3))
    with pytest.raises(fd.FdError) as e:
        s.energy_spectrum(torch.zeros((1, 2, 32, 32), dtype=torch.float64, device="cuda"),
                          torch.empty((1, 9), dtype=torch.float64, device="cuda"))
    assert e.value.status == fd.FD_EUNSUPPORTED
    s.close()
