"""Pins of the oracle's spectral Poisson solve against brute force (CPU):

* the library FFT the oracle calls (numpy's fft2 / ifft2) equals a naive
  O(N^2) DFT sum with the oracle's axis order (rows = y) on square and
  rectangular grids up to 64;
* every entry of the oracle's Poisson symbol equals the eigenvalue found by
  applying the oracle's own D2 G2 (divergence of the face gradient) to that
  single Fourier mode in real space, on a rectangular grid with unequal spacings,
  so the symbol's frequency ordering matches the FFT's;
* the solve inverts D2 G2 on mean-free right-hand sides to round-off.
"""

import numpy as np
import pytest

import oracle as O


def naive_dft2(x):
    ny, nx = x.shape
    j = np.arange(ny)[:, None]
    i = np.arange(nx)[None, :]
    out = np.zeros((ny, nx), dtype=complex)
    for ky in range(ny):
        for kx in range(nx):
            out[ky, kx] = np.sum(x * np.exp(-2j * np.pi * (kx * i / nx + ky * j / ny)))
    return out


@pytest.mark.parametrize("shape", [(8, 8), (12, 8), (16, 64), (64, 16)])
def test_fft_matches_naive_dft(shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal(shape)
    X = naive_dft2(x)
    assert np.abs(np.fft.fft2(x) - X).max() <= 1e-11 * np.abs(X).max()
    assert np.abs(np.fft.ifft2(X).real - x).max() <= 1e-12 * np.abs(x).max()


def test_poisson_symbol_is_the_eigenvalue_of_d2g2():
    p = O.Problem(nx=12, ny=8, lx=2.7, ly=1.3)
    sym = O.poisson_symbol(p)
    j = np.arange(p.ny)[:, None]
    i = np.arange(p.nx)[None, :]
    kxs = np.fft.fftfreq(p.nx) * p.nx
    kys = np.fft.fftfreq(p.ny) * p.ny
    for a, ky in enumerate(kys):
        for b, kx in enumerate(kxs):
            mode = np.exp(2j * np.pi * (kx * i / p.nx + ky * j / p.ny))
            # the operators are real-linear: apply them to both parts
            lap = O.divergence(O.gradient(mode.real, p.dx, p.dy), p.dx, p.dy) + \
                1j * O.divergence(O.gradient(mode.imag, p.dx, p.dy), p.dx, p.dy)
            lam = lap / mode
            assert np.abs(lam - lam.flat[0]).max() <= 1e-9 * (1.0 + abs(lam.flat[0]))
            assert abs(lam.flat[0] - sym[a, b]) <= 1e-9 * (1.0 + abs(sym[a, b]))


def test_poisson_solve_inverts_d2g2():
    p = O.Problem(nx=16, ny=12, lx=1.9, ly=3.1)
    rng = np.random.default_rng(5)
    rhs = rng.standard_normal((p.ny, p.nx))
    rhs -= rhs.mean()
    pc = O.poisson_solve(rhs, p)
    back = O.divergence(O.gradient(pc, p.dx, p.dy), p.dx, p.dy)
    assert np.abs(back - rhs).max() <= 1e-11 * np.abs(rhs).max()
    assert abs(pc.mean()) <= 1e-12 * np.abs(pc).max()
