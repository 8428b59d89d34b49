"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the solver itself: it only draws initial
conditions and network weights from seeded generators, in float64 numpy, for
the flow types the paper studies (App. C.1): viscous Burgers, decaying and
Kolmogorov-forced turbulence, and a periodic double shear layer. Every field is
laid out as ``U[2, ny, nx]`` on the staggered grid (u on west faces at
``(i dx, (j+1/2) dy)``, v on south faces at ``((i+1/2) dx, j dy)``).
"""

from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


def face_coords(nx: int, ny: int, lx: float = TWO_PI, ly: float = TWO_PI):
    """Coordinates of the u-faces and v-faces: ``(xu, yu), (xv, yv)`` as [ny, nx] grids."""
    dx, dy = lx / nx, ly / ny
    i = np.arange(nx)
    j = np.arange(ny)
    xu, yu = np.meshgrid(i * dx, (j + 0.5) * dy)
    xv, yv = np.meshgrid((i + 0.5) * dx, j * dy)
    return (xu, yu), (xv, yv)


def burgers_ic(n: int, seed: int = 0, lx: float = TWO_PI, kmax: int = 4, ny: int = None,
               ly: float = None) -> np.ndarray:
    """Random smooth Burgers initial condition on n x n cells of [0, lx]^2 (or, with
    ny / ly, on n columns x ny rows of [0, lx] x [0, ly]; wavevector k has phase
    2 pi (kx x / lx + ky y / ly)).

    Each component is a sum over integer wavevectors k != 0 with |k| <= kmax of
    ``a_k cos(k.x) + b_k sin(k.x)``, one (a_k, b_k) per half-plane wavevector,
    a, b ~ N(0, 1) from ``numpy.random.default_rng(seed)`` drawn in a fixed k
    order (u first, then v). Both components are scaled by one factor so that
    max(|u|, |v|) over the grid is 1. Each component is sampled at its own faces.
    """
    rng = np.random.default_rng(seed)
    ks = []
    for kx in range(-kmax, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            if kx * kx + ky * ky == 0 or kx * kx + ky * ky > kmax * kmax:
                continue
            if kx > 0 or (kx == 0 and ky > 0):
                ks.append((kx, ky))
    ny = n if ny is None else ny
    ly = lx if ly is None else ly
    (xu, yu), (xv, yv) = face_coords(n, ny, lx, ly)
    sx, sy = TWO_PI / lx, TWO_PI / ly
    out = np.zeros((2, ny, n))
    for comp, (x, y) in enumerate(((xu, yu), (xv, yv))):
        for kx, ky in ks:
            a, b = rng.standard_normal(2)
            ph = sx * kx * x + sy * ky * y
            out[comp] += a * np.cos(ph) + b * np.sin(ph)
    return out / np.abs(out).max()


def streamfunction_field(n: int, seed: int, kpeak: float = 4.0, lx: float = TWO_PI) -> np.ndarray:
    """Divergence-free random field from a random-phase streamfunction.

    psi lives on the corners with amplitude spectrum chosen so that the energy
    spectrum is E(k) ~ k^4 exp(-2 (k / kpeak)^2) (peak at kpeak) and uniform
    random phases. u = (psi[j+1, i] - psi[j, i]) / dy and
    v = -(psi[j, i+1] - psi[j, i]) / dx, so the face-difference divergence
    vanishes identically. Scaled to unit RMS velocity, sqrt(mean(u^2 + v^2)) = 1.
    """
    rng = np.random.default_rng(seed)
    k1 = np.fft.fftfreq(n) * n * (TWO_PI / lx)
    kx, ky = np.meshgrid(k1, k1)
    kk = np.sqrt(kx * kx + ky * ky)
    with np.errstate(divide="ignore", invalid="ignore"):
        energy = kk**4 * np.exp(-2.0 * (kk / kpeak) ** 2)
        amp = np.where(kk > 0, np.sqrt(energy / np.maximum(kk, 1e-30) ** 3), 0.0)
    phase = np.exp(2j * math.pi * rng.random((n, n)))
    psi = np.real(np.fft.ifft2(amp * phase)) * n * n
    h = lx / n
    u = (np.roll(psi, -1, axis=0) - psi) / h
    v = -(np.roll(psi, -1, axis=1) - psi) / h
    U = np.stack([u, v])
    return U / math.sqrt(np.mean(u * u + v * v))


def decaying_ic(n: int, seed: int = 0) -> np.ndarray:
    """Decaying-turbulence initial condition (random field peaked at k = 4)."""
    return streamfunction_field(n, seed, kpeak=4.0)


def kolmogorov_ic(n: int, seed: int = 0) -> np.ndarray:
    """Kolmogorov-flow initial condition: the same random field family."""
    return streamfunction_field(n, seed, kpeak=4.0)


def shear_ic(n: int, delta: float = math.pi / 15, eps: float = 0.05) -> np.ndarray:
    """Periodic double shear layer on [0, 2 pi]^2.

    u = tanh((y - pi/2) / delta) for y <= pi, tanh((3 pi / 2 - y) / delta)
    otherwise; v = eps sin(x). u depends on y only and v on x only, so the
    face-difference divergence is exactly zero.
    """
    (xu, yu), (xv, yv) = face_coords(n, n)
    u = np.where(yu <= math.pi, np.tanh((yu - math.pi / 2) / delta), np.tanh((1.5 * math.pi - yu) / delta))
    v = eps * np.sin(xv)
    return np.stack([u, v])


def shear_scalar_ic(nx: int = 128, ny: int = 64, lx: float = 8.0, ly: float = 4.0, seed: int = 0,
                    eps: float = 0.05, n_blobs: int = 2, w: float = 0.5):
    """Shear-flow initial state with its passive scalar on [0, lx] x [0, ly]
    (the shear-flow case's recipe: two tanh shear layers of width w, vortices
    sin(n_blobs pi x) exp(-25 w^2 (y - y_k)^2) in v, seeded noise of amplitude eps,
    the scalar aligned with the layers). The layers sit at y_1 = ly / 4 and
    y_2 = 3 ly / 4 with opposite signs, u = tanh(5 (y - y_1) / w) - tanh(5 (y -
    y_2) / w) - 1, so the profile is periodic in y; s = (1 + u_profile) / 2 at the
    cell centres. Returns (U [2, ny, nx], S [ny, nx]); U is not projected."""
    rng = np.random.default_rng(seed)
    (xu, yu), (xv, yv) = face_coords(nx, ny, lx, ly)
    yc = (np.arange(ny)[:, None] + 0.5) * (ly / ny) * np.ones((1, nx))
    ys = (0.25 * ly, 0.75 * ly)

    def prof(y):
        return np.tanh(5 * (y - ys[0]) / w) - np.tanh(5 * (y - ys[1]) / w) - 1.0

    u = prof(yu) + eps * rng.standard_normal(yu.shape)
    v = sum(np.sin(n_blobs * np.pi * xv) * np.exp(-25 * w * w * (yv - yk) ** 2) for yk in ys)
    v = v + eps * rng.standard_normal(yv.shape)
    return np.stack([u, v]), 0.5 * (1.0 + prof(yc))


def taylor_green(n: int, t: float = 0.0, nu: float = 0.0) -> np.ndarray:
    """Taylor-Green vortex u = sin x cos y, v = -cos x sin y, times exp(-2 nu t)."""
    (xu, yu), (xv, yv) = face_coords(n, n)
    d = math.exp(-2.0 * nu * t)
    return np.stack([np.sin(xu) * np.cos(yu) * d, -np.cos(xv) * np.sin(yv) * d])


def ic_batch(kind: str, n: int, batch: int, seed0: int = 0) -> np.ndarray:
    """Batch ``[B, 2, n, n]`` of initial conditions; trajectory b uses seed seed0 + b."""
    fn = {
        "burgers": lambda s: burgers_ic(n, s),
        "decaying": lambda s: decaying_ic(n, s),
        "kolmogorov": lambda s: kolmogorov_ic(n, s),
        "shear": lambda s: shear_ic(n),
        "taylor_green": lambda s: taylor_green(n),
    }[kind]
    return np.stack([fn(seed0 + b) for b in range(batch)])


# ----------------------------------------------------------------------------
# network weights
# ----------------------------------------------------------------------------
def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even) and widen back to float64."""
    f = np.asarray(x, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def conv_stack_shapes(cin: int, hidden: int, cout: int, layers: int = 6):
    """(Cout, Cin) of each conv3x3 layer of a ``layers``-deep stack."""
    chans = [cin] + [hidden] * (layers - 1) + [cout]
    return [(chans[l + 1], chans[l]) for l in range(layers)]


def random_conv_stack(seed: int, cin: int, hidden: int, cout: int, layers: int = 6,
                      scale: float = 1.0, last_scale: float = 0.0):
    """Seeded conv3x3 stack with bf16-representable weights (float64 values).

    Hidden layers use N(0, scale / sqrt(9 Cin)) weights and N(0, 0.02) biases;
    the last layer uses ``last_scale`` times that (0 = zero-initialised, so an
    untrained model is the plain solver plus W_L).
    """
    rng = np.random.default_rng(seed)
    out = []
    shapes = conv_stack_shapes(cin, hidden, cout, layers)
    for l, (co, ci) in enumerate(shapes):
        s = scale / math.sqrt(9 * ci)
        if l == layers - 1:
            s *= last_scale
        W = round_bf16(rng.standard_normal((co, ci, 3, 3)) * s)
        b = rng.standard_normal(co) * 0.02 * (last_scale if l == layers - 1 else 1.0)
        b = np.asarray(b, dtype=np.float32).astype(np.float64)
        out.append((W, b))
    return out


def random_wl(seed: int, std: float = 1e-3) -> np.ndarray:
    """Learnable-conv kernels W_L[kind, axis, 5, 4] ~ N(0, std), float32-representable."""
    rng = np.random.default_rng(seed)
    return np.asarray(rng.standard_normal((2, 2, 5, 4)) * std, dtype=np.float32).astype(np.float64)


def random_fno(seed: int, width: int, modes: int, layers: int, scale: float = 1.0,
               out_scale: float = 0.01, cin: int = 2, cout: int = 8) -> dict:
    """Seeded parameters of a Fourier neural operator (float32-representable
    float64 arrays): P_w[width, cin], P_b[width]; per layer R[2M, M, width, width]
    (complex), W[width, width], Wb[width]; Q_w[cout, width], Q_b[cout]. Weights are
    N(0, scale / sqrt(fan-in)) (the spectral ones also divided by the number of
    kept modes), biases N(0, 0.02); Q is scaled by ``out_scale``. The defaults
    (cin 2, cout 8) are the frequency-domain operator O_F; (2 k_c, 2) is the
    FNO temporal correction."""
    rng = np.random.default_rng(seed)

    def f32(a):
        return np.asarray(a, dtype=np.float32).astype(np.float64)

    m = modes
    R = [f32(rng.standard_normal((2 * m, m, width, width)) * scale / (width * m))
         + 1j * f32(rng.standard_normal((2 * m, m, width, width)) * scale / (width * m)) for _ in range(layers)]
    return {
        "P_w": f32(rng.standard_normal((width, cin)) * scale / np.sqrt(cin)),
        "P_b": f32(rng.standard_normal(width) * 0.02),
        "R": R,
        "W": [f32(rng.standard_normal((width, width)) * scale / np.sqrt(width)) for _ in range(layers)],
        "Wb": [f32(rng.standard_normal(width) * 0.02) for _ in range(layers)],
        "Q_w": f32(rng.standard_normal((cout, width)) * out_scale / np.sqrt(width)),
        "Q_b": f32(rng.standard_normal(cout) * out_scale * 0.1),
    }


def pack_params(W_L: np.ndarray, stencil, tc=None, fno=None, W_Ls=None) -> np.ndarray:
    """Flat float32 parameter array in the layout fd_set_params documents:
    W_L[2][2][5][4], (for a model that learns the scalar) W_Ls[2][2][5][4], then
    every stencil layer's W[Cout][Cin][3][3] and b[Cout],
    then (optionally) the temporal correction: every CNN layer's weights and
    biases (``tc`` a list of (W, b)) or a Fourier neural operator (``tc`` a dict
    from random_fno), then (optionally) the frequency-domain operator. An operator
    is P_w, P_b, per layer R as [2M][M][Cin][Cout][re, im], W[Cout][Cin], b, and
    Q_w, Q_b."""
    def operator(f):
        out = [f["P_w"].ravel(), f["P_b"].ravel()]
        for R, W, b in zip(f["R"], f["W"], f["Wb"]):
            out += [np.stack([R.real, R.imag], axis=-1).ravel(), W.ravel(), b.ravel()]
        return out + [f["Q_w"].ravel(), f["Q_b"].ravel()]

    parts = [np.asarray(W_L, dtype=np.float64).ravel()]
    if W_Ls is not None:
        parts.append(np.asarray(W_Ls, dtype=np.float64).ravel())
    for W, b in stencil:
        parts += [np.asarray(W).ravel(), np.asarray(b).ravel()]
    if isinstance(tc, dict):
        parts += operator(tc)
    else:
        for W, b in (tc or []):
            parts += [np.asarray(W).ravel(), np.asarray(b).ravel()]
    if fno is not None:
        parts += operator(fno)
    return np.concatenate(parts).astype(np.float32)
