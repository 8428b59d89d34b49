"""Frequency-domain operator O_F of the flux block, FP64 reference.

Test infrastructure only: imported by tests/, smoke() and bench.py's CPU arms,
never by the CUDA path.

The flux block's integrated operator is O = O_P + O_L + O_F (Sec. 3.4, the
flux-block equation). O_F is a Fourier neural operator (Sec. 3.4, "Frequency
Domain Operator"; the FNO appendix; hyperparameters in Table S3: forced flow 6
layers, 32 modes, width 16, GELU): a pointwise lift P of the velocity, L
Fourier layers

    v <- sigma(W_l v + b_l + F^-1(R_l . F(v)))   (sigma omitted after the last)

whose spectral part multiplies each kept Fourier mode's channel vector by a
complex matrix, and a pointwise projection Q. Readings (the paper does not fix
them): the input is the two velocity components on their own grids; F is the
real 2D DFT (numpy rfft2 / irfft2, the FNO convention), keeping kx < M and the
rows ky in [0, M) and [N - M, N), each row block with its own weights (M <= N/2);
Q maps to one channel per face-operator instance (the eight of the flux block,
in the order of fv.INSTANCES), whose value at index (j, i) is added to that
instance's face value at (j, i).

The same operator with 2 k_c input channels (the last k_c states, component c
of state s as channel 2 s + c) and 2 output channels is the paper's temporal
correction (Sec. 3.5; Table S3: 4 layers, 32 modes, width 8).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .fv import gelu, gelu_grad


@dataclass
class FNOParams:
    """``P_w[width, c_in]``, ``P_b[width]``; per layer ``R[l][2M, M, width_in, width_out]``
    (complex; rows 0 .. M-1 for ky = 0 .. M-1, rows M .. 2M-1 for ky = N-M .. N-1),
    ``W[l][width_out, width_in]``, ``Wb[l][width]``; ``Q_w[c_out, width]``, ``Q_b[c_out]``
    (c_in = 2, c_out = 8 for O_F; c_in = 2 k_c, c_out = 2 for the temporal correction)."""

    P_w: np.ndarray
    P_b: np.ndarray
    R: list
    W: list
    Wb: list
    Q_w: np.ndarray
    Q_b: np.ndarray

    @property
    def layers(self) -> int:
        return len(self.R)

    @property
    def modes(self) -> int:
        return self.R[0].shape[1]

    @property
    def width(self) -> int:
        return self.P_w.shape[0]


def pointwise(w: np.ndarray, b: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Channel map out[o, y, x] = sum_i w[o, i] v[i, y, x] + b[o] (1x1 convolution)."""
    return np.einsum("oi,iyx->oyx", w, v) + b[:, None, None]


def spectral_conv(v: np.ndarray, R: np.ndarray) -> np.ndarray:
    """F^-1(R . F(v)) for v[C, N, N]: real 2D DFT, per kept mode a complex channel
    matrix, zero elsewhere, inverse real 2D DFT (numpy's rfft2 / irfft2)."""
    n = v.shape[1]
    m = R.shape[1]
    assert 2 * m <= n
    vh = np.fft.rfft2(v)
    out = np.zeros((R.shape[3], n, n // 2 + 1), dtype=np.complex128)
    out[:, :m, :m] = np.einsum("iyx,yxio->oyx", vh[:, :m, :m], R[:m])
    out[:, n - m:, :m] = np.einsum("iyx,yxio->oyx", vh[:, n - m:, :m], R[m:])
    return np.fft.irfft2(out, s=(n, n))


def fno_forward(U: np.ndarray, prm: FNOParams) -> np.ndarray:
    """The operator on U[c_in, N, N]: for O_F the eight face-value corrections
    [8, N, N] of the state U[2, N, N]; for the temporal correction the correction
    [2, N, N] of the stacked history U[2 k_c, N, N]."""
    v = pointwise(prm.P_w, prm.P_b, U)
    for l in range(prm.layers):
        v = spectral_conv(v, prm.R[l]) + pointwise(prm.W[l], prm.Wb[l], v)
        if l < prm.layers - 1:
            v = gelu(v)
    return pointwise(prm.Q_w, prm.Q_b, v)


# ----------------------------------------------------------------------------
# reverse mode (vector-Jacobian products), for training the operators
# ----------------------------------------------------------------------------
def _kept(a: np.ndarray, m: int) -> np.ndarray:
    """The kept modes [C, 2M, M] of a spectrum [C, N, >= M] (rows 0 .. M-1 and N-M .. N-1)."""
    n = a.shape[1]
    return np.concatenate([a[:, :m, :m], a[:, n - m:, :m]], axis=1)


def spectral_conv_vjp(v: np.ndarray, R: np.ndarray, ybar: np.ndarray):
    """Adjoint of y = spectral_conv(v, R) for a cotangent ybar [C_out, N, N]:
    (vbar [C_in, N, N], Rbar [2M, M, C_in, C_out]).

    y is real-linear in v: y(x) = N^-2 sum_k c_k Re(Z_k e^{2 pi i k.x / N}) with Z
    the mixed kept modes, c = 1 for kx = 0 and 2 otherwise (irfft2 counts each
    kept half-plane mode with its mirror and drops the imaginary part of the kx = 0
    column after the inverse along y). Hence Zbar = c N^-2 fft2(ybar) on the kept
    modes, Sbar = conj(R)^T Zbar per mode, vbar = Re(sum_k Sbar_k e^{2 pi i k.x / N})
    (the adjoint of the kept part of rfft2), and for the complex weights, with the
    gradient written d/dRe + i d/dIm, Rbar = Zbar conj(S)."""
    n = v.shape[1]
    m = R.shape[1]
    S = _kept(np.fft.rfft2(v), m)
    c = np.where(np.arange(m) == 0, 1.0, 2.0)
    Zbar = _kept(np.fft.fft2(ybar), m) * c[None, None, :] / n**2
    Rbar = np.einsum("oyx,iyx->yxio", Zbar, np.conj(S))
    Sbar = np.einsum("yxio,oyx->iyx", np.conj(R), Zbar)
    E = np.zeros((v.shape[0], n, n), dtype=np.complex128)
    E[:, :m, :m] = Sbar[:, :m]
    E[:, n - m:, :m] = Sbar[:, m:]
    return n**2 * np.real(np.fft.ifft2(E)), Rbar


def fno_vjp(U: np.ndarray, prm: FNOParams, gbar: np.ndarray):
    """Reverse mode of fno_forward: for the cotangent gbar of the output [c_out, N, N],
    (Ubar [c_in, N, N], FNOParams of gradients; the R entries complex, d/dRe + i d/dIm).
    Every rule is the transpose of a forward line: pointwise maps, GELU (its
    derivative at the saved pre-activation), spectral_conv_vjp."""
    v = [pointwise(prm.P_w, prm.P_b, U)]
    pre = []
    for l in range(prm.layers):
        a = spectral_conv(v[-1], prm.R[l]) + pointwise(prm.W[l], prm.Wb[l], v[-1])
        pre.append(a)
        v.append(gelu(a) if l < prm.layers - 1 else a)
    Q_w = np.einsum("qyx,iyx->qi", gbar, v[-1])
    Q_b = gbar.sum(axis=(1, 2))
    vbar = np.einsum("qi,qyx->iyx", prm.Q_w, gbar)
    R, W, Wb = [None] * prm.layers, [None] * prm.layers, [None] * prm.layers
    for l in reversed(range(prm.layers)):
        abar = vbar * gelu_grad(pre[l]) if l < prm.layers - 1 else vbar
        Wb[l] = abar.sum(axis=(1, 2))
        W[l] = np.einsum("oyx,iyx->oi", abar, v[l])
        vs, R[l] = spectral_conv_vjp(v[l], prm.R[l], abar)
        vbar = np.einsum("oi,oyx->iyx", prm.W[l], abar) + vs
    P_w = np.einsum("oyx,iyx->oi", vbar, U)
    P_b = vbar.sum(axis=(1, 2))
    Ubar = np.einsum("oi,oyx->iyx", prm.P_w, vbar)
    return Ubar, FNOParams(P_w=P_w, P_b=P_b, R=R, W=W, Wb=Wb, Q_w=Q_w, Q_b=Q_b)
