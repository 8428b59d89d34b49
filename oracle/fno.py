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

from .fv import gelu


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
