"""The host-side parameter packer writes the layout include/fd.h documents for
fd_set_params (CPU only): W_L, (with a scalar-learning model) W_Ls, every stencil
layer's weights and biases, then the correction network's; its length is the
documented count, and each block sits at its documented offset."""

import numpy as np
import pytest

from paper_2507_01975_gb300 import inputs as I


def stencil_count(cin0, cout5):
    shapes = [(64, cin0)] + [(64, 64)] * 4 + [(cout5, 64)]
    return sum(co * ci * 9 + co for co, ci in shapes)


@pytest.mark.parametrize("scalar,kc", [(False, 0), (False, 4), (True, 0), (True, 2)])
def test_pack_params_length_and_block_offsets(scalar, kc):
    cin0, cout5 = (3, 240) if scalar else (2, 160)
    wl = np.full((2, 2, 5, 4), 1.0)
    wls = np.full((2, 2, 5, 4), 2.0) if scalar else None
    st = [(np.full(W.shape, 3.0 + l), np.full(b.shape, -1.0 - l))
          for l, (W, b) in enumerate(I.random_conv_stack(0, cin0, 64, cout5))]
    tc = [(np.full(W.shape, 10.0 + l), np.full(b.shape, -10.0 - l))
          for l, (W, b) in enumerate(I.random_conv_stack(1, 2 * kc, 64, 2))] if kc else []
    flat = I.pack_params(wl, st, tc, W_Ls=wls)
    expect = 80 + (80 if scalar else 0) + stencil_count(cin0, cout5)
    if kc:
        expect += sum(co * ci * 9 + co for co, ci in [(64, 2 * kc)] + [(64, 64)] * 4 + [(2, 64)])
    assert flat.size == expect and flat.dtype == np.float32
    o = 0
    assert np.all(flat[o:o + 80] == 1.0)
    o += 80
    if scalar:
        assert np.all(flat[o:o + 80] == 2.0)
        o += 80
    for l, (W, b) in enumerate(st):
        assert np.all(flat[o:o + W.size] == 3.0 + l)
        o += W.size
        assert np.all(flat[o:o + b.size] == -1.0 - l)
        o += b.size
    for l, (W, b) in enumerate(tc):
        assert np.all(flat[o:o + W.size] == 10.0 + l)
        o += W.size
        assert np.all(flat[o:o + b.size] == -10.0 - l)
        o += b.size
    assert o == flat.size
