"""Pins of the oracle's general face operator (CPU only).

The symbol tests pin the physics kernels W_P, which live on the centre row of
the 5x4 tap grid. The learned kernels K_f = W_P + proj(W_L + C_theta(u)_f)
(Sec. 3.4, the O_P / O_L convolutions) use every row, so the transverse rows,
the transposition of the tap grid for the y-axis instances and the division of
the learned derivative part by the spacing are pinned here, each against a fact
fixed outside the oracle's index arithmetic:

* geometry: a kernel with a single unit tap returns the field's value at the
  point that lies (c - 3/2) cells along the instance's axis and (r - 2) cells
  across it from the instance's output location; the point is found from the
  staggered MAC coordinates (App. B.1), not from the oracle's shifts;
* consistency: W_P plus any learned part that passed the consistency projection
  interpolates (differentiates) a linear field exactly at every output point,
  for all eight instances, on a rectangular grid with unequal spacings;
* dimensions: the learned kernels see only nodal values, so rescaling the box
  leaves interpolated face values unchanged and scales derivative face values
  by the inverse of the spacing along the instance's axis.

Planted mistakes (a row/column swap for the y-axis instances, a sign flip of the
transverse offset, a dropped 1/h on the learned derivative part) each fail one
of these checks; the tests below plant them in the oracle on the CPU.
"""

import math

import numpy as np
import pytest

import oracle as O
import oracle.fv as OF
from paper_2507_01975_gb300 import inputs as I

NX, NY = 16, 12
LX, LY = 2.0, 3.7  # unequal spacings: dx = 0.125, dy = 0.3083...


def _positions(fld, nx, ny, lx, ly):
    """Coordinates of the samples of field ``fld`` (0 = u on west faces, 1 = v on
    south faces), App. B.1."""
    (xu, yu), (xv, yv) = I.face_coords(nx, ny, lx, ly)
    return (xu, yu) if fld == 0 else (xv, yv)


def _output_positions(q, nx, ny, lx, ly):
    """Output location of instance q: cell centres or corners (App. B.2 table)."""
    fld, axis, _kind, _shift = O.INSTANCES[q]
    dx, dy = lx / nx, ly / ny
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    centre = (fld == 0 and axis == 0) or (fld == 1 and axis == 1)
    if centre:
        return (i + 0.5) * dx + 0 * j, (j + 0.5) * dy + 0 * i
    return i * dx + 0 * j, j * dy + 0 * i


def _lookup(f, fld, x, y, nx, ny, lx, ly):
    """Value of the sampled field f at physical points (x, y), which must be
    sample points of that field up to periodicity."""
    dx, dy = lx / nx, ly / ny
    x0, y0 = (0.0, 0.5 * dy) if fld == 0 else (0.5 * dx, 0.0)
    fi = (x - x0) / dx
    fj = (y - y0) / dy
    ii = np.rint(fi).astype(int)
    jj = np.rint(fj).astype(int)
    assert np.max(np.abs(fi - ii)) < 1e-9 and np.max(np.abs(fj - jj)) < 1e-9, "not a sample point"
    return f[jj % ny, ii % nx]


def single_tap_error(q, r, c):
    """Max deviation of a single-unit-tap kernel from the geometric lookup."""
    fld, axis, _kind, _shift = O.INSTANCES[q]
    dx, dy = LX / NX, LY / NY
    rng = np.random.default_rng(100 + 20 * q + 4 * r + c)
    U = rng.standard_normal((2, NY, NX))
    K = np.zeros((5, 4))
    K[r, c] = 1.0
    kernels = [np.zeros((5, 4)) for _ in range(8)]
    kernels[q] = K
    out = O.face_values(U, kernels)[q]
    xo, yo = _output_positions(q, NX, NY, LX, LY)
    along = (c - 1.5)
    across = (r - 2)
    if axis == 0:
        xt, yt = xo + along * dx, yo + across * dy
    else:
        xt, yt = xo + across * dx, yo + along * dy
    want = _lookup(U[fld], fld, xt, yt, NX, NY, LX, LY)
    return float(np.max(np.abs(out - want)))


def _random_model(seed, wl_std=0.3, last_scale=2.0):
    st = I.random_conv_stack(seed, 2, O.CNN_HIDDEN, O.N_COEF, last_scale=last_scale)
    return O.LearnedModel(W_L=I.random_wl(seed + 1, std=wl_std), stencil=st)


def linear_field_error(q, order=4, seed=3):
    """Max error of the learned instance q on a linear field, at the interior
    output points whose taps do not wrap around the periodic box."""
    p = O.Problem(nx=NX, ny=NY, lx=LX, ly=LY, deriv_order=order)
    fld, axis, kind, _shift = O.INSTANCES[q]
    coef = np.array([[0.7, 1.3, -0.4], [-0.2, 0.5, 0.9]])  # (a, b, c) of a + b x + c y per component
    U = np.zeros((2, NY, NX))
    for f in range(2):
        x, y = _positions(f, NX, NY, LX, LY)
        U[f] = coef[f, 0] + coef[f, 1] * x + coef[f, 2] * y
    model = _random_model(seed)
    kernels = O.learned_kernels(U, p, model)
    # the learned part is far from zero: the check below exercises every tap
    assert np.max(np.abs(kernels[q] - O.physics_kernel(kind, order, p.dx if axis == 0 else p.dy)[:, :, None, None])) > 1e-2
    out = O.face_values(U, kernels)[q]
    xo, yo = _output_positions(q, NX, NY, LX, LY)
    a, b, c = coef[fld]
    if kind == 0:
        want = a + b * xo + c * yo
    else:
        want = np.full_like(xo, b if axis == 0 else c)
    inner = (slice(3, NY - 3), slice(3, NX - 3))
    return float(np.max(np.abs(out[inner] - want[inner])))


def scaling_error(q, seed=5):
    """Rescale the box by (alpha, beta) with the same nodal values: interpolated
    face values must not change, derivative face values must scale by 1/alpha
    (x-axis instances) or 1/beta (y-axis instances). Returns the max relative error."""
    alpha, beta = 2.5, 0.4
    p1 = O.Problem(nx=NX, ny=NY, lx=LX, ly=LY)
    p2 = O.Problem(nx=NX, ny=NY, lx=alpha * LX, ly=beta * LY)
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((2, NY, NX))
    model = _random_model(seed)
    _fld, axis, kind, _shift = O.INSTANCES[q]
    a = O.face_values(U, O.learned_kernels(U, p1, model))[q]
    b = O.face_values(U, O.learned_kernels(U, p2, model))[q]
    s = 1.0 if kind == 0 else (alpha if axis == 0 else beta)
    return float(np.max(np.abs(b * s - a)) / np.max(np.abs(a)))


# ----------------------------------------------------------------------------
# the pins
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("q", range(8))
def test_single_tap_matches_geometry(q):
    """Every one of the 20 taps of every instance reads the sample that lies at
    its axial / transverse offset from the output location."""
    for r in range(5):
        for c in range(4):
            assert single_tap_error(q, r, c) == 0.0, (q, r, c)


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("q", range(8))
def test_learned_kernels_exact_on_linear_fields(q, order):
    """W_P + proj(W_L + C_theta) with random, far-from-zero learned parts
    interpolates / differentiates a linear field exactly (consistency,
    Sec. 3.4), on a 16 x 12 grid of a 2.0 x 3.7 box."""
    assert linear_field_error(q, order) < 1e-12


@pytest.mark.parametrize("q", range(8))
def test_learned_derivatives_scale_with_the_spacing(q):
    assert scaling_error(q) < 1e-12


# ----------------------------------------------------------------------------
# planted mistakes: each must fail a pin
# ----------------------------------------------------------------------------
def _apply_axial_swapped_y(f, K, axis, shift):
    """Mistake: the y-axis instances read the tap grid untransposed
    (row index along the axis, column index across)."""
    out = np.zeros_like(f)
    for r in range(5):
        for c in range(4):
            tap = OF.shifted(f, r - 2, c + shift) if axis == 0 else OF.shifted(f, r - 2, c + shift)
            out += K[r, c] * tap
    return out


def _apply_axial_flipped_transverse(f, K, axis, shift):
    """Mistake: the transverse offset enters with the wrong sign."""
    out = np.zeros_like(f)
    for r in range(5):
        for c in range(4):
            if axis == 0:
                tap = OF.shifted(f, 2 - r, c + shift)
            else:
                tap = OF.shifted(f, c + shift, 2 - r)
            out += K[r, c] * tap
    return out


def _learned_kernels_without_h(U, p, model):
    """Mistake: the learned derivative part is not divided by the spacing."""
    ny, nx = U.shape[1:]
    C = O.cnn_forward(U, model.stencil)
    ks = []
    for q, (_fld, axis, kind, _shift) in enumerate(O.INSTANCES):
        h = p.dx if axis == 0 else p.dy
        L = model.W_L[kind, axis][:, :, None, None] + C[q * 20:(q + 1) * 20].reshape(5, 4, ny, nx)
        ks.append(O.physics_kernel(kind, p.deriv_order, h)[:, :, None, None] + O.consistency_project(L))
    return ks


def test_planted_row_column_swap_fails(monkeypatch):
    monkeypatch.setattr(OF, "apply_axial", _apply_axial_swapped_y)
    worst = max(single_tap_error(q, r, c) for q in (2, 3, 6, 7) for r in (0, 4) for c in (0, 3))
    assert worst > 0.1
    assert max(linear_field_error(q) for q in (2, 3, 6, 7)) > 1e-2


def test_planted_transverse_sign_flip_fails(monkeypatch):
    monkeypatch.setattr(OF, "apply_axial", _apply_axial_flipped_transverse)
    for q in range(8):
        assert single_tap_error(q, 0, 1) > 0.1
        assert single_tap_error(q, 3, 2) > 0.1


def test_planted_missing_spacing_division_fails(monkeypatch):
    monkeypatch.setattr(OF, "learned_kernels", _learned_kernels_without_h)
    monkeypatch.setattr(O, "learned_kernels", _learned_kernels_without_h)
    for q in (1, 3, 5, 7):
        assert scaling_error(q) > 1e-3
