"""FP64 oracle of the coarse-grid FV time step (plain and learned).

TEST INFRASTRUCTURE ONLY -- see the package docstring. Plain numpy float64,
written for readability, not speed: every stencil is a sum of ``np.roll``-shifted
copies, every network layer a loop over its nine taps.

Grid and layout (paper App. B.1, staggered MAC grid with periodic padding):

* a state is ``U[2, ny, nx]``: ``U[0] = u`` and ``U[1] = v``;
* ``u[j, i]`` sits on the west face of cell (i, j), at ``(i dx, (j + 1/2) dy)``;
* ``v[j, i]`` sits on the south face, at ``((i + 1/2) dx, j dy)``;
* pressure and the cell divergence sit at centres ``((i + 1/2) dx, (j + 1/2) dy)``;
* vorticity sits at corners ``(i dx, j dy)``.

Face operators (Sec. 3.4, Eqs. for O_P and O_L; App. B.2 physics kernels). A
kernel is a 5x4 array ``K[r, c]``: ``r = 0..4`` is the transverse offset
``r - 2`` and ``c = 0..3`` the axial tap at offset ``c - 3/2`` (in cells) from
the output location. Applied along x it computes
``out[j, i] = sum_rc K[r, c] f[j + r - 2, i + c + shift]``; along y the kernel is
transposed, ``out[j, i] = sum_rc K[r, c] f[j + c + shift, i + r - 2]``.

The eight operator instances (field, axis, kind, output location, shift)::

    0 u x interp  -> centre  -1      4 v x interp  -> corner  -2
    1 u x deriv   -> centre  -1      5 v x deriv   -> corner  -2
    2 u y interp  -> corner  -2      6 v y interp  -> centre  -1
    3 u y deriv   -> corner  -2      7 v y deriv   -> centre  -1
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

# ----------------------------------------------------------------------------
# instance table
# ----------------------------------------------------------------------------
#: (field index, axis 0=x 1=y, kind 0=interp 1=deriv, shift)
INSTANCES = [
    (0, 0, 0, -1),
    (0, 0, 1, -1),
    (0, 1, 0, -2),
    (0, 1, 1, -2),
    (1, 0, 0, -2),
    (1, 0, 1, -2),
    (1, 1, 0, -1),
    (1, 1, 1, -1),
]

FLOW_BURGERS = 0
FLOW_NAVIER_STOKES = 1

#: axial tap offsets (cells) and transverse offsets (cells) of the 5x4 grid
AXIAL = np.array([-1.5, -0.5, 0.5, 1.5])
TRANSVERSE = np.array([-2.0, -1.0, 0.0, 1.0, 2.0])


@dataclass
class Problem:
    """One coarse-grid problem: the PDE parameters mu of Eq. 1 and the box.

    ``flow``: FLOW_BURGERS (S = 0, no pressure) or FLOW_NAVIER_STOKES.
    ``forcing_kind``: 0 none, 1 Kolmogorov ``f = [amp sin(kf y) - drag u, -drag v]``
    (App. C.1, forced flow).
    ``deriv_order``: 4 (the paper's physics kernel, App. B.2) or 2.
    ``poisson_symbol``: 0 = symbol of the discrete operators D2 G2 (exact
    projection), 1 = the continuous symbol -(eta_x^2 + eta_y^2) of App. B.4.
    """

    nx: int
    ny: int
    lx: float = 2 * math.pi
    ly: float = 2 * math.pi
    nu: float = 1e-3
    dt: float = 1e-3
    flow: int = FLOW_NAVIER_STOKES
    forcing_kind: int = 0
    amp: float = 1.0
    kf: int = 4
    drag: float = 0.1
    deriv_order: int = 4
    poisson_symbol: int = 0

    @property
    def dx(self) -> float:
        return self.lx / self.nx

    @property
    def dy(self) -> float:
        return self.ly / self.ny


# ----------------------------------------------------------------------------
# physics kernels (App. B.2)
# ----------------------------------------------------------------------------
def physics_kernel(kind: int, order: int, h: float) -> np.ndarray:
    """Fixed 5x4 kernel W_P of App. B.2 along an axis of spacing ``h``.

    Derivative, 4th order: the printed row [1, -27, 27, -1] / (24 h).
    Derivative, 2nd order: [0, -1, 1, 0] / h.
    Interpolation: [0, 1/2, 1/2, 0], the linear interpolation the paper names.
    (The printed interpolation row [0, -1, 1, 0] / (2h) is a difference, not an
    interpolation; this is the reading listed in the design notes.)
    Only the centre row (transverse offset 0) is non-zero.
    """
    k = np.zeros((5, 4))
    if kind == 0:
        k[2] = [0.0, 0.5, 0.5, 0.0]
    elif order == 4:
        k[2] = np.array([1.0, -27.0, 27.0, -1.0]) / (24.0 * h)
    elif order == 2:
        k[2] = np.array([0.0, -1.0, 1.0, 0.0]) / h
    else:
        raise ValueError("deriv_order must be 2 or 4")
    return k


def shifted(f: np.ndarray, dj: int, di: int) -> np.ndarray:
    """``g[j, i] = f[j + dj, i + di]`` with periodic wrap (App. B.1 padding)."""
    return np.roll(f, (-dj, -di), axis=(0, 1))


def apply_axial(f: np.ndarray, K: np.ndarray, axis: int, shift: int) -> np.ndarray:
    """Apply a 5x4 kernel (global ``[5,4]`` or per-face ``[5,4,ny,nx]``).

    This is the convolution ``W * u`` of the O_P / O_L equations (Sec. 3.4),
    with the kernel transposed for the y direction.
    """
    out = np.zeros_like(f)
    for r in range(5):
        for c in range(4):
            if axis == 0:
                tap = shifted(f, r - 2, c + shift)
            else:
                tap = shifted(f, c + shift, r - 2)
            out += K[r, c] * tap
    return out


def plain_kernels(p: Problem) -> list:
    """The eight instance kernels of the plain solver (O_P only)."""
    ks = []
    for (_fld, axis, kind, _shift) in INSTANCES:
        h = p.dx if axis == 0 else p.dy
        ks.append(physics_kernel(kind, p.deriv_order, h))
    return ks


def face_values(U: np.ndarray, kernels: Sequence[np.ndarray]) -> list:
    """The eight interpolated / differentiated face quantities (flux block)."""
    out = []
    for q, (fld, axis, _kind, shift) in enumerate(INSTANCES):
        out.append(apply_axial(U[fld], kernels[q], axis, shift))
    return out


# ----------------------------------------------------------------------------
# tendency: flux assembly and divergence (Eq. 4; App. B.2)
# ----------------------------------------------------------------------------
def forcing(U: np.ndarray, p: Problem) -> np.ndarray:
    """Source term S of Eq. 1 at the faces (App. C.1, forced flow).

    f_x = amp sin(kf y) - drag u at u-faces (y = (j + 1/2) dy), f_y = -drag v.
    Zero when ``forcing_kind == 0``.
    """
    f = np.zeros_like(U)
    if p.forcing_kind == 1:
        y_u = (np.arange(p.ny) + 0.5) * p.dy
        f[0] = p.amp * np.sin(p.kf * y_u)[:, None] - p.drag * U[0]
        f[1] = -p.drag * U[1]
    return f


def tendency(U: np.ndarray, p: Problem, kernels: Optional[Sequence] = None,
             extra: Optional[np.ndarray] = None) -> np.ndarray:
    """Right-hand side H(u) of the momentum equation without the pressure flux.

    Finite-volume form of Eq. 4 (App. B.2): for the u control volume centred on
    the u-face (i, j+1/2), the east/west faces are the cell centres (i, j) and
    (i-1, j) and the north/south faces the corners (i, j+1) and (i, j):

      T_u = -[(Uc Uc)_e - (Uc Uc)_w]/dx - [(Vk Uk)_n - (Vk Uk)_s]/dy
            + nu [(Gxc_e - Gxc_w)/dx + (Gyu_n - Gyu_s)/dy] + f_x

    and symmetrically for v. Both factors of each advective flux are
    interpolated face velocities (advection term), the diffusive fluxes are
    the face derivatives (dissipation term).

    Burgers (Eq. 1 with F = u^2/2 - nu grad u; App. C.1 advective form
    u_t = nu lap u - u . grad u): the conservative flux divergence above minus
    u times the cell divergence (Gxc + Gyc) averaged to the face, which equals
    u . grad u for the continuum operators.

    ``extra[q]`` (optional, [8, ny, nx]) is added to instance q's face values:
    the frequency-domain operator O_F of the integrated operator (Sec. 3.4).
    """
    if kernels is None:
        kernels = plain_kernels(p)
    dx, dy = p.dx, p.dy
    fv = face_values(U, kernels)
    if extra is not None:
        fv = [f + extra[q] for q, f in enumerate(fv)]
    Uc, Gxc, Uk, Gyu, Vk, Gxv, Vc, Gyc = fv
    P = Uk * Vk  # (u v) at corners, shared by both momentum equations
    Tu = (
        -(Uc**2 - shifted(Uc**2, 0, -1)) / dx
        - (shifted(P, 1, 0) - P) / dy
        + p.nu * ((Gxc - shifted(Gxc, 0, -1)) / dx + (shifted(Gyu, 1, 0) - Gyu) / dy)
    )
    Tv = (
        -(shifted(P, 0, 1) - P) / dx
        - (Vc**2 - shifted(Vc**2, -1, 0)) / dy
        + p.nu * ((shifted(Gxv, 0, 1) - Gxv) / dx + (Gyc - shifted(Gyc, -1, 0)) / dy)
    )
    if p.flow == FLOW_BURGERS:
        divc = Gxc + Gyc
        Tu = Tu + U[0] * 0.5 * (shifted(divc, 0, -1) + divc)
        Tv = Tv + U[1] * 0.5 * (shifted(divc, -1, 0) + divc)
    T = np.stack([Tu, Tv])
    return T + forcing(U, p)


# ----------------------------------------------------------------------------
# projection (Sec. 3.6; App. B.3, B.4)
# ----------------------------------------------------------------------------
def divergence(U: np.ndarray, dx: float, dy: float) -> np.ndarray:
    """Cell-centred divergence D2 of a MAC field (difference of adjacent faces)."""
    return (shifted(U[0], 0, 1) - U[0]) / dx + (shifted(U[1], 1, 0) - U[1]) / dy


def gradient(p_c: np.ndarray, dx: float, dy: float) -> np.ndarray:
    """Face gradient G2 of a centred scalar: differences of adjacent pressures (App. B.1)."""
    gu = (p_c - shifted(p_c, 0, -1)) / dx
    gv = (p_c - shifted(p_c, -1, 0)) / dy
    return np.stack([gu, gv])


def poisson_symbol(p: Problem) -> np.ndarray:
    """Fourier symbol of the Laplacian used by the spectral Poisson solve (App. B.4).

    ``poisson_symbol == 0``: symbol of D2 G2,
    -(4/dx^2) sin^2(pi kx / nx) - (4/dy^2) sin^2(pi ky / ny).
    ``poisson_symbol == 1``: the continuous -(eta_x^2 + eta_y^2) printed in App. B.4.
    Shape ``[ny, nx]`` in numpy's fft2 ordering.
    """
    kx = np.fft.fftfreq(p.nx) * p.nx
    ky = np.fft.fftfreq(p.ny) * p.ny
    if p.poisson_symbol == 0:
        sx = -(4.0 / p.dx**2) * np.sin(np.pi * kx / p.nx) ** 2
        sy = -(4.0 / p.dy**2) * np.sin(np.pi * ky / p.ny) ** 2
    else:
        sx = -((2 * np.pi / p.lx) * kx) ** 2
        sy = -((2 * np.pi / p.ly) * ky) ** 2
    return sy[:, None] + sx[None, :]


def poisson_solve(rhs: np.ndarray, p: Problem) -> np.ndarray:
    """Solve lap p = rhs spectrally (App. B.4), p_hat = rhs_hat / symbol.

    The zero mode is excluded (the paper assumes eta != 0) and set to zero,
    i.e. the mean pressure is zero (App. C.1, shear flow: integral of p = 0).
    """
    sym = poisson_symbol(p)
    rh = np.fft.fft2(rhs)
    ph = np.zeros_like(rh)
    nz = sym != 0.0
    ph[nz] = rh[nz] / sym[nz]
    return np.real(np.fft.ifft2(ph))


def project(U: np.ndarray, p: Problem) -> np.ndarray:
    """Projection step of App. B.3: w = w* - grad p with lap p = div w*.

    The dt of the printed corrector cancels between the Poisson right-hand
    side (div w* / dt) and the correction (dt grad p), so it is omitted.
    """
    d = divergence(U, p.dx, p.dy)
    pc = poisson_solve(d, p)
    return U - gradient(pc, p.dx, p.dy)


# ----------------------------------------------------------------------------
# RK4 step and rollout (App. B.5; Sec. 3.2)
# ----------------------------------------------------------------------------
def rk4_step(U: np.ndarray, p: Problem, kernels_fn=None) -> np.ndarray:
    """One FV-module update u_k -> u_{k+1} (Sec. 3.2, App. B.5).

    r1 = H(u), r2 = H(u + dt/2 r1), r3 = H(u + dt/2 r2), r4 = H(u + dt r3),
    u' = u + dt/6 (r1 + 2 r2 + 2 r3 + r4). For Navier-Stokes every sub-step's
    intermediate field and the final combination are projected (Sec. 3.2:
    the projection completes each RK4 sub-step). ``kernels_fn(W)`` returns the
    eight face kernels for stage state W (plain kernels when None), or a pair
    (kernels, extra face values) when the operator has a frequency-domain part.
    """
    ns = p.flow == FLOW_NAVIER_STOKES
    P = (lambda W: project(W, p)) if ns else (lambda W: W)
    K = (lambda W: None) if kernels_fn is None else kernels_fn

    def H(W):
        k = K(W)
        return tendency(W, p, *k) if isinstance(k, tuple) else tendency(W, p, k)

    r1 = H(U)
    w = P(U + 0.5 * p.dt * r1)
    r2 = H(w)
    w = P(U + 0.5 * p.dt * r2)
    r3 = H(w)
    w = P(U + p.dt * r3)
    r4 = H(w)
    return P(U + (p.dt / 6.0) * (r1 + 2.0 * r2 + 2.0 * r3 + r4))


def rollout(U0: np.ndarray, p: Problem, n_steps: int, save_every: int = 0,
            model: "Optional[LearnedModel]" = None):
    """Autoregressive rollout of Eq. for u_k (Sec. 3.2).

    Plain when ``model`` is None; otherwise the learned step, with the temporal
    correction applied at k = M k_c when the model has one. Returns
    ``(u_final, snapshots)`` where snapshots holds u_0 and every
    ``save_every``-th state (empty when save_every == 0).
    """
    U = np.array(U0, dtype=np.float64)
    snaps = [U.copy()] if save_every else []
    hist = [U.copy()]
    for k in range(1, n_steps + 1):
        if model is None:
            U = rk4_step(U, p)
        else:
            U = learned_step(U, p, model)
            if model.k_c > 0 and k % model.k_c == 0:
                U = temporal_correction(U, hist[-model.k_c:], p, model)
        hist.append(U.copy())
        if len(hist) > 16:
            hist.pop(0)
        if save_every and k % save_every == 0:
            snaps.append(U.copy())
    return U, snaps


def rollout_batch(U0: np.ndarray, p: Problem, n_steps: int, model=None) -> np.ndarray:
    """Rollout of every trajectory of a batch ``[B, 2, ny, nx]`` independently."""
    return np.stack([rollout(U0[b], p, n_steps, model=model)[0] for b in range(U0.shape[0])])


# ----------------------------------------------------------------------------
# learnable module (Sec. 3.4, 3.5)
# ----------------------------------------------------------------------------
CNN_HIDDEN = 64
CNN_LAYERS = 6
N_COEF = 8 * 20  # per-face 5x4 correction for each of the eight instances


def gelu(x: np.ndarray) -> np.ndarray:
    """GELU activation (the sigma of the paper's network tables), erf form."""
    from scipy.special import erf

    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x: np.ndarray) -> np.ndarray:
    """d GELU / dx = Phi(x) + x phi(x)."""
    from scipy.special import erf

    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


def conv3x3(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """3x3 cross-correlation with periodic (circular) padding.

    ``out[o, j, i] = b[o] + sum_{c, a, e} W[o, c, a+1, e+1] x[c, j+a, i+e]``
    for a, e in {-1, 0, 1}; ``x[Cin, ny, nx]``, ``W[Cout, Cin, 3, 3]``.
    """
    out = np.broadcast_to(b[:, None, None], (W.shape[0],) + x.shape[1:]).astype(np.float64).copy()
    for a in (-1, 0, 1):
        for e in (-1, 0, 1):
            xs = shifted_c(x, a, e)
            out += np.einsum("oc,cji->oji", W[:, :, a + 1, e + 1], xs)
    return out


def shifted_c(x: np.ndarray, dj: int, di: int) -> np.ndarray:
    """Per-channel periodic shift ``g[c, j, i] = x[c, j + dj, i + di]``."""
    return np.roll(x, (-dj, -di), axis=(1, 2))


def cnn_forward(x: np.ndarray, layers: Sequence, keep: bool = False):
    """Six conv3x3 layers with GELU between them (no activation after the last).

    Returns the output, and with ``keep`` also the list of pre-activations.
    """
    h = x
    pre = []
    for l, (W, b) in enumerate(layers):
        z = conv3x3(h, W, b)
        pre.append(z)
        h = gelu(z) if l < len(layers) - 1 else z
    return (h, pre) if keep else h


def consistency_project(L: np.ndarray) -> np.ndarray:
    """Project a learned 5x4 kernel part onto the consistency null space.

    The paper requires the kernels to keep discrete conservation and
    consistency (Sec. 3.4) without writing the constraints; the reading used
    here: the learned part L (W_L plus the network's per-face correction) must
    have zero sum, zero first axial moment and zero first transverse moment,
    so that W_P + L still interpolates (differentiates) linear fields exactly.
    The three moment vectors 1, c, r are orthogonal on the 5x4 grid, so the
    projection removes each component independently. Works on ``[5, 4, ...]``.
    """
    c = AXIAL[None, :] * np.ones((5, 1))
    r = TRANSVERSE[:, None] * np.ones((1, 4))
    ext = (slice(None), slice(None)) + (None,) * (L.ndim - 2)
    one = np.ones((5, 4))
    out = L.copy()
    for m in (one, c, r):
        coef = np.tensordot(m, L, axes=([0, 1], [0, 1])) / np.sum(m * m)
        out = out - m[ext] * coef
    return out


@dataclass
class LearnedModel:
    """Parameters of the learnable module.

    ``W_L[kind, axis, 5, 4]``: learnable conv O_L (Sec. 3.4), one kernel per
    (interp/deriv, axis), shared by u and v.
    ``stencil``: list of six ``(W, b)`` conv3x3 layers, 2 -> 64 x5 -> 160,
    emitting the per-face 5x4 corrections of the eight instances (channel
    ``q * 20 + r * 4 + c``).
    ``tc``: list of six ``(W, b)`` layers, 2 k_c -> 64 x5 -> 2, the temporal
    correction network (Sec. 3.5); empty or k_c == 0 disables it.
    ``tc_fno``: the temporal correction as a Fourier neural operator instead
    (the paper's form, Sec. 3.5 and Table S3): ``oracle.fno.FNOParams`` with
    2 k_c input and 2 output channels; when set it replaces ``tc``.
    ``fno``: the frequency-domain operator O_F (``oracle.fno``), whose eight
    output channels add to the eight instances' face values; None disables it.
    Learned derivative parts are dimensionless and divided by the spacing
    along the instance's axis.
    """

    W_L: np.ndarray
    stencil: list
    tc: list = field(default_factory=list)
    k_c: int = 0
    #: frequency-domain operator O_F (oracle.fno.FNOParams) or None
    fno: object = None
    #: FNO temporal correction (oracle.fno.FNOParams, 2 k_c -> 2 channels) or None
    tc_fno: object = None
    #: ablation variant of the flux block (Sec. 4 ablation study, Table 4):
    #: 0 the full operator, 1 without the physics-based convolution
    #: (K = (W_L + C_theta) / h^deriv, no W_P and hence no consistency projection),
    #: 2 the frequency-domain operator only (face values = O_F(u))
    ablation: int = 0
    #: learnable conv of the passive scalar's four operator instances
    #: ``W_Ls[kind, axis, 5, 4]`` (shear flow, oracle.scalar). When set the model
    #: also learns the scalar's face operators: the stencil network then takes
    #: (u, v, s) (3 channels) and emits 240 channels, the eight velocity
    #: instances' 160 followed by the scalar instances' 80.
    W_Ls: Optional[np.ndarray] = None


def learned_kernels(U: np.ndarray, p: Problem, model: LearnedModel, C: Optional[np.ndarray] = None) -> list:
    """Per-face kernels K_f = W_P + proj(W_L + C_theta(u)_f) (Sec. 3.4, integrated operator).

    Ablation 1 (without the physics-based convolution) drops W_P and with it the
    consistency projection, whose job is to keep W_P's consistency: K_f = W_L +
    C_theta(u)_f. Ablation 2 (frequency-domain operator only) has zero kernels.
    ``C`` is the network's output when the caller has it (a model that also
    learns the scalar runs the network on (u, v, s))."""
    ny, nx = U.shape[1:]
    if model.ablation == 2:
        return [np.zeros((5, 4, ny, nx)) for _ in INSTANCES]
    if C is None:
        C = cnn_forward(U, model.stencil)
    ks = []
    for q, (_fld, axis, kind, _shift) in enumerate(INSTANCES):
        h = p.dx if axis == 0 else p.dy
        L = model.W_L[kind, axis][:, :, None, None] + C[q * 20:(q + 1) * 20].reshape(5, 4, ny, nx)
        if model.ablation == 0:
            L = consistency_project(L)
        if kind == 1:
            L = L / h
        ks.append(L if model.ablation == 1 else physics_kernel(kind, p.deriv_order, h)[:, :, None, None] + L)
    return ks


def learned_step(U: np.ndarray, p: Problem, model: LearnedModel) -> np.ndarray:
    """FV-module step with the learned flux block evaluated at every RK stage
    (O = O_P + O_L + O_F when the model has a frequency-domain operator)."""
    if model.fno is None:
        return rk4_step(U, p, kernels_fn=lambda W: learned_kernels(W, p, model))
    from .fno import fno_forward

    return rk4_step(U, p, kernels_fn=lambda W: (learned_kernels(W, p, model), fno_forward(W, model.fno)))


def temporal_correction(U: np.ndarray, hist: Sequence[np.ndarray], p: Problem,
                        model: LearnedModel) -> np.ndarray:
    """Temporal correction at k = M k_c (Sec. 3.2, Eq. for u_k; Sec. 3.5).

    u_k = FV(u_{k-1}) + TC(u_{k-k_c}, ..., u_{k-1}); the correction has its
    per-component mean removed (so mean momentum is kept) and, for
    Navier-Stokes, the corrected field is projected.
    """
    x = np.concatenate([h for h in hist], axis=0)
    if model.tc_fno is not None:
        from .fno import fno_forward

        c = fno_forward(x, model.tc_fno)
    else:
        c = cnn_forward(x, model.tc)
    c = c - c.mean(axis=(1, 2), keepdims=True)
    out = U + c
    return project(out, p) if p.flow == FLOW_NAVIER_STOKES else out


# ----------------------------------------------------------------------------
# diagnostics and metrics (App. D.1)
# ----------------------------------------------------------------------------
def shell_index(q: np.ndarray) -> np.ndarray:
    """Nearest integer to sqrt(q) for integer q >= 0, in exact integer arithmetic:
    the k with (k - 1/2)^2 <= q < (k + 1/2)^2, i.e. k^2 - k < q <= k^2 + k."""
    q = np.asarray(q, dtype=np.int64)
    k = np.floor(np.sqrt(q.astype(np.float64))).astype(np.int64)
    k = np.where(k * k > q, k - 1, k)
    k = np.where((k + 1) * (k + 1) <= q, k + 1, k)
    return np.where(q > k * k + k, k + 1, k)


def energy_spectrum(U: np.ndarray, kmax: int) -> np.ndarray:
    """Shell-summed kinetic-energy spectrum (the energy spectra the paper compares for
    the forced flow, Sec. 4 "Forced Flow" / Fig. 5). With the discrete Fourier
    coefficients u^(k) = N^-2 sum_x u(x) exp(-2 pi i k.x / N) over integer wavevectors
    k in [-N/2, N/2)^2, E(k) = 1/2 sum over |k| rounded to k of (|u^|^2 + |v^|^2), for
    k = 0 .. kmax. The half-cell offsets of the MAC faces change phases only. Summed
    over every shell, E equals 1/2 mean(u^2 + v^2) (Parseval)."""
    ny, nx = U.shape[1:]
    uh = np.fft.fft2(U[0]) / (nx * ny)
    vh = np.fft.fft2(U[1]) / (nx * ny)
    e = 0.5 * (np.abs(uh) ** 2 + np.abs(vh) ** 2)
    ky = np.rint(np.fft.fftfreq(ny) * ny).astype(np.int64)
    kx = np.rint(np.fft.fftfreq(nx) * nx).astype(np.int64)
    kk = shell_index(ky[:, None] ** 2 + kx[None, :] ** 2)
    E = np.zeros(kmax + 1)
    m = kk <= kmax
    np.add.at(E, kk[m], e[m])
    return E


def vorticity(U: np.ndarray, dx: float, dy: float) -> np.ndarray:
    """Corner vorticity w = dv/dx - du/dy by differences of adjacent faces."""
    return (U[1] - shifted(U[1], 0, -1)) / dx - (U[0] - shifted(U[0], -1, 0)) / dy


def pcc(a: np.ndarray, b: np.ndarray) -> float:
    """Pearson correlation coefficient cov(a, b) / (sigma_a sigma_b) (App. D.1)."""
    a = a.ravel() - a.mean()
    b = b.ravel() - b.mean()
    return float(np.dot(a, b) / math.sqrt(np.dot(a, a) * np.dot(b, b)))


def mse(a: np.ndarray, b: np.ndarray) -> float:
    """Mean squared error, the per-sample term of the training loss (Sec. 4.1)."""
    return float(np.mean((a - b) ** 2))
