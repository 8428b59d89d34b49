"""ctypes binding of the C ABI in ``include/fd.h`` (argument marshalling only).

Every computation runs in ``libldfv.so``; this module converts Python values
and torch CUDA tensors into the plain pointers and sizes the ABI takes. There
is no fallback: if the library cannot be loaded, every call raises.
"""

from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass
from typing import Optional

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libldfv.so")

FD_OK, FD_EINVAL, FD_ENOMEM, FD_ECUDA, FD_ENONFINITE, FD_ETIMEOUT, FD_EUNSUPPORTED = range(7)
FD_F32, FD_F64 = 0, 1
FD_BURGERS, FD_NAVIER_STOKES = 0, 1

#: every symbol include/fd.h declares
EXPORTS = [
    "fd_init",
    "fd_step",
    "fd_rollout",
    "fd_rollout_host",
    "fd_rollout_guarded",
    "fd_rollout_scalar",
    "fd_check_finite",
    "fd_check_finite_noalloc",
    "fd_last_launch_count",
    "fd_param_count",
    "fd_set_params",
    "fd_set_params_device",
    "fd_network_forward",
    "fd_step_adjoint",
    "fd_tc_adjoint",
    "fd_rollout_adjoint",
    "fd_train_step",
    "fd_train_step_scalar",
    "fd_step_adjoint_scalar",
    "fd_mse_loss",
    "fd_vorticity_pcc",
    "fd_energy_spectrum",
    "fd_adam_step",
    "fd_downsample",
    "fd_get_plan",
    "fd_set_plan",
    "fd_autotune",
    "fd_batch_create",
    "fd_batch_add",
    "fd_batch_run",
    "fd_batch_launch_count",
    "fd_batch_set_persistent",
    "fd_batch_persistent_count",
    "fd_batch_last_error",
    "fd_batch_destroy",
    "fd_destroy",
    "fd_last_error",
    "fd_version",
]


class FdGrid(C.Structure):
    _fields_ = [
        ("nx", C.c_int32),
        ("ny", C.c_int32),
        ("lx", C.c_double),
        ("ly", C.c_double),
        ("batch", C.c_int32),
        ("dtype", C.c_int32),
        ("flow", C.c_int32),
    ]


class FdForcing(C.Structure):
    _fields_ = [("kind", C.c_int32), ("amp", C.c_double), ("k", C.c_int32), ("drag", C.c_double)]


class FdOptions(C.Structure):
    _fields_ = [
        ("deriv_order", C.c_int32),
        ("interp_order", C.c_int32),
        ("learned", C.c_int32),
        ("k_c", C.c_int32),
        ("poisson_symbol", C.c_int32),
        ("ckpt_every", C.c_int32),
        ("spin_limit", C.c_int64),
        ("path", C.c_int32),
        ("fno_layers", C.c_int32),
        ("fno_modes", C.c_int32),
        ("fno_width", C.c_int32),
        ("tc_fno_layers", C.c_int32),
        ("tc_fno_modes", C.c_int32),
        ("tc_fno_width", C.c_int32),
        ("ablation", C.c_int32),
        ("scalar_learned", C.c_int32),
    ]


class FdPlan(C.Structure):
    _fields_ = [
        ("path", C.c_int32),
        ("cluster", C.c_int32),
        ("n_onchip", C.c_int32),
        ("n_stream", C.c_int32),
        ("resident", C.c_int32),
        ("us_per_step", C.c_double),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class FdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"fd status {status}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load ``libldfv.so`` and declare the ABI's signatures (raises if missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FdError(FD_EUNSUPPORTED, f"CUDA library {path} is not built; run __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, i32 = C.c_void_p, C.c_int32
    lib.fd_init.argtypes = [C.POINTER(FdGrid), C.c_double, C.c_double, C.POINTER(FdForcing),
                            C.POINTER(FdOptions), C.POINTER(vp)]
    lib.fd_init.restype = C.c_int
    lib.fd_step.argtypes = [vp, vp, vp, vp]
    lib.fd_step.restype = C.c_int
    lib.fd_rollout.argtypes = [vp, vp, vp, vp, i32, i32, vp]
    lib.fd_rollout.restype = C.c_int
    lib.fd_rollout_host.argtypes = [vp, vp, vp, i32, vp]
    lib.fd_rollout_host.restype = C.c_int
    lib.fd_rollout_guarded.argtypes = [vp, vp, vp, i32, i32, vp, vp]
    lib.fd_rollout_guarded.restype = C.c_int
    lib.fd_rollout_scalar.argtypes = [vp, C.c_double, vp, vp, vp, vp, i32, vp]
    lib.fd_rollout_scalar.restype = C.c_int
    lib.fd_check_finite.argtypes = [vp, vp, vp]
    lib.fd_check_finite.restype = C.c_int
    lib.fd_last_launch_count.argtypes = [vp]
    lib.fd_last_launch_count.restype = i32
    lib.fd_param_count.argtypes = [vp]
    lib.fd_param_count.restype = C.c_int64
    lib.fd_set_params.argtypes = [vp, vp, C.c_int64, vp]
    lib.fd_set_params.restype = C.c_int
    lib.fd_set_params_device.argtypes = [vp, vp, C.c_int64, vp]
    lib.fd_set_params_device.restype = C.c_int
    lib.fd_network_forward.argtypes = [vp, vp, vp, vp]
    lib.fd_network_forward.restype = C.c_int
    lib.fd_step_adjoint.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.fd_step_adjoint.restype = C.c_int
    lib.fd_tc_adjoint.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.fd_tc_adjoint.restype = C.c_int
    lib.fd_rollout_adjoint.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp]
    lib.fd_rollout_adjoint.restype = C.c_int
    lib.fd_train_step.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp]
    lib.fd_train_step.restype = C.c_int
    lib.fd_train_step_scalar.argtypes = [vp, C.c_double, vp, vp, vp, vp, i32, i32, vp, vp, vp]
    lib.fd_train_step_scalar.restype = C.c_int
    lib.fd_step_adjoint_scalar.argtypes = [vp, C.c_double, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.fd_step_adjoint_scalar.restype = C.c_int
    lib.fd_mse_loss.argtypes = [vp, vp, vp, C.c_int64, vp, vp, vp]
    lib.fd_mse_loss.restype = C.c_int
    lib.fd_energy_spectrum.argtypes = [vp, vp, vp, i32, vp]
    lib.fd_energy_spectrum.restype = C.c_int
    lib.fd_vorticity_pcc.argtypes = [vp, vp, vp, vp, vp]
    lib.fd_vorticity_pcc.restype = C.c_int
    lib.fd_adam_step.argtypes = [vp, vp, vp, vp, C.c_int64, i32, C.c_float, C.c_float, C.c_float, C.c_float, i32, vp]
    lib.fd_adam_step.restype = C.c_int
    lib.fd_downsample.argtypes = [vp, vp, i32, i32, i32, i32, vp]
    lib.fd_downsample.restype = C.c_int
    lib.fd_get_plan.argtypes = [vp, C.POINTER(FdPlan)]
    lib.fd_get_plan.restype = C.c_int
    lib.fd_set_plan.argtypes = [vp, C.POINTER(FdPlan)]
    lib.fd_set_plan.restype = C.c_int
    lib.fd_autotune.argtypes = [vp, i32, C.POINTER(FdPlan), i32, C.POINTER(i32), vp]
    lib.fd_autotune.restype = C.c_int
    lib.fd_batch_create.argtypes = [C.POINTER(C.c_void_p)]
    lib.fd_batch_create.restype = C.c_int
    lib.fd_batch_add.argtypes = [vp, vp, vp, vp, i32]
    lib.fd_batch_add.restype = C.c_int
    lib.fd_batch_run.argtypes = [vp, vp]
    lib.fd_batch_run.restype = C.c_int
    lib.fd_batch_launch_count.argtypes = [vp]
    lib.fd_batch_launch_count.restype = i32
    lib.fd_batch_set_persistent.argtypes = [vp, i32]
    lib.fd_batch_set_persistent.restype = C.c_int
    lib.fd_batch_persistent_count.argtypes = [vp]
    lib.fd_batch_persistent_count.restype = i32
    lib.fd_batch_last_error.argtypes = [vp]
    lib.fd_batch_last_error.restype = C.c_char_p
    lib.fd_batch_destroy.argtypes = [vp]
    lib.fd_batch_destroy.restype = C.c_int
    lib.fd_check_finite_noalloc.argtypes = [vp, C.c_int64, i32, C.POINTER(C.c_int64), vp]
    lib.fd_check_finite_noalloc.restype = C.c_int
    lib.fd_destroy.argtypes = [vp]
    lib.fd_destroy.restype = C.c_int
    lib.fd_last_error.argtypes = [vp]
    lib.fd_last_error.restype = C.c_char_p
    lib.fd_version.argtypes = []
    lib.fd_version.restype = C.c_char_p
    _lib = lib
    return lib


@dataclass
class Config:
    """Python mirror of fd_grid + fd_forcing + fd_options."""

    n: int
    batch: int = 1
    dtype: str = "f32"
    flow: str = "ns"  # "ns" or "burgers"
    nu: float = 1e-3
    dt: float = 1e-3
    lx: float = 2 * math.pi
    ly: float = 2 * math.pi
    forcing: Optional[str] = None  # None or "kolmogorov"
    amp: float = 1.0
    kf: int = 4
    drag: float = 0.1
    deriv_order: int = 4
    poisson_symbol: int = 0
    learned: bool = False
    k_c: int = 0
    path: int = 0  # 0 automatic, 1 on chip, 2 streaming through HBM, 3 generic grid
    fno_layers: int = 0  # frequency-domain operator O_F: Fourier layers (0 = off)
    fno_modes: int = 0
    fno_width: int = 0
    tc_fno_layers: int = 0  # temporal correction as an FNO (0 = CNN head); needs k_c > 0
    tc_fno_modes: int = 0
    tc_fno_width: int = 0
    ablation: int = 0  # 0 full flux block, 1 without the physics conv, 2 frequency operator only (Table 4)
    scalar_learned: bool = False  # the model also learns the passive scalar (network on (u, v, s), 240 channels)
    ny: Optional[int] = None  # rows when the grid is rectangular (generic-grid path); n = columns
    spin_limit: int = 0  # iteration limit of the tensor-core kernels' bounded waits (0 = library default)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> int:
    return t.data_ptr() if hasattr(t, "data_ptr") else int(t)


class Solver:
    """One fd_ctx: a batch of trajectories of one grid, flow and time step."""

    def __init__(self, cfg: Config):
        self.lib = load()
        self.cfg = cfg
        g = FdGrid(cfg.n, cfg.ny or cfg.n, cfg.lx, cfg.ly, cfg.batch, FD_F64 if cfg.dtype == "f64" else FD_F32,
                   FD_BURGERS if cfg.flow == "burgers" else FD_NAVIER_STOKES)
        f = FdForcing(1 if cfg.forcing == "kolmogorov" else 0, cfg.amp, cfg.kf, cfg.drag)
        o = FdOptions(cfg.deriv_order, 2, 1 if cfg.learned else 0, cfg.k_c, cfg.poisson_symbol, 8, cfg.spin_limit, cfg.path,
                      cfg.fno_layers, cfg.fno_modes, cfg.fno_width, cfg.tc_fno_layers, cfg.tc_fno_modes,
                      cfg.tc_fno_width, cfg.ablation, 1 if cfg.scalar_learned else 0)
        h = C.c_void_p()
        st = self.lib.fd_init(C.byref(g), cfg.nu, cfg.dt, C.byref(f), C.byref(o), C.byref(h))
        if st != FD_OK:
            raise FdError(st, self.lib.fd_last_error(None).decode())
        self.h = h

    # --- helpers --------------------------------------------------------
    def _check(self, st):
        if st != FD_OK:
            raise FdError(st, self.lib.fd_last_error(self.h).decode())

    @property
    def state_shape(self):
        return (self.cfg.batch, 2, self.cfg.ny or self.cfg.n, self.cfg.n)

    @property
    def torch_dtype(self):
        import torch

        return torch.float64 if self.cfg.dtype == "f64" else torch.float32

    # --- ABI calls --------------------------------------------------------
    def step(self, u_in, u_out, stream=None):
        self._check(self.lib.fd_step(self.h, _ptr(u_in), _ptr(u_out), _stream_handle(stream)))

    def rollout(self, u0, u_final, n_steps: int, traj=None, save_every: int = 0, stream=None):
        tp = _ptr(traj) if traj is not None else None
        self._check(self.lib.fd_rollout(self.h, _ptr(u0), tp, _ptr(u_final), int(n_steps), int(save_every),
                                        _stream_handle(stream)))

    def rollout_scalar(self, u0, s0, u_final, s_final, n_steps: int, diffusivity: float, stream=None):
        """Velocity and passive scalar s [B, ny, nx] together (generic-grid path)."""
        self._check(self.lib.fd_rollout_scalar(self.h, float(diffusivity), _ptr(u0), _ptr(s0), _ptr(u_final),
                                               _ptr(s_final), int(n_steps), _stream_handle(stream)))

    def rollout_guarded(self, u0, u_final, n_steps: int, fell_back, chunk: int = 0, stream=None):
        """Learned rollout with the plain FV step as fallback; fell_back (device int32[batch])
        receives -1 or the step at which the trajectory switched to the plain solver."""
        self._check(self.lib.fd_rollout_guarded(self.h, _ptr(u0), _ptr(u_final), int(n_steps), int(chunk),
                                                _ptr(fell_back), _stream_handle(stream)))

    def rollout_host(self, u0_host, u_final_host, n_steps: int, stream=None):
        self._check(self.lib.fd_rollout_host(self.h, _ptr(u0_host), _ptr(u_final_host), int(n_steps),
                                             _stream_handle(stream)))

    def plan(self) -> dict:
        """The context's launch plan (path, cluster, n_onchip, n_stream, resident, us_per_step)."""
        p = FdPlan()
        self._check(self.lib.fd_get_plan(self.h, C.byref(p)))
        return p.as_dict()

    def set_plan(self, cluster: int, n_onchip: int, n_stream: int = 0):
        p = FdPlan(0, int(cluster), int(n_onchip), int(n_stream), 0, 0.0)
        self._check(self.lib.fd_set_plan(self.h, C.byref(p)))

    def autotune(self, probe_steps: int = 32, stream=None) -> list:
        """Time every candidate launch plan, keep the fastest; returns the candidates."""
        rep = (FdPlan * 32)()
        n = C.c_int32(0)
        self._check(self.lib.fd_autotune(self.h, int(probe_steps), rep, 32, C.byref(n), _stream_handle(stream)))
        return [rep[i].as_dict() for i in range(min(n.value, 32))]

    def check_finite(self, u, stream=None) -> bool:
        st = self.lib.fd_check_finite(self.h, _ptr(u), _stream_handle(stream))
        if st == FD_ENONFINITE:
            return False
        self._check(st)
        return True

    def param_count(self) -> int:
        return int(self.lib.fd_param_count(self.h))

    def set_params(self, params, stream=None):
        """Upload the learnable parameters (host float32 array, layout of include/fd.h)."""
        import numpy as np

        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        self._check(self.lib.fd_set_params(self.h, p.ctypes.data, int(p.size), _stream_handle(stream)))

    def set_params_device(self, params, stream=None):
        """Upload the learnable parameters from a device float32 tensor (no synchronisation)."""
        self._check(self.lib.fd_set_params_device(self.h, _ptr(params), int(params.numel()), _stream_handle(stream)))

    def network_forward(self, u, coef_out=None, stream=None):
        """coef_out[batch, 160, n, n] float32 = C_theta(u); None runs the network only.
        With scalar_learned, u is [batch, 3, ny, n] (u, v, s) and coef_out has 240 channels."""
        cp = _ptr(coef_out) if coef_out is not None else None
        self._check(self.lib.fd_network_forward(self.h, _ptr(u), cp, _stream_handle(stream)))

    def step_adjoint(self, u_in, lam_out, lam_in, dparams=None, stream=None):
        """lam_in = (du'/du)^T lam_out for u' = step(u_in); dparams (device
        float32, fd_param_count values) accumulates (du'/dtheta)^T lam_out."""
        dp = _ptr(dparams) if dparams is not None else None
        self._check(self.lib.fd_step_adjoint(self.h, _ptr(u_in), _ptr(lam_out), _ptr(lam_in), dp,
                                             _stream_handle(stream)))

    def tc_adjoint(self, hist, lam, hist_bar, vbar=None, dparams=None, stream=None):
        """Reverse mode of one temporal correction: hist [k_c, batch, 2, n, n] (oldest first),
        lam the cotangent of the corrected state; writes hist_bar [k_c, batch, 2, n, n] and
        vbar = P(lam) when given; dparams accumulates the correction network's gradients."""
        self._check(self.lib.fd_tc_adjoint(self.h, _ptr(hist), _ptr(lam), _ptr(vbar) if vbar is not None else None,
                                           _ptr(hist_bar), _ptr(dparams) if dparams is not None else None,
                                           _stream_handle(stream)))

    def rollout_adjoint(self, u0, n_steps: int, ckpt_every: int, lam_traj, lam0, dparams=None, stream=None):
        """lam0 = dL/du0 for the cotangents lam_traj of the states after steps 1..n."""
        dp = _ptr(dparams) if dparams is not None else None
        self._check(self.lib.fd_rollout_adjoint(self.h, _ptr(u0), int(n_steps), int(ckpt_every), _ptr(lam_traj),
                                                _ptr(lam0), dp, _stream_handle(stream)))

    def step_adjoint_scalar(self, diffusivity: float, u_in, s_in, lam_u_out, lam_s_out, lam_u_in, lam_s_in,
                            dparams=None, stream=None):
        """Reverse mode of one joint velocity-scalar step: (lam_u_in, lam_s_in) from the
        cotangents of (u', s'); dparams accumulates the gradient of a scalar-learning model."""
        dp = _ptr(dparams) if dparams is not None else None
        self._check(self.lib.fd_step_adjoint_scalar(self.h, float(diffusivity), _ptr(u_in), _ptr(s_in),
                                                    _ptr(lam_u_out), _ptr(lam_s_out), _ptr(lam_u_in),
                                                    _ptr(lam_s_in), dp, _stream_handle(stream)))

    def train_step_scalar(self, diffusivity: float, u0, s0, targets_u, targets_s, n_steps: int, ckpt_every: int,
                          dparams, loss, stream=None):
        """MSE of the joint n-step rollout against targets_u [n, B, 2, ny, nx] and
        targets_s [n, B, ny, nx] -> loss (device float64), dparams += gradient."""
        self._check(self.lib.fd_train_step_scalar(self.h, float(diffusivity), _ptr(u0), _ptr(s0), _ptr(targets_u),
                                                  _ptr(targets_s), int(n_steps), int(ckpt_every), _ptr(dparams),
                                                  _ptr(loss), _stream_handle(stream)))

    def train_step(self, u0, targets, n_steps: int, ckpt_every: int, dparams, loss, stream=None):
        """MSE of the n-step rollout against targets -> loss (device float64), dparams += gradient."""
        self._check(self.lib.fd_train_step(self.h, _ptr(u0), _ptr(targets), int(n_steps), int(ckpt_every),
                                           _ptr(dparams), _ptr(loss), _stream_handle(stream)))

    def mse_loss(self, pred, target, loss, grad=None, stream=None):
        g = _ptr(grad) if grad is not None else None
        self._check(self.lib.fd_mse_loss(self.h, _ptr(pred), _ptr(target), int(pred.numel()), _ptr(loss), g,
                                         _stream_handle(stream)))

    def energy_spectrum(self, u, out, stream=None):
        """Shell-summed kinetic-energy spectrum into out (device float64 [batch, kmax + 1])."""
        self._check(self.lib.fd_energy_spectrum(self.h, _ptr(u), _ptr(out), int(out.shape[-1]) - 1,
                                                _stream_handle(stream)))

    def vorticity_pcc(self, a, b, out, stream=None):
        """out[batch] (device float64) = vorticity correlation of states a and b per trajectory."""
        self._check(self.lib.fd_vorticity_pcc(self.h, _ptr(a), _ptr(b), _ptr(out), _stream_handle(stream)))

    def last_launch_count(self) -> int:
        return int(self.lib.fd_last_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.fd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """fd_batch: rollouts of several solvers (mixed sizes, flows, learned and
    plain) replayed as one CUDA graph; the plain FP32 trajectories of N <= 64
    run in one persistent launch, every other solver is a parallel branch."""

    def __init__(self):
        self.lib = load()
        h = C.c_void_p()
        _check_free(self.lib, self.lib.fd_batch_create(C.byref(h)))
        self.h = h
        self._keep = []

    def add(self, solver: "Solver", u0, u_final, n_steps: int):
        st = self.lib.fd_batch_add(self.h, solver.h, _ptr(u0), _ptr(u_final), int(n_steps))
        if st != FD_OK:
            raise FdError(st, self.lib.fd_batch_last_error(self.h).decode())
        self._keep.append((solver, u0, u_final))

    def run(self, stream=None):
        st = self.lib.fd_batch_run(self.h, _stream_handle(stream))
        if st != FD_OK:
            raise FdError(st, self.lib.fd_batch_last_error(self.h).decode())

    def launch_count(self) -> int:
        return int(self.lib.fd_batch_launch_count(self.h))

    def set_persistent(self, enable: bool):
        _check_free(self.lib, self.lib.fd_batch_set_persistent(self.h, 1 if enable else 0))

    def persistent_count(self) -> int:
        return int(self.lib.fd_batch_persistent_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.fd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_free(lib, st):
    if st != FD_OK:
        raise FdError(st, lib.fd_last_error(None).decode())


def adam_step(params, grads, m, v, t: int, lr: float = 1e-4, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8, zero_grads: bool = True, stream=None):
    """One Adam update of device float32 tensors (fd_adam_step)."""
    lib = load()
    _check_free(lib, lib.fd_adam_step(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), int(params.numel()), int(t),
                                      float(lr), float(beta1), float(beta2), float(eps), 1 if zero_grads else 0,
                                      _stream_handle(stream)))


def downsample(fine, coarse, ratio: int, stream=None):
    """Face-average coarse-graining fine[B,2,n,n] -> coarse[B,2,n/ratio,n/ratio] (fd_downsample)."""
    import torch

    lib = load()
    dt = FD_F64 if fine.dtype == torch.float64 else FD_F32
    _check_free(lib, lib.fd_downsample(_ptr(fine), _ptr(coarse), int(fine.shape[0]), int(fine.shape[-1]), int(ratio),
                                       dt, _stream_handle(stream)))


def version() -> str:
    return load().fd_version().decode()
