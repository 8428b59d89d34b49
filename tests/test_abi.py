"""The C ABI library loads, exports every symbol include/*.h declares, and
validates its arguments on the host (no GPU needed for any of this)."""

import ctypes as C
import glob
import os
import re

import pytest

from paper_2507_01975_gb300 import fd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(fd_[a-z_0-9]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2507_01975_gb300 import build

    build.build()
    return fd.load()


def test_library_exports_every_declared_symbol(lib):
    declared = _declared()
    assert declared, "no fd_* declarations found"
    assert declared <= set(fd.EXPORTS) | declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(fd.EXPORTS) == declared


def test_version_string(lib):
    assert fd.version().startswith("ldfv")


def _init(lib, n=32, batch=1, dtype=fd.FD_F32, flow=fd.FD_NAVIER_STOKES, nu=1e-3, dt=1e-3, opts=None,
          lx=6.283185307179586):
    g = fd.FdGrid(n, n, lx, lx, batch, dtype, flow)
    h = C.c_void_p()
    o = C.byref(opts) if opts is not None else None
    return lib.fd_init(C.byref(g), nu, dt, None, o, C.byref(h)), h


@pytest.mark.parametrize(
    "kw",
    [
        dict(n=12),
        dict(n=4),
        dict(n=4096),
        # Burgers runs on any grid in [4, 8192]^2 (generic-grid path), but not beyond
        dict(n=3, flow=fd.FD_BURGERS),
        dict(n=9000, flow=fd.FD_BURGERS),
        dict(n=25, flow=fd.FD_BURGERS, opts=fd.FdOptions(4, 2, 0, 0, 0, 8, 1 << 26, 4)),
        dict(batch=0),
        dict(dt=0.0),
        dict(dt=-1e-3),
        dict(nu=-1.0),
        dict(dtype=7),
        dict(flow=3),
        dict(lx=0.0),
        dict(opts=fd.FdOptions(3, 2, 0, 0, 0, 8, 1)),
        dict(opts=fd.FdOptions(4, 4, 0, 0, 0, 8, 1)),
        # frequency-domain operator: too many layers, without the learned module,
        # width and modes out of range (modes <= N/2)
        dict(n=64, opts=fd.FdOptions(4, 2, 1, 0, 0, 8, 1 << 26, 0, 9, 16, 8)),
        dict(n=64, opts=fd.FdOptions(4, 2, 0, 0, 0, 8, 1 << 26, 0, 2, 16, 8)),
        dict(n=64, opts=fd.FdOptions(4, 2, 1, 0, 0, 8, 1 << 26, 0, 2, 16, 0)),
        dict(n=64, opts=fd.FdOptions(4, 2, 1, 0, 0, 8, 1 << 26, 0, 2, 16, 33)),
        dict(n=64, opts=fd.FdOptions(4, 2, 1, 0, 0, 8, 1 << 26, 0, 2, 16, 12)),
        dict(n=64, opts=fd.FdOptions(4, 2, 1, 0, 0, 8, 1 << 26, 0, 2, 33, 8)),
        dict(n=64, opts=fd.FdOptions(4, 2, 1, 0, 0, 8, 1 << 26, 0, 2, 0, 8)),
        # FNO temporal correction: without k_c, too many layers, width and modes out of range
        dict(n=64, opts=fd.FdOptions(4, 2, 1, 0, 0, 8, 1 << 26, 0, 0, 0, 0, 4, 32, 8)),
        dict(n=64, opts=fd.FdOptions(4, 2, 1, 4, 0, 8, 1 << 26, 0, 0, 0, 0, 9, 32, 8)),
        dict(n=64, opts=fd.FdOptions(4, 2, 1, 4, 0, 8, 1 << 26, 0, 0, 0, 0, 4, 32, 12)),
        dict(n=64, opts=fd.FdOptions(4, 2, 1, 4, 0, 8, 1 << 26, 0, 0, 0, 0, 4, 33, 8)),
        dict(n=32, opts=fd.FdOptions(4, 2, 1, 4, 0, 8, 1 << 26, 0, 0, 0, 0, 4, 17, 8)),
        # ablation variants: out of range, without the learned module, O_F only without O_F
        dict(n=64, opts=fd.FdOptions(4, 2, 1, 0, 0, 8, 1 << 26, 0, 0, 0, 0, 0, 0, 0, 3)),
        dict(n=64, opts=fd.FdOptions(4, 2, 0, 0, 0, 8, 1 << 26, 0, 0, 0, 0, 0, 0, 0, 1)),
        dict(n=64, opts=fd.FdOptions(4, 2, 1, 0, 0, 8, 1 << 26, 0, 0, 0, 0, 0, 0, 0, 2)),
        # the learned scalar: without the learned module, out of range
        dict(n=64, opts=fd.FdOptions(4, 2, 0, 0, 0, 8, 1 << 26, 0, 0, 0, 0, 0, 0, 0, 0, 1)),
        dict(n=64, opts=fd.FdOptions(4, 2, 1, 0, 0, 8, 1 << 26, 0, 0, 0, 0, 0, 0, 0, 0, 2)),
    ],
)
def test_init_rejects_invalid_arguments(lib, kw):
    st, h = _init(lib, **kw)
    assert st == fd.FD_EINVAL
    assert h.value is None
    assert len(lib.fd_last_error(None)) > 0


def test_init_rejects_null_pointers(lib):
    h = C.c_void_p()
    assert lib.fd_init(None, 1e-3, 1e-3, None, None, C.byref(h)) == fd.FD_EINVAL
    g = fd.FdGrid(32, 32, 1.0, 1.0, 1, 0, 1)
    assert lib.fd_init(C.byref(g), 1e-3, 1e-3, None, None, None) == fd.FD_EINVAL


def test_calls_on_null_context_are_rejected(lib):
    assert lib.fd_step(None, None, None, None) == fd.FD_EINVAL
    assert lib.fd_rollout(None, None, None, None, 1, 0, None) == fd.FD_EINVAL
    assert lib.fd_rollout_host(None, None, None, 1, None) == fd.FD_EINVAL
    assert lib.fd_rollout_guarded(None, None, None, 1, 0, None, None) == fd.FD_EINVAL
    assert lib.fd_check_finite(None, None, None) == fd.FD_EINVAL
    assert lib.fd_destroy(None) == fd.FD_OK
    assert lib.fd_last_launch_count(None) == 0
    assert lib.fd_batch_set_persistent(None, 1) == fd.FD_EINVAL
    assert lib.fd_batch_persistent_count(None) == 0
    assert lib.fd_batch_run(None, None) == fd.FD_EINVAL
    assert lib.fd_step_adjoint_scalar(None, 1e-3, None, None, None, None, None, None, None, None) == fd.FD_EINVAL
    assert lib.fd_train_step_scalar(None, 1e-3, None, None, None, None, 1, 1, None, None, None) == fd.FD_EINVAL
    assert lib.fd_tc_adjoint(None, None, None, None, None, None, None) == fd.FD_EINVAL
    assert lib.fd_rollout_scalar(None, 1e-3, None, None, None, None, 1, None) == fd.FD_EINVAL


def test_grids_without_a_kernel_are_unsupported_not_invalid(lib):
    # FP64 runs on chip only (N <= 128); the streaming path is FP32
    st, _ = _init(lib, n=512, dtype=fd.FD_F64)
    assert st == fd.FD_EUNSUPPORTED
    # forcing the on-chip path beyond its sizes
    st, _ = _init(lib, n=512, opts=fd.FdOptions(4, 2, 0, 0, 0, 8, 1 << 26, 1))
    assert st == fd.FD_EUNSUPPORTED
    # the learned module is FP32, and its Fourier operators are built for the
    # tensor-core grids (32^2, 64^2) only
    st, _ = _init(lib, n=128, dtype=fd.FD_F64, opts=fd.FdOptions(4, 2, 1, 0, 0, 8, 1 << 26, 0))
    assert st == fd.FD_EUNSUPPORTED
    st, _ = _init(lib, n=128, opts=fd.FdOptions(4, 2, 1, 0, 0, 8, 1 << 26, 0, 2, 16, 8))
    assert st == fd.FD_EUNSUPPORTED
    # Navier-Stokes on the generic-grid path is FP32 with nx, ny in [32, 2048]; an
    # unknown path value is invalid
    st, _ = _init(lib, n=64, dtype=fd.FD_F64, opts=fd.FdOptions(4, 2, 0, 0, 0, 8, 1 << 26, 3))
    assert st == fd.FD_EUNSUPPORTED
    st, _ = _init(lib, n=16, opts=fd.FdOptions(4, 2, 0, 0, 0, 8, 1 << 26, 3))
    assert st == fd.FD_EUNSUPPORTED
    st, _ = _init(lib, n=25, flow=fd.FD_BURGERS, dtype=fd.FD_F64, opts=fd.FdOptions(4, 2, 1, 0, 0, 8, 1 << 26, 0))
    assert st == fd.FD_EUNSUPPORTED
    # learned Navier-Stokes on the generic-grid path needs nx, ny >= 32
    st, _ = _init(lib, n=16, opts=fd.FdOptions(4, 2, 1, 0, 0, 8, 1 << 26, 0))
    assert st == fd.FD_EUNSUPPORTED
    st, _ = _init(lib, n=64, opts=fd.FdOptions(4, 2, 0, 0, 0, 8, 1 << 26, 4))
    assert st == fd.FD_EINVAL
    # a model that learns the scalar: FP32 generic-grid path, full operator only
    st, _ = _init(lib, n=64, dtype=fd.FD_F64, opts=fd.FdOptions(4, 2, 1, 0, 0, 8, 1 << 26, 0, 0, 0, 0, 0, 0, 0, 0, 1))
    assert st == fd.FD_EUNSUPPORTED
    st, _ = _init(lib, n=64, opts=fd.FdOptions(4, 2, 1, 0, 0, 8, 1 << 26, 0, 0, 0, 0, 0, 0, 0, 1, 1))
    assert st == fd.FD_EUNSUPPORTED
    st, _ = _init(lib, n=64, opts=fd.FdOptions(4, 2, 1, 0, 0, 8, 1 << 26, 1, 0, 0, 0, 0, 0, 0, 0, 1))
    assert st == fd.FD_EUNSUPPORTED


def test_options_struct_layout():
    # int32 x 6, int64, int32 x 9, padded to the int64's alignment
    assert C.sizeof(fd.FdOptions) == 72
    assert fd.FdOptions.scalar_learned.offset == 64
