"""fd_check_finite_noalloc: the NaN/Inf scan for callers that may not allocate.

Callers running under a framework memory pool that forbids raw cudaMalloc, or
on a path that must not enter the allocator, use this entry point instead of
fd_check_finite; its scratch is a static device array inside the library. The
test calls it through the C ABI and checks its answer against fd_check_finite
(the allocating entry point) and against a host count, on two calls in a row
with different inputs, so that the previous call's leftovers in the shared
array cannot leak into the next answer. This file is collected last.
"""

import ctypes as C

import numpy as np
import pytest

from paper_2507_01975_gb300 import fd

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_01975_gb300 import build

    build.build()
    lib = fd.load()
    lib.fd_check_finite_noalloc.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_int64), C.c_void_p]
    lib.fd_check_finite_noalloc.restype = C.c_int
    return lib


def _noalloc(lib, u, dtype_code):
    cnt = C.c_int64(-1)
    st = lib.fd_check_finite_noalloc(u.data_ptr(), u.numel(), dtype_code, C.byref(cnt),
                                     torch.cuda.current_stream().cuda_stream)
    return st, cnt.value


@pytest.mark.parametrize("dtype,code", [(torch.float32, fd.FD_F32), (torch.float64, fd.FD_F64)])
def test_noalloc_matches_allocating_scan_two_calls(lib, dtype, code):
    n, b = (128, 16) if code == fd.FD_F64 else (256, 16)  # largest grid built for each type
    cfg = fd.Config(n=n, batch=b, dtype="f64" if code == fd.FD_F64 else "f32")
    s = fd.Solver(cfg)
    g = torch.Generator(device="cpu").manual_seed(5)
    bad = torch.randn((b, 2, n, n), generator=g, dtype=dtype).cuda()
    flat = bad.view(-1)
    idx = torch.tensor([0, 17, 65_536 * 3 + 5, flat.numel() - 1])
    flat[idx[:2]] = float("nan")
    flat[idx[2]] = float("inf")
    flat[idx[3]] = float("-inf")
    good = torch.randn((b, 2, n, n), generator=g, dtype=dtype).cuda()
    for u, expect_count in ((bad, 4), (good, 0)):  # two calls in a row, different answers
        st, cnt = _noalloc(lib, u, code)
        ref_ok = s.check_finite(u)
        host_count = int(np.count_nonzero(~np.isfinite(u.cpu().numpy())))
        assert cnt == host_count == expect_count
        assert (st == fd.FD_OK) == ref_ok
        assert st in (fd.FD_OK, fd.FD_ENONFINITE)


def test_noalloc_rejects_oversize_and_bad_arguments(lib):
    u = torch.zeros(8, device="cuda")
    cnt = C.c_int64(0)
    s = torch.cuda.current_stream().cuda_stream
    too_many = (1 << 24) + 1
    assert lib.fd_check_finite_noalloc(u.data_ptr(), too_many, fd.FD_F32, C.byref(cnt), s) == fd.FD_EINVAL
    assert lib.fd_check_finite_noalloc(u.data_ptr(), -1, fd.FD_F32, C.byref(cnt), s) == fd.FD_EINVAL
    assert lib.fd_check_finite_noalloc(u.data_ptr(), 8, 9, C.byref(cnt), s) == fd.FD_EINVAL
    assert lib.fd_check_finite_noalloc(None, 8, fd.FD_F32, C.byref(cnt), s) == fd.FD_EINVAL
    assert lib.fd_check_finite_noalloc(u.data_ptr(), 0, fd.FD_F32, C.byref(cnt), s) == fd.FD_OK
    assert cnt.value == 0


def test_noalloc_at_the_maximum_count_and_allocates_nothing(lib):
    # FD_NOALLOC_MAX_ELEMS elements: every per-block slot is used and the last
    # one sits next to the total; the only non-finite value is the last element
    n = 1 << 24
    u = torch.zeros(n, dtype=torch.float32, device="cuda")
    u[-1] = float("nan")
    st, cnt = _noalloc(lib, u, fd.FD_F32)
    assert st == fd.FD_ENONFINITE and cnt == 1
    u[-1] = 0.0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k in range(5):
        u[k * 1000] = float("inf") if k % 2 else 0.0
        st, cnt = _noalloc(lib, u, fd.FD_F32)
        assert cnt == (k + 1) // 2 and (st == fd.FD_ENONFINITE) == (cnt > 0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
