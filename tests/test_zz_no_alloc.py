"""bfcs_body_force_noalloc, the allocation-free body-force generator.

It serves callers that may not allocate device memory while they run (their
memory belongs to their own pool or caching allocator, or an allocation could
stall a time-critical loop).  Its output must match bfcs_body_force within
the tolerance the other body-force tests use, on two calls in a row (the
fixed scratch array is reused and keeps the previous call's contents).
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2601_00822_gb300 import _lib

pytestmark = pytest.mark.gpu

TOL = {_lib.FP64: 1e-15, _lib.FP32: 1e-7}


def _field(lib, fn, dims, centre, a, precision):
    nx, ny, nz = dims
    dt = torch.float64 if precision == _lib.FP64 else torch.float32
    out = torch.full((3, nz, ny, nx), float("nan"), dtype=dt, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = getattr(lib, fn)(nx, ny, nz, float(centre[0]), float(centre[1]), float(centre[2]), float(a),
                            precision, C.c_void_p(out.data_ptr()), stream)
    assert code == _lib.OK, (fn, code)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("precision", [_lib.FP64, _lib.FP32])
def test_noalloc_matches_allocating_entry_point_twice(precision):
    lib = _lib.load()
    small = ((48, 24, 96), (24.0, 12.0, 48.0), 7.0)
    large = ((256, 256, 256), (128.0, 128.0, 128.0), 24.0)
    # calls in a row: small then large, then small again after the large call has
    # left partial sums in scratch slots the small grid does not use
    for dims, centre, a in (small, large, small):
        ref = _field(lib, "bfcs_body_force", dims, centre, a, precision)
        got = _field(lib, "bfcs_body_force_noalloc", dims, centre, a, precision)
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= TOL[precision] * np.abs(ref).max()
        assert abs(float(got[0].astype(np.float64).sum())) <= 1e-6 * np.abs(got[0]).sum()


def test_noalloc_leaves_device_memory_unchanged():
    """After a first call (which may load the library's device code), further calls
    change neither the device's free memory nor torch's allocator state."""
    lib = _lib.load()
    dims, centre, a = (128, 96, 64), (64.0, 48.0, 32.0), 9.0
    nx, ny, nz = dims
    out = torch.empty((3, nz, ny, nx), dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call():
        code = lib.bfcs_body_force_noalloc(nx, ny, nz, *centre, a, _lib.FP64, C.c_void_p(out.data_ptr()),
                                           stream)
        assert code == _lib.OK
        torch.cuda.synchronize()
    call()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_reserved() == reserved0


def test_noalloc_rejects_grids_beyond_its_scratch():
    lib = _lib.load()
    small = torch.empty(3, dtype=torch.float32, device="cuda")
    code = lib.bfcs_body_force_noalloc(1024, 1024, 256, 1.0, 1.0, 1.0, 4.0, _lib.FP32,
                                       C.c_void_p(small.data_ptr()),
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == _lib.ERR_INVALID_ARG
