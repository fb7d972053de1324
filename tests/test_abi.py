"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
symbol include/bfcs.h declares (no compute calls here)."""
import ctypes
import os
import re

from paper_2601_00822_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bfcs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bfcs_[a-z0-9_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert sorted(_lib.EXPORTS) == declared_functions()


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    raw = ctypes.CDLL(_lib.library_path(build=False))
    for name in declared_functions():
        assert getattr(raw, name) is not None


def test_every_export_has_a_ctypes_signature():
    lib = _lib.load()
    for name in _lib.EXPORTS:
        assert getattr(lib, name).argtypes is not None, name


def test_effective_stiffness_rejects_null_arguments():
    lib = _lib.load()
    out = (ctypes.c_double * 36)()
    lame = (_lib.Lame * 1)(_lib.Lame(1.0, 0.5))
    assert lib.bfcs_effective_stiffness(None, None, 1, lame, _lib.Lame(1.0, 0.5), 1e-6, 10, out, None,
                                        None) == _lib.ERR_INVALID_ARG


def test_status_strings_without_gpu():
    lib = _lib.load()
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7):
        assert len(lib.bfcs_status_string(code)) > 0


def test_invalid_plan_rejected_before_any_device_work():
    lib = _lib.load()
    h = ctypes.c_void_p()
    assert lib.bfcs_plan_create(ctypes.byref(h), 30, 32, 32, 1, 0, None) == _lib.ERR_INVALID_ARG  # odd/unsupported
    assert lib.bfcs_plan_create(ctypes.byref(h), 32, 32, 31, 1, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.bfcs_plan_create(ctypes.byref(h), 32, 32, 32, 0, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.bfcs_plan_create(ctypes.byref(h), 32, 32, 32, 65, 0, None) == _lib.ERR_INVALID_ARG  # > 64 members
    assert lib.bfcs_plan_create(None, 32, 32, 32, 1, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.bfcs_plan_create(ctypes.byref(h), 32, 32, 32, 1, 128, None) == _lib.ERR_INVALID_ARG  # unknown flag
    # conjugate gradients of Algorithm 2 and of Algorithm 3 exclude each other
    assert lib.bfcs_plan_create(ctypes.byref(h), 32, 32, 32, 1, _lib.CG | _lib.CD, None) == _lib.ERR_INVALID_ARG
    assert lib.bfcs_plan_create(ctypes.byref(h), 32, 32, 32, 1, 3, None) == _lib.ERR_INVALID_ARG  # no precision 3
    assert lib.bfcs_plan_tuning(None, None, None, None, None) == _lib.ERR_INVALID_ARG


def test_sweep_step_entry_points_reject_bad_arguments():
    lib = _lib.load()
    lame = (_lib.Lame * 1)(_lib.Lame(1.0, 0.5))
    E = (ctypes.c_double * 6)()
    n = ctypes.c_longlong()
    assert lib.bfcs_polarize(None, None, 1, lame, _lib.Lame(1.0, 0.5), None, None) == _lib.ERR_INVALID_ARG
    assert lib.bfcs_green_apply(None, _lib.Lame(1.0, 0.5), E, None, None, None, None) == _lib.ERR_INVALID_ARG
    assert lib.bfcs_profile_green_io(None, ctypes.byref(n), ctypes.byref(n)) == _lib.ERR_INVALID_ARG


def test_network_parameter_count_and_invalid_contexts():
    from oracle import unet_oracle as U
    lib = _lib.load()
    assert lib.bfcs_net_param_count() == U.param_count() == _lib.NET_PARAMS
    h = ctypes.c_void_p()
    assert lib.bfcs_net_create(ctypes.byref(h), 12, 16, 16, 1, 0, None) == _lib.ERR_INVALID_ARG  # not /8
    assert lib.bfcs_net_create(ctypes.byref(h), 16, 16, 16, 0, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.bfcs_net_create(ctypes.byref(h), 16, 16, 16, 1, 4, None) == _lib.ERR_INVALID_ARG  # flags
    assert lib.bfcs_net_create(None, 16, 16, 16, 1, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.bfcs_net_destroy(None) == _lib.ERR_INVALID_ARG


def test_new_entry_points_reject_bad_arguments_before_device_work():
    lib = _lib.load()
    lame = (_lib.Lame * 2)(_lib.Lame(1.0, 0.5), _lib.Lame(6.0, 3.0))
    c0 = _lib.Lame(3.5, 1.75)
    out = (ctypes.c_double * 64)()
    centre = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    cfg = (ctypes.c_void_p * 1)(None)
    assert lib.bfcs_radial_profile(None, None, 6, centre, 4, out, None) == _lib.ERR_INVALID_ARG
    assert lib.bfcs_ensemble_average(None, 1, cfg, 2, lame, c0, None, out, 1e-6, 10, None, None, None) == \
        _lib.ERR_INVALID_ARG
    assert lib.bfcs_kernel_fit(None, 1, cfg, cfg, 2.0, 3, 0.0, 10, 0.01, out, None, None, None, None) == \
        _lib.ERR_INVALID_ARG
    assert lib.bfcs_kernel_apply(None, 3, out, 2.0, None, None) == _lib.ERR_INVALID_ARG
    rec = (_lib.RveRecord * 2)()
    acc = ctypes.c_int(7)
    sph = (ctypes.c_int32 * 5)(8, 8, 8, 25, 1)
    sizes = (ctypes.c_int * 2)(16, 20)                     # 20 is not a whole number of 8^3 cells
    assert lib.bfcs_rve_size(8, 8, 8, 1, sph, 2, lame, c0, 3.0, 2, sizes, 0, 1e-6, 100, 0.05, rec, None,
                             ctypes.byref(acc), None) == _lib.ERR_INVALID_ARG
    sizes_ok = (ctypes.c_int * 2)(16, 24)
    for a, tol_f in ((0.0, 0.05), (3.0, 0.0), (-1.0, 0.05)):  # support radius and field tolerance must be positive
        assert lib.bfcs_rve_size(8, 8, 8, 1, sph, 2, lame, c0, a, 2, sizes_ok, 0, 1e-6, 100, tol_f, rec, None,
                                 ctypes.byref(acc), None) == _lib.ERR_INVALID_ARG


# the four-step split L = R1 R2 of every supported line length (the first radix
# runs first; the y passes' swapped variants run R2 first)
SPLITS = {4: (2, 2), 6: (3, 2), 8: (4, 2), 12: (4, 3), 16: (4, 4), 24: (8, 3), 32: (8, 4), 48: (8, 6),
          64: (8, 8), 96: (16, 6), 128: (16, 8), 192: (16, 12), 256: (16, 16)}


def test_twiddle_tables_hold_the_factored_stage_one_blocks():
    """The table a plan uploads (host-only call): W^j for j < n, then one block per
    distinct first radix r (r % 4 == 0, r >= 8) read by the transform's first step
    as block[entry][n2]: every value read there, at the offset the device computes,
    is inside the table and equals W^((n2 b) mod n) or W^((4 n2 a) mod n) bit for
    bit (the same entries of the plain table)."""
    import numpy as np
    lib = _lib.load()
    for n, (r1, r2) in SPLITS.items():
        for prec, dt, tol in ((_lib.FP32, np.float32, 2e-7), (_lib.FP64, np.float64, 2e-15)):
            cnt = lib.bfcs_twiddles(n, prec, None, 0)
            buf = np.zeros(2 * cnt, dtype=dt)
            assert lib.bfcs_twiddles(n, prec, buf.ctypes.data, cnt) == cnt
            tab = buf[0::2].astype(np.float64) + 1j * buf[1::2].astype(np.float64)
            j = np.arange(n)
            assert np.abs(tab[:n] - np.exp(-2j * np.pi * j / n)).max() <= tol, (n, prec)

            def block(r):
                return (r // 4 + 2) * (n // r) if r % 4 == 0 and r >= 8 else 0

            expect = n + block(r1) + (block(r2) if r2 != r1 else 0)
            assert cnt == expect, (n, prec, cnt, expect)
            for r in (r1, r2):
                if block(r) == 0:
                    continue
                off = n + (0 if r == r1 else block(r1))            # the device's offset rule
                n2s = n // r
                assert off + block(r) <= cnt, (n, r)
                for n2 in range(n2s):
                    for b in (1, 2, 3):
                        assert tab[off + (b - 1) * n2s + n2] == tab[(n2 * b) % n], (n, r, n2, b)
                    for a in range(1, r // 4):
                        assert tab[off + (a + 2) * n2s + n2] == tab[(4 * n2 * a) % n], (n, r, n2, a)
    assert lib.bfcs_twiddles(10, _lib.FP32, None, 0) == _lib.ERR_INVALID_ARG
    assert lib.bfcs_twiddles(256, 7, None, 0) == _lib.ERR_INVALID_ARG


def test_float_float_twiddle_tables_hold_the_stage_one_block():
    """The ladder's float-float table (host-only call): W^j for j < n to float-float
    accuracy, then the block [k1 - 1][n2] that the transform's first step reads, at
    the offset n, equal bit for bit to the plain entries W^((n2 k1) mod n)."""
    import numpy as np
    lib = _lib.load()
    for n, (r1, _) in SPLITS.items():
        cnt = lib.bfcs_twiddles(n, _lib.MIXED, None, 0)
        assert cnt == n + (r1 - 1) * (n // r1), (n, cnt)
        buf = np.zeros(4 * cnt, dtype=np.float32)
        assert lib.bfcs_twiddles(n, _lib.MIXED, buf.ctypes.data, cnt) == cnt
        q = buf.reshape(cnt, 4).astype(np.float64)
        tab = (q[:, 0] + q[:, 1]) + 1j * (q[:, 2] + q[:, 3])
        j = np.arange(n)
        assert np.abs(tab[:n] - np.exp(-2j * np.pi * j / n)).max() <= 1e-14, n
        raw = buf.reshape(cnt, 4)
        n2s = n // r1
        for k1 in range(1, r1):
            for n2 in range(n2s):
                assert np.array_equal(raw[n + (k1 - 1) * n2s + n2], raw[(n2 * k1) % n]), (n, k1, n2)


def test_plan_options_are_checked_before_any_device_work():
    """Unknown precisions and Krylov options, and CG together with Algorithm 3
    (the library rejects BFCS_CG | BFCS_CD too), fail in the binding with a
    ValueError before a stream or a device is touched."""
    import pytest
    from paper_2601_00822_gb300 import api
    with pytest.raises(ValueError):
        api.Plan((16, 16, 16), "fp16")
    with pytest.raises(ValueError):
        api.Plan((16, 16, 16), "fp32", cd="jacobi")
    with pytest.raises(ValueError):
        api.Plan((16, 16, 16), "fp32", cg=True, cd="g0")
