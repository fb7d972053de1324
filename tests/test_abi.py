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
    assert lib.bfcs_plan_create(None, 32, 32, 32, 1, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.bfcs_plan_create(ctypes.byref(h), 32, 32, 32, 1, 16, None) == _lib.ERR_INVALID_ARG  # unknown flag
    assert lib.bfcs_plan_create(ctypes.byref(h), 32, 32, 32, 1, 3, None) == _lib.ERR_INVALID_ARG  # no precision 3
    assert lib.bfcs_plan_tuning(None, None, None, None, None) == _lib.ERR_INVALID_ARG


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
