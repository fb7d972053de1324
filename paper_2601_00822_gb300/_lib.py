"""ctypes loader of libbfcs.so with the C-ABI signatures of include/bfcs.h.

The library is built in-tree on first use (paper_2601_00822_gb300/_build).
There is no fallback: if the library cannot be built or loaded, load() raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_LOCK = threading.Lock()
_LIB = None

OK = 0
NOT_CONVERGED = 1
ERR_INVALID_ARG = -1
ERR_NONZERO_MEAN = -2
ERR_OOM = -3
ERR_CUDA = -4
ERR_TIMEOUT = -5
ERR_DIVERGED = -6
ERR_UNSUPPORTED = -7
FP32 = 0
FP64 = 1
MIXED = 2
AUTOTUNE = 4
CG = 8
SPARSE_RESID = 16
CD = 32
CD_PRECOND = 64

# every symbol declared in include/bfcs.h
EXPORTS = (
    "bfcs_plan_create", "bfcs_plan_destroy", "bfcs_voxelize", "bfcs_body_force", "bfcs_solve",
    "bfcs_solve_batched", "bfcs_translate_average", "bfcs_surrogate_infer", "bfcs_fft3d",
    "bfcs_last_history", "bfcs_status_string", "bfcs_kernel_launches", "bfcs_profile_kernel",
    "bfcs_profile_read", "bfcs_body_force_noalloc", "bfcs_net_param_count", "bfcs_net_create",
    "bfcs_net_destroy", "bfcs_net_prepare", "bfcs_net_forward", "bfcs_net_grad", "bfcs_net_adam",
    "bfcs_net_train_step", "bfcs_net_predict", "bfcs_plan_tuning", "bfcs_solve_group", "bfcs_net_status",
    "bfcs_effective_stiffness", "bfcs_ensemble_average", "bfcs_radial_profile", "bfcs_rve_size",
    "bfcs_kernel_fit", "bfcs_kernel_apply", "bfcs_polarize", "bfcs_green_apply", "bfcs_profile_green_io",
    "bfcs_twiddles",
)
NET_PARAMS = 523654
NET_TRAIN = 1


class Lame(C.Structure):
    _fields_ = [("lam", C.c_double), ("mu", C.c_double)]


class Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("resid", C.c_double),
                ("resid_prev", C.c_double), ("precision_path", C.c_int), ("stalled", C.c_int),
                ("ms", C.c_double)]


class Problem(C.Structure):
    _fields_ = [("phase", C.c_void_p), ("b", C.c_void_p), ("E", C.c_double * 6),
                ("shift", C.c_int * 3), ("eps_init", C.c_void_p), ("eps_out", C.c_void_p),
                ("sig_out", C.c_void_p), ("u_out", C.c_void_p)]


class RveRecord(C.Structure):
    _fields_ = [("n", C.c_int), ("r_rve", C.c_int), ("contained", C.c_int), ("iters", C.c_int),
                ("status", C.c_int), ("centre", C.c_double * 3), ("resid", C.c_double), ("eps_max", C.c_double),
                ("sig_max", C.c_double)]


class GroupItem(C.Structure):
    _fields_ = [("plan", C.c_void_p), ("batch", C.c_int), ("problems", C.POINTER(Problem)),
                ("infos", C.POINTER(Info))]


def _declare(lib):
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    lib.bfcs_plan_create.argtypes = [C.POINTER(vp), i, i, i, i, i, vp]
    lib.bfcs_plan_destroy.argtypes = [vp]
    lib.bfcs_voxelize.argtypes = [i, i, i, i, i, i, i, vp, vp, vp]
    lib.bfcs_body_force.argtypes = [i, i, i, d, d, d, d, i, vp, vp]
    lib.bfcs_body_force_noalloc.argtypes = [i, i, i, d, d, d, d, i, vp, vp]
    lib.bfcs_solve.argtypes = [vp, vp, i, C.POINTER(Lame), Lame, vp, C.POINTER(d), d, i, vp, vp, vp,
                               vp, C.POINTER(Info)]
    lib.bfcs_solve_batched.argtypes = [vp, i, C.POINTER(Problem), i, C.POINTER(Lame), Lame, d, i,
                                       C.POINTER(Info)]
    lib.bfcs_translate_average.argtypes = [vp, vp, i, C.POINTER(Lame), Lame, vp, C.POINTER(d), i, vp,
                                           d, i, vp, vp, C.POINTER(Info)]
    lib.bfcs_surrogate_infer.argtypes = [vp, vp, vp, vp, i, C.POINTER(Lame), vp]
    lib.bfcs_fft3d.argtypes = [vp, i, i, vp, vp]
    lib.bfcs_polarize.argtypes = [vp, vp, i, C.POINTER(Lame), Lame, vp, vp]
    lib.bfcs_green_apply.argtypes = [vp, Lame, C.POINTER(d), vp, vp, vp, vp]
    lib.bfcs_last_history.argtypes = [vp, C.POINTER(d), i]
    lib.bfcs_twiddles.argtypes = [i, i, vp, i]
    lib.bfcs_kernel_launches.argtypes = []
    lib.bfcs_profile_kernel.argtypes = [vp, i]
    lib.bfcs_profile_read.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(d)]
    lib.bfcs_profile_green_io.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    ll, f = C.c_longlong, C.c_float
    lib.bfcs_net_param_count.argtypes = []
    lib.bfcs_net_create.argtypes = [C.POINTER(vp), i, i, i, i, i, vp]
    lib.bfcs_net_destroy.argtypes = [vp]
    lib.bfcs_net_status.argtypes = [vp]
    lib.bfcs_net_prepare.argtypes = [vp, i, vp, vp, i, C.POINTER(Lame), vp, vp, vp]
    lib.bfcs_net_forward.argtypes = [vp, vp, i, vp, vp]
    lib.bfcs_net_grad.argtypes = [vp, vp, i, vp, vp, vp, vp]
    lib.bfcs_net_adam.argtypes = [vp, vp, vp, vp, vp, ll, f]
    lib.bfcs_net_train_step.argtypes = [vp, vp, vp, vp, vp, ll, f, i, vp, vp, vp]
    lib.bfcs_net_predict.argtypes = [vp, vp, i, i, C.POINTER(vp), C.POINTER(vp), i, C.POINTER(Lame),
                                     C.POINTER(vp)]
    lib.bfcs_solve_group.argtypes = [i, C.POINTER(GroupItem), i, C.POINTER(Lame), Lame, d, i]
    lib.bfcs_plan_tuning.argtypes = [vp, C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(d)]
    lib.bfcs_ensemble_average.argtypes = [vp, i, C.POINTER(vp), i, C.POINTER(Lame), Lame, vp, C.POINTER(d), d, i,
                                         vp, vp, C.POINTER(Info)]
    lib.bfcs_radial_profile.argtypes = [vp, vp, i, C.POINTER(d), i, vp, vp]
    lib.bfcs_rve_size.argtypes = [i, i, i, i, vp, i, C.POINTER(Lame), Lame, d, i, vp, i, d, i, d,
                                  C.POINTER(RveRecord), vp, C.POINTER(i), vp]
    lib.bfcs_kernel_fit.argtypes = [vp, i, C.POINTER(vp), C.POINTER(vp), d, i, d, i, d, vp, vp, vp, vp, vp]
    lib.bfcs_kernel_apply.argtypes = [vp, i, C.POINTER(d), d, vp, vp]
    lib.bfcs_effective_stiffness.argtypes = [vp, vp, i, C.POINTER(Lame), Lame, d, i, vp, vp, C.POINTER(Info)]
    lib.bfcs_status_string.argtypes = [i]
    lib.bfcs_status_string.restype = C.c_char_p
    for name in EXPORTS:
        if name != "bfcs_status_string":
            getattr(lib, name).restype = C.c_int
    lib.bfcs_kernel_launches.restype = C.c_longlong
    lib.bfcs_net_param_count.restype = C.c_longlong
    return lib


def library_path(build: bool = True) -> str:
    from . import build as _build
    if build:
        return _build.build()
    return _build.LIB_PATH


def load(build: bool = True):
    """Build (if needed) and dlopen libbfcs.so; raises if anything is missing."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = library_path(build)
            if not os.path.exists(path):
                raise RuntimeError(f"libbfcs.so not found at {path}; run the build first")
            _LIB = _declare(C.CDLL(path, mode=C.RTLD_GLOBAL))
        return _LIB


def status_string(code: int) -> str:
    return load().bfcs_status_string(code).decode()


class BfcsError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: status {code} ({status_string(code)})")


def check(code: int, what: str, allow=(OK,)) -> int:
    if code not in allow:
        raise BfcsError(code, what)
    return code
