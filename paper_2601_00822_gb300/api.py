"""Thin Python binding of the C ABI (include/bfcs.h).

Only argument marshalling lives here: torch tensors supply device memory and
the current CUDA stream; every step of the solver runs in libbfcs.so.
Field tensors are contiguous, shaped (components, nz, ny, nx), float32 for
'fp32' plans and float64 for 'fp64' and 'mixed' plans.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _check_tensor(t, shape, dtype, what):
    if t is None:
        return
    if not t.is_cuda or t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{what}: need a contiguous CUDA tensor {tuple(shape)} {dtype}, got "
                         f"{tuple(t.shape)} {t.dtype} on {t.device}")


def _lames(phases):
    arr = (_lib.Lame * len(phases))()
    for i, (lam, mu) in enumerate(phases):
        arr[i].lam, arr[i].mu = float(lam), float(mu)
    return arr


@dataclass
class SolveInfo:
    iters: int
    status: int
    resid: float
    resid_prev: float
    precision_path: int
    ms: float
    stalled: int = 0

    @staticmethod
    def of(info: _lib.Info) -> "SolveInfo":
        return SolveInfo(info.iters, info.status, info.resid, info.resid_prev, info.precision_path,
                         info.ms, info.stalled)


def kernel_launches() -> int:
    """bfcs_kernel_launches: kernels launched by the library so far in this process."""
    return int(_lib.load().bfcs_kernel_launches())


def voxelize(dims, cell, spheres, device="cuda", stream=None) -> torch.Tensor:
    """bfcs_voxelize: int8 phase map (nz, ny, nx) of spheres (n, 5) int32 in a periodic cell."""
    lib = _lib.load()
    nx, ny, nz = dims
    sph = np.ascontiguousarray(np.asarray(spheres, dtype=np.int32).reshape(-1, 5))
    out = torch.empty((nz, ny, nx), dtype=torch.int8, device=device)
    _lib.check(lib.bfcs_voxelize(nx, ny, nz, cell[0], cell[1], cell[2], sph.shape[0],
                                 sph.ctypes.data_as(C.c_void_p), _ptr(out), _stream_ptr(stream)),
               "bfcs_voxelize")
    return out


def body_force(dims, centre, a, precision="fp32", device="cuda", stream=None) -> torch.Tensor:
    """bfcs_body_force: mean-free BFCS field (3, nz, ny, nx)."""
    lib = _lib.load()
    nx, ny, nz = dims
    dt = torch.float32 if precision == "fp32" else torch.float64
    out = torch.empty((3, nz, ny, nx), dtype=dt, device=device)
    flag = _lib.FP32 if precision == "fp32" else _lib.FP64
    _lib.check(lib.bfcs_body_force(nx, ny, nz, float(centre[0]), float(centre[1]), float(centre[2]),
                                   float(a), flag, _ptr(out), _stream_ptr(stream)), "bfcs_body_force")
    return out


class Plan:
    """bfcs_plan_create / bfcs_plan_destroy with the solver calls as methods."""

    def __init__(self, dims, precision="fp32", max_batch=1, stream=None, autotune=False, cg=False,
                 sparse_resid=False, cd=None):
        """cd: None, or the displacement-based CG of Algorithm 3: "plain" (as printed,
        BFCS_CD) or "g0" (preconditioned by the reference medium's G0, BFCS_CD_PRECOND)."""
        precisions = {"fp32": _lib.FP32, "fp64": _lib.FP64, "mixed": _lib.MIXED}
        if precision not in precisions:
            raise ValueError(f"precision must be one of {sorted(precisions)}, not {precision!r}")
        if cd not in (None, "plain", "g0"):
            raise ValueError(f"cd must be None, 'plain' or 'g0', not {cd!r}")
        if cd is not None and cg:
            raise ValueError("cg (Algorithm 2) and cd (Algorithm 3) exclude each other")
        self.lib = _lib.load()
        self.dims = tuple(int(d) for d in dims)
        self.precision = precision
        self.dtype = torch.float32 if precision == "fp32" else torch.float64
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        flag = precisions[precision]
        if autotune:
            flag |= _lib.AUTOTUNE
        if cg:
            flag |= _lib.CG
        if sparse_resid:
            flag |= _lib.SPARSE_RESID
        if cd is not None:
            flag |= {"plain": _lib.CD, "g0": _lib.CD_PRECOND}[cd]
        nx, ny, nz = self.dims
        _lib.check(self.lib.bfcs_plan_create(C.byref(h), nx, ny, nz, int(max_batch), flag,
                                             _stream_ptr(self.stream)), "bfcs_plan_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.bfcs_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _shape(self, ncomp):
        nx, ny, nz = self.dims
        return (ncomp, nz, ny, nx)

    def _alloc(self, ncomp):
        return torch.empty(self._shape(ncomp), dtype=self.dtype, device="cuda")

    def solve(self, phase, phases, c0, b, E=(0.0,) * 6, tol=1e-6, maxit=10000, eps_init=None,
              eps_out=None, sig_out=None, u_out=None, want_sig=True, want_u=True,
              allow=(_lib.OK, _lib.NOT_CONVERGED)):
        """bfcs_solve; returns (eps, sig or None, u or None, SolveInfo)."""
        nx, ny, nz = self.dims
        _check_tensor(phase, (nz, ny, nx), torch.int8, "phase")
        _check_tensor(b, self._shape(3), self.dtype, "b")
        _check_tensor(eps_init, self._shape(6), self.dtype, "eps_init")
        eps_out = eps_out if eps_out is not None else self._alloc(6)
        if sig_out is None and want_sig:
            sig_out = self._alloc(6)
        if u_out is None and want_u:
            u_out = self._alloc(3)
        for t, n, w in ((eps_out, 6, "eps_out"), (sig_out, 6, "sig_out"), (u_out, 3, "u_out")):
            _check_tensor(t, self._shape(n), self.dtype, w)
        lam = _lames(phases)
        e = (C.c_double * 6)(*[float(v) for v in E])
        info = _lib.Info()
        code = self.lib.bfcs_solve(self.handle, _ptr(phase), len(phases), lam, _lib.Lame(*c0), _ptr(b), e,
                                   float(tol), int(maxit), _ptr(eps_init), _ptr(eps_out), _ptr(sig_out),
                                   _ptr(u_out), C.byref(info))
        _lib.check(code, "bfcs_solve", allow)
        return eps_out, sig_out, u_out, SolveInfo.of(info)

    def solve_batched(self, members, phases, c0, tol=1e-6, maxit=10000,
                      allow=(_lib.OK, _lib.NOT_CONVERGED)):
        """bfcs_solve_batched; members: list of dicts with phase, b, E, shift, eps_init,
        eps_out, sig_out, u_out (outputs allocated when missing). Returns (members, infos)."""
        n = len(members)
        arr = (_lib.Problem * n)()
        for m, mem in enumerate(members):
            mem.setdefault("eps_out", self._alloc(6))
            for key, comp in (("sig_out", 6), ("u_out", 3)):
                if key not in mem:
                    mem[key] = self._alloc(comp)
            arr[m].phase = mem["phase"].data_ptr()
            arr[m].b = mem["b"].data_ptr()
            arr[m].E = (C.c_double * 6)(*[float(v) for v in mem.get("E", (0.0,) * 6)])
            arr[m].shift = (C.c_int * 3)(*[int(v) for v in mem.get("shift", (0, 0, 0))])
            arr[m].eps_init = mem["eps_init"].data_ptr() if mem.get("eps_init") is not None else None
            arr[m].eps_out = mem["eps_out"].data_ptr()
            arr[m].sig_out = mem["sig_out"].data_ptr() if mem["sig_out"] is not None else None
            arr[m].u_out = mem["u_out"].data_ptr() if mem["u_out"] is not None else None
        infos = (_lib.Info * max(n, 1))()
        code = self.lib.bfcs_solve_batched(self.handle, n, arr, len(phases), _lames(phases),
                                           _lib.Lame(*c0), float(tol), int(maxit), infos)
        _lib.check(code, "bfcs_solve_batched", allow)
        return members, [SolveInfo.of(infos[m]) for m in range(n)]

    def _problems(self, members):
        n = len(members)
        arr = (_lib.Problem * n)()
        for m, mem in enumerate(members):
            mem.setdefault("eps_out", self._alloc(6))
            for key, comp in (("sig_out", 6), ("u_out", 3)):
                if key not in mem:
                    mem[key] = self._alloc(comp)
            arr[m].phase = mem["phase"].data_ptr()
            arr[m].b = mem["b"].data_ptr()
            arr[m].E = (C.c_double * 6)(*[float(v) for v in mem.get("E", (0.0,) * 6)])
            arr[m].shift = (C.c_int * 3)(*[int(v) for v in mem.get("shift", (0, 0, 0))])
            arr[m].eps_init = mem["eps_init"].data_ptr() if mem.get("eps_init") is not None else None
            arr[m].eps_out = mem["eps_out"].data_ptr()
            arr[m].sig_out = mem["sig_out"].data_ptr() if mem["sig_out"] is not None else None
            arr[m].u_out = mem["u_out"].data_ptr() if mem["u_out"] is not None else None
        return arr

    def translate_average(self, phase, phases, c0, b, shifts, E=(0.0,) * 6, tol=1e-6, maxit=10000,
                          allow=(_lib.OK, _lib.NOT_CONVERGED)):
        """bfcs_translate_average; returns (avg (30, nz, ny, nx) float64, hits int32, infos)."""
        nx, ny, nz = self.dims
        sh = np.ascontiguousarray(np.asarray(shifts, dtype=np.int32).reshape(-1, 3))
        avg = torch.empty((30, nz, ny, nx), dtype=torch.float64, device="cuda")
        hits = torch.empty((nz, ny, nx), dtype=torch.int32, device="cuda")
        infos = (_lib.Info * sh.shape[0])()
        e = (C.c_double * 6)(*[float(v) for v in E])
        code = self.lib.bfcs_translate_average(self.handle, _ptr(phase), len(phases), _lames(phases),
                                               _lib.Lame(*c0), _ptr(b), e, sh.shape[0],
                                               sh.ctypes.data_as(C.c_void_p), float(tol), int(maxit),
                                               _ptr(avg), _ptr(hits), infos)
        _lib.check(code, "bfcs_translate_average", allow)
        return avg, hits, [SolveInfo.of(infos[m]) for m in range(sh.shape[0])]

    def ensemble_average(self, configs, phases, c0, b, E=(0.0,) * 6, tol=1e-6, maxit=10000,
                         allow=(_lib.OK, _lib.NOT_CONVERGED)):
        """bfcs_ensemble_average (Eq. 3.8); returns (avg (30, nz, ny, nx) float64, hits int32, infos)."""
        nx, ny, nz = self.dims
        for ph in configs:
            _check_tensor(ph, (nz, ny, nx), torch.int8, "configs[j]")
        ptrs = (C.c_void_p * len(configs))(*[_ptr(ph) for ph in configs])
        avg = torch.empty((30, nz, ny, nx), dtype=torch.float64, device="cuda")
        hits = torch.empty((nz, ny, nx), dtype=torch.int32, device="cuda")
        infos = (_lib.Info * len(configs))()
        e = (C.c_double * 6)(*[float(v) for v in E])
        code = self.lib.bfcs_ensemble_average(self.handle, len(configs), ptrs, len(phases), _lames(phases),
                                              _lib.Lame(*c0), _ptr(b), e, float(tol), int(maxit), _ptr(avg),
                                              _ptr(hits), infos)
        _lib.check(code, "bfcs_ensemble_average", allow)
        return avg, hits, [SolveInfo.of(infos[m]) for m in range(len(configs))]

    def radial_profile(self, field, centre, nbins):
        """bfcs_radial_profile: (shell maxima of the pointwise norm (nbins,), voxel counts (nbins,))."""
        nx, ny, nz = self.dims
        if field.shape[0] not in (3, 6):
            raise ValueError("field: 3 (vector) or 6 (symmetric tensor) components")
        _check_tensor(field, (field.shape[0], nz, ny, nx), self.dtype, "field")
        prof = np.zeros(int(nbins))
        counts = np.zeros(int(nbins), dtype=np.int64)
        c = (C.c_double * 3)(*[float(v) for v in centre])
        _lib.check(self.lib.bfcs_radial_profile(self.handle, _ptr(field), int(field.shape[0]), c, int(nbins),
                                                prof.ctypes.data_as(C.c_void_p), counts.ctypes.data_as(C.c_void_p)),
                   "bfcs_radial_profile")
        return prof, counts

    def kernel_fit(self, us, gammas, delta, degree, lam=0.0, iters=2000, lr=0.05):
        """bfcs_kernel_fit (Eqs. 6.5-6.6): dict(coef (Adam), exact, loss, exact_loss, G, g)."""
        nx, ny, nz = self.dims
        for t in list(us) + list(gammas):
            _check_tensor(t, (3, nz, ny, nx), torch.float64, "u / gamma")
        if len(us) != len(gammas) or not us:
            raise ValueError("one gamma per u")
        nb = int(degree) + 1
        pu = (C.c_void_p * len(us))(*[_ptr(t) for t in us])
        pg = (C.c_void_p * len(gammas))(*[_ptr(t) for t in gammas])
        coef, exact, loss = np.zeros(nb), np.zeros(nb), np.zeros(2)
        G, g = np.zeros((nb, nb)), np.zeros(nb)
        _lib.check(self.lib.bfcs_kernel_fit(self.handle, len(us), pu, pg, float(delta), int(degree), float(lam),
                                            int(iters), float(lr), coef.ctypes.data_as(C.c_void_p),
                                            exact.ctypes.data_as(C.c_void_p), loss.ctypes.data_as(C.c_void_p),
                                            G.ctypes.data_as(C.c_void_p), g.ctypes.data_as(C.c_void_p)),
                   "bfcs_kernel_fit")
        return dict(coef=coef, exact=exact, loss=loss[0], exact_loss=loss[1], G=G, g=g)

    def kernel_apply(self, coef, delta, u):
        """bfcs_kernel_apply: L[u] (3, nz, ny, nx) float64 for Bernstein coefficients coef."""
        nx, ny, nz = self.dims
        _check_tensor(u, (3, nz, ny, nx), torch.float64, "u")
        c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64))
        out = torch.empty_like(u)
        _lib.check(self.lib.bfcs_kernel_apply(self.handle, c.size - 1, c.ctypes.data_as(C.POINTER(C.c_double)),
                                              float(delta), _ptr(u), _ptr(out)), "bfcs_kernel_apply")
        return out

    def effective_stiffness(self, phase, phases, c0, tol=1e-6, maxit=10000,
                            allow=(_lib.OK, _lib.NOT_CONVERGED)):
        """bfcs_effective_stiffness: (L* (6, 6), A* (6, 6), infos) with column J the
        response to the unit tensorial mean strain J (Eqs. 6.1-6.3, 3.2)."""
        _check_tensor(phase, (self.dims[2], self.dims[1], self.dims[0]), torch.int8, "phase")
        ls = np.zeros(36)
        as_ = np.zeros(36)
        infos = (_lib.Info * 6)()
        code = self.lib.bfcs_effective_stiffness(self.handle, _ptr(phase), len(phases), _lames(phases),
                                                 _lib.Lame(*c0), float(tol), int(maxit),
                                                 ls.ctypes.data_as(C.c_void_p),
                                                 as_.ctypes.data_as(C.c_void_p), infos)
        _lib.check(code, "bfcs_effective_stiffness", allow)
        return ls.reshape(6, 6), as_.reshape(6, 6), [SolveInfo.of(infos[m]) for m in range(6)]

    def polarize(self, phase, phases, c0, eps, tau=None):
        """bfcs_polarize: tau = (L(x) - L0) : eps (Eq. 5.7); returns tau (6 x N)."""
        _check_tensor(eps, self._shape(6), self.dtype, "eps")
        tau = tau if tau is not None else self._alloc(6)
        _check_tensor(tau, self._shape(6), self.dtype, "tau")
        nx, ny, nz = self.dims
        _check_tensor(phase, (nz, ny, nx), torch.int8, "phase")
        _lib.check(self.lib.bfcs_polarize(self.handle, _ptr(phase), len(phases), _lames(phases), _lib.Lame(*c0),
                                          _ptr(eps), _ptr(tau)), "bfcs_polarize")
        return tau

    def green_apply(self, c0, b_hat, spec, E=(0.0,) * 6, d_prev=None, num_out=None):
        """bfcs_green_apply on a dense half spectrum (ncomp, nz, ny, nx//2 + 1),
        complex, in place: tau_hat -> eps_hat^{s+1} (unnormalised); with d_prev
        (3 components) and num_out (one float64) also the residual numerator."""
        nx, ny, nz = self.dims
        cdt = torch.complex64 if self.dtype == torch.float32 else torch.complex128
        _check_tensor(spec, (6, nz, ny, nx // 2 + 1), cdt, "spec")
        _check_tensor(b_hat, (3, nz, ny, nx // 2 + 1), cdt, "b_hat")
        _check_tensor(d_prev, (3, nz, ny, nx // 2 + 1), cdt, "d_prev")
        _check_tensor(num_out, (1,), torch.float64, "num_out")
        e = (C.c_double * 6)(*[float(v) for v in E])
        _lib.check(self.lib.bfcs_green_apply(self.handle, _lib.Lame(*c0), e, _ptr(b_hat), _ptr(spec), _ptr(d_prev),
                                             _ptr(num_out)), "bfcs_green_apply")
        return spec

    def fft3d(self, x, direction=-1):
        """bfcs_fft3d: forward real (c, nz, ny, nx) -> complex (c, nz, ny, nx/2+1) or back
        (inverse without the 1/N factor)."""
        nx, ny, nz = self.dims
        if direction < 0:
            c = x.shape[0]
            _check_tensor(x, self._shape(c), self.dtype, "x")
            cdt = torch.complex128 if self.dtype == torch.float64 else torch.complex64
            out = torch.empty((c, nz, ny, nx // 2 + 1), dtype=cdt, device="cuda")
        else:
            c = x.shape[0]
            out = self._alloc(c)
        _lib.check(self.lib.bfcs_fft3d(self.handle, int(direction), int(c), _ptr(x), _ptr(out)),
                   "bfcs_fft3d")
        return out

    def profile(self, kind):
        """bfcs_profile_kernel: 0 off, 1 x pass, 2 y passes, 3 fused z/Green pass."""
        _lib.check(self.lib.bfcs_profile_kernel(self.handle, int(kind)), "bfcs_profile_kernel")

    def profile_read(self):
        """bfcs_profile_read: (launches timed, summed milliseconds) since the last read."""
        n = C.c_longlong()
        ms = C.c_double()
        _lib.check(self.lib.bfcs_profile_read(self.handle, C.byref(n), C.byref(ms)), "bfcs_profile_read")
        return n.value, ms.value

    def profile_green_io(self):
        """bfcs_profile_green_io: (d_prev reads, d writes) of the timed z/Green launches."""
        r = C.c_longlong()
        w = C.c_longlong()
        _lib.check(self.lib.bfcs_profile_green_io(self.handle, C.byref(r), C.byref(w)), "bfcs_profile_green_io")
        return r.value, w.value

    def history(self, cap=1 << 16):
        """bfcs_last_history: residuals r(eps^s) of the last solve."""
        buf = (C.c_double * cap)()
        n = self.lib.bfcs_last_history(self.handle, buf, cap)
        if n < 0:
            raise _lib.BfcsError(n, "bfcs_last_history")
        return np.array(buf[:n])

    def tuning(self):
        """bfcs_plan_tuning: dict(variant, tile, swap, variant_ms)."""
        v, t, sw = C.c_int(), C.c_int(), C.c_int()
        ms = (C.c_double * 8)()
        _lib.check(self.lib.bfcs_plan_tuning(self.handle, C.byref(v), C.byref(t), C.byref(sw), ms),
                   "bfcs_plan_tuning")
        return {"variant": v.value, "tile": t.value, "swap": bool(sw.value), "variant_ms": list(ms)}

    def surrogate_infer(self, weights, b, phase, phases, eps_out=None):
        """bfcs_surrogate_infer: the network's strain prediction (6, nz, ny, nx) on this plan's grid."""
        _check_tensor(weights, (_lib.NET_PARAMS,), torch.float32, "weights")
        _check_tensor(b, self._shape(3), self.dtype, "b")
        _check_tensor(phase, self._shape(1)[1:], torch.int8, "phase")
        eps = eps_out if eps_out is not None else self._alloc(6)
        _check_tensor(eps, self._shape(6), self.dtype, "eps_out")
        arr = _lames(phases)
        _lib.check(self.lib.bfcs_surrogate_infer(self.handle, _ptr(weights), _ptr(b), _ptr(phase), len(phases),
                                                 arr, _ptr(eps)), "bfcs_surrogate_infer")
        return eps


def rve_size(cell, spheres, phases, c0, a, sizes, precision="mixed", tol=1e-6, maxit=20000, tol_f=1e-3,
             stream=None, allow=(_lib.OK, _lib.NOT_CONVERGED)):
    """bfcs_rve_size (Def. 2.2, Sec. 5): returns (records as dicts, profiles (nsizes, 2, max n/2), accepted index)."""
    lib = _lib.load()
    sph = np.ascontiguousarray(np.asarray(spheres, dtype=np.int32).reshape(-1, 5))
    sz = np.ascontiguousarray(np.asarray(sizes, dtype=np.int32).reshape(-1))
    flag = {"fp32": _lib.FP32, "fp64": _lib.FP64, "mixed": _lib.MIXED}[precision]
    recs = (_lib.RveRecord * sz.size)()
    prof = np.zeros((sz.size, 2, int(sz.max()) // 2))
    acc = C.c_int(-1)
    code = lib.bfcs_rve_size(int(cell[0]), int(cell[1]), int(cell[2]), sph.shape[0], sph.ctypes.data_as(C.c_void_p),
                             len(phases), _lames(phases), _lib.Lame(*c0), float(a), int(sz.size),
                             sz.ctypes.data_as(C.c_void_p), int(flag), float(tol), int(maxit), float(tol_f), recs,
                             prof.ctypes.data_as(C.c_void_p), C.byref(acc), _stream_ptr(stream))
    _lib.check(code, "bfcs_rve_size", allow)
    out = []
    for r in recs:
        if r.n == 0:
            break
        out.append(dict(n=r.n, r_rve=(None if r.r_rve < 0 else r.r_rve), contained=bool(r.contained),
                        iters=r.iters, status=r.status, centre=tuple(r.centre), resid=r.resid,
                        eps_max=r.eps_max, sig_max=r.sig_max))
    return out, prof, acc.value


def _ptr_array(ts):
    arr = (C.c_void_p * len(ts))()
    for k, t in enumerate(ts):
        arr[k] = t.data_ptr()
    return arr


class Net:
    """bfcs_net_create / bfcs_net_destroy with the network calls as methods.

    params, grads and Adam moments are float32 CUDA tensors of NET_PARAMS
    entries (layout of include/bfcs.h); x is (batch, 4, nz, ny, nx), targets
    and outputs (batch, 6, nz, ny, nx), float32.
    """

    def __init__(self, dims, max_batch=1, train=False, stream=None):
        self.lib = _lib.load()
        self.dims = tuple(int(d) for d in dims)
        self.max_batch = int(max_batch)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        nx, ny, nz = self.dims
        _lib.check(self.lib.bfcs_net_create(C.byref(h), nx, ny, nz, self.max_batch,
                                            _lib.NET_TRAIN if train else 0, _stream_ptr(self.stream)),
                   "bfcs_net_create")
        self.handle = h

    @staticmethod
    def param_count() -> int:
        return int(_lib.load().bfcs_net_param_count())

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.bfcs_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self):
        """bfcs_net_status: raises if a network kernel gave up a bounded wait."""
        _lib.check(self.lib.bfcs_net_status(self.handle), "bfcs_net_status")

    def _vol(self, batch, ch):
        nx, ny, nz = self.dims
        return (batch, ch, nz, ny, nx)

    def prepare(self, b, phase, phases, eps=None, x_out=None, target_out=None):
        """bfcs_net_prepare: network input (4, nz, ny, nx) [and target (6, ...)] of one sample."""
        nx, ny, nz = self.dims
        prec = _lib.FP64 if b.dtype == torch.float64 else _lib.FP32
        _check_tensor(b, (3, nz, ny, nx), b.dtype, "b")
        _check_tensor(phase, (nz, ny, nx), torch.int8, "phase")
        _check_tensor(eps, (6, nz, ny, nx), b.dtype, "eps")
        x = x_out if x_out is not None else torch.empty((4, nz, ny, nx), dtype=torch.float32, device="cuda")
        t = None
        if eps is not None:
            t = target_out if target_out is not None else torch.empty((6, nz, ny, nx), dtype=torch.float32,
                                                                      device="cuda")
        _check_tensor(x, (4, nz, ny, nx), torch.float32, "x_out")
        _check_tensor(t, (6, nz, ny, nx), torch.float32, "target_out")
        arr = _lames(phases)
        _lib.check(self.lib.bfcs_net_prepare(self.handle, prec, _ptr(b), _ptr(phase), len(phases), arr,
                                             _ptr(eps), _ptr(x), _ptr(t)), "bfcs_net_prepare")
        return x if eps is None else (x, t)

    def forward(self, params, x, y=None):
        """bfcs_net_forward."""
        B = x.shape[0]
        _check_tensor(params, (_lib.NET_PARAMS,), torch.float32, "params")
        _check_tensor(x, self._vol(B, 4), torch.float32, "x")
        y = y if y is not None else torch.empty(self._vol(B, 6), dtype=torch.float32, device="cuda")
        _check_tensor(y, self._vol(B, 6), torch.float32, "y")
        _lib.check(self.lib.bfcs_net_forward(self.handle, _ptr(params), B, _ptr(x), _ptr(y)), "bfcs_net_forward")
        return y

    def grad(self, params, x, target, grad=None, loss=None):
        """bfcs_net_grad: (grad, loss) with loss a 1-element float64 CUDA tensor."""
        B = x.shape[0]
        _check_tensor(params, (_lib.NET_PARAMS,), torch.float32, "params")
        _check_tensor(x, self._vol(B, 4), torch.float32, "x")
        _check_tensor(target, self._vol(B, 6), torch.float32, "target")
        grad = grad if grad is not None else torch.empty(_lib.NET_PARAMS, dtype=torch.float32, device="cuda")
        loss = loss if loss is not None else torch.empty(1, dtype=torch.float64, device="cuda")
        _check_tensor(grad, (_lib.NET_PARAMS,), torch.float32, "grad")
        _lib.check(self.lib.bfcs_net_grad(self.handle, _ptr(params), B, _ptr(x), _ptr(target), _ptr(grad),
                                          _ptr(loss)), "bfcs_net_grad")
        return grad, loss

    def adam(self, params, grad, m, v, t, lr):
        """bfcs_net_adam: one Adam step in place on params, m, v."""
        for name, ten in (("params", params), ("grad", grad), ("m", m), ("v", v)):
            _check_tensor(ten, (_lib.NET_PARAMS,), torch.float32, name)
        _lib.check(self.lib.bfcs_net_adam(self.handle, _ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(t),
                                          float(lr)), "bfcs_net_adam")

    def train_step(self, params, grad, m, v, t, lr, x, target, loss=None):
        """bfcs_net_train_step: gradient then Adam; returns the loss tensor (device)."""
        B = x.shape[0]
        for name, ten in (("params", params), ("grad", grad), ("m", m), ("v", v)):
            _check_tensor(ten, (_lib.NET_PARAMS,), torch.float32, name)
        _check_tensor(x, self._vol(B, 4), torch.float32, "x")
        _check_tensor(target, self._vol(B, 6), torch.float32, "target")
        loss = loss if loss is not None else torch.empty(1, dtype=torch.float64, device="cuda")
        _lib.check(self.lib.bfcs_net_train_step(self.handle, _ptr(params), _ptr(grad), _ptr(m), _ptr(v),
                                                int(t), float(lr), B, _ptr(x), _ptr(target), _ptr(loss)),
                   "bfcs_net_train_step")
        return loss

    def predict(self, params, bs, phases_maps, phases, eps_out=None):
        """bfcs_net_predict: strain warm starts (6, nz, ny, nx) for lists of b and phase maps."""
        nx, ny, nz = self.dims
        B = len(bs)
        dt = bs[0].dtype
        prec = _lib.FP64 if dt == torch.float64 else _lib.FP32
        for b in bs:
            _check_tensor(b, (3, nz, ny, nx), dt, "b")
        for ph in phases_maps:
            _check_tensor(ph, (nz, ny, nx), torch.int8, "phase")
        outs = eps_out if eps_out is not None else [
            torch.empty((6, nz, ny, nx), dtype=dt, device="cuda") for _ in range(B)]
        for e in outs:
            _check_tensor(e, (6, nz, ny, nx), dt, "eps_out")
        arr = _lames(phases)
        _lib.check(self.lib.bfcs_net_predict(self.handle, _ptr(params), prec, B, _ptr_array(bs),
                                             _ptr_array(phases_maps), len(phases), arr, _ptr_array(outs)),
                   "bfcs_net_predict")
        return outs


def solve_group(groups, phases, c0, tol=1e-6, maxit=10000, allow=(_lib.OK, _lib.NOT_CONVERGED)):
    """bfcs_solve_group: groups = [(plan, members), ...] with plans of different grids (all
    'fp32' or all 'fp64'); members as for Plan.solve_batched.  Returns [(members, infos), ...]."""
    lib = _lib.load()
    n = len(groups)
    items = (_lib.GroupItem * n)()
    keep = []
    for i, (plan, members) in enumerate(groups):
        arr = plan._problems(members)
        infos = (_lib.Info * len(members))()
        keep.append((arr, infos))
        items[i].plan = plan.handle.value
        items[i].batch = len(members)
        items[i].problems = C.cast(arr, C.POINTER(_lib.Problem))
        items[i].infos = C.cast(infos, C.POINTER(_lib.Info))
    code = lib.bfcs_solve_group(n, items, len(phases), _lames(phases), _lib.Lame(*c0), float(tol), int(maxit))
    _lib.check(code, "bfcs_solve_group", allow)
    return [(members, [SolveInfo.of(infos[m]) for m in range(len(members))])
            for (plan, members), (_, infos) in zip(groups, keep)]
