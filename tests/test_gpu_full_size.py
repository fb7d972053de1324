"""Parity at the benchmarked sizes: the 256^3 sweep kernels against the FP64 oracle,
and the 128^3 batched translated averaging in its launch configuration.

At 256^3 every line of the sweep has length 256, so these are the
`k_xpass/k_colpass/k_zgreen<., 256>` instantiations in the launch configuration
bench.py times (autotuned y passes, sweeps launched from captured CUDA graphs).
The oracle runs Algorithm 1 (Eqs. 5.7-5.10) for a few sweeps on the same
seeded input; the GPU path must match it field by field at the same sweep
count (relative L2 <= 1e-10 in FP64, <= 1e-5 in FP32) and reproduce its
residual history of Eq. 5.11 (reading R4).

The converged results are compared with an all-FP64 GPU solve of the same
problem, itself checked by the oracle's own residual of the returned field.
"""
import os

import numpy as np
import pytest
import scipy.fft as sfft
import torch

from oracle import bfcs_oracle as O
from paper_2601_00822_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}
SWEEPS = 3


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _oracle_fixed(p):
    ph = O.phase_map(p.dims, p.cell, p.spheres)
    b = O.body_force(p.dims, p.bf_centre, p.bf_radius)
    # the oracle's arithmetic is unchanged; only its library FFT runs on all host cores
    with sfft.set_workers(os.cpu_count() or 1):
        ref = O.solve(ph, p.phases, p.c0, b, tol=0.0, maxit=SWEEPS, history=True)
    ref["phase"] = ph
    return ref


PROBLEMS = {
    # the bench's workload: 8^3 cells of 32^3, RSA vf 0.25, contrast 10, a = 24
    "c2_256": lambda: W.config_c2(contrast=10.0, seed=1),
    # stiff inclusions: RSA vf 0.3, Young contrast 1000 (the precision study's problem)
    "c4_256": lambda: W.config_c4(seed=1),
}
_REFS = {}


def oracle_ref(name):
    if name not in _REFS:
        _REFS.clear()                      # one 256^3 oracle result held at a time
        p = PROBLEMS[name]()
        _REFS[name] = (p, _oracle_fixed(p))
    return _REFS[name]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", sorted(PROBLEMS))
def test_full_size_fixed_sweeps_parity(name, precision, monkeypatch):
    p, ref = oracle_ref(name)
    # one sweep per captured graph, so that the three sweeps are graph launches as in the bench
    monkeypatch.setenv("BFCS_GRAPH_SWEEPS", "1")
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    assert np.array_equal(ph.cpu().numpy(), ref["phase"])
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, precision)
    t = TOL[precision]
    slack = 1e-12 if precision == "fp64" else 1e-6
    h_ref = np.array(ref["hist"])
    # the bench's plan (autotuned y passes, sparse residual evaluation) and the dense evaluation
    for sparse in (True, False):
        with api.Plan(p.dims, precision, autotune=True, sparse_resid=sparse) as plan:
            eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, tol=0.0, maxit=SWEEPS)
            hist = plan.history()
        assert info.iters == ref["sweeps"] == SWEEPS
        for got, key in ((eps, "eps"), (sig, "sig"), (u, "u")):
            err = rel(got.cpu().numpy(), ref[key])
            assert err < t, (name, precision, sparse, key, err)
        del eps, sig, u
        assert len(hist) == len(h_ref)
        ev = ~np.isnan(hist)
        assert ev[0] and (ev.all() or sparse)
        assert np.all(np.abs(hist[ev] - h_ref[ev]) <= 1e-4 * h_ref[ev] + slack), (hist, h_ref)
        assert abs(info.resid - ref["resid"]) <= 1e-3 * ref["resid"] + slack


def test_full_size_converged_error_against_fp64():
    """The bench's configuration (mixed ladder, residual 1e-6) against an all-FP64
    GPU solve converged to 1e-10, whose field the oracle's residual confirms.

    Bound: the basic scheme's error after reaching residual r is at most about
    (contrast) x r in relative terms (the operator's condition number is bounded
    by the stiffness contrast, 10 here), so 1e-6 admits an error of ~1e-5."""
    p = W.config_c2(contrast=10.0, seed=1)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp64")
    with api.Plan(p.dims, "fp64") as plan:
        e64, s64, u64, i64 = plan.solve(ph, p.phases, p.c0, b, tol=1e-10, maxit=4000)
    assert i64.status == _lib.OK and i64.resid <= 1e-10
    ph_o = O.phase_map(p.dims, p.cell, p.spheres)
    b_o = O.body_force(p.dims, p.bf_centre, p.bf_radius)
    with sfft.set_workers(os.cpu_count() or 1):
        r_ref = O.residual(ph_o, p.phases, e64.cpu().numpy(), O.fft3(b_o), O.wavevectors(p.dims))
    assert r_ref <= 1.05e-10, r_ref
    with api.Plan(p.dims, "mixed", autotune=True, sparse_resid=True) as plan:
        em, sm, um, im = plan.solve(ph, p.phases, p.c0, b, tol=p.tol, maxit=p.maxit)
    assert im.status == _lib.OK and im.resid <= p.tol
    errs = {k: rel(a.cpu().numpy(), r.cpu().numpy()) for k, a, r in (("eps", em, e64), ("sig", sm, s64),
                                                                     ("u", um, u64))}
    assert max(errs.values()) < 10.0 * 10.0 * p.tol, (errs, im.iters, i64.iters)


def test_full_size_contrast_1000_converged_against_fp64():
    """Stiff inclusions at 256^3 (RSA vf 0.3, contrast 1000): the mixed ladder with
    conjugate gradients to residual 1e-6 against an all-FP64 conjugate-gradient
    solve to 1e-9 (confirmed by the oracle's residual), for the strain, the stress
    and translated averages over two shifts.  At this contrast the condition
    number is ~1e3, so residual 1e-6 admits a relative error of ~1e-3."""
    p = W.config_c4(seed=1)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp64")
    shifts = [(0, 0, 0), (16, 8, 0)]
    with api.Plan(p.dims, "fp64", cg=True) as plan:
        e64, s64, _, i64 = plan.solve(ph, p.phases, p.c0, b, tol=1e-9, maxit=20000, want_u=False)
        a64, h64, _ = plan.translate_average(ph, p.phases, p.c0, b, shifts, tol=1e-9, maxit=20000)
    assert i64.status == _lib.OK and i64.resid <= 1e-9
    ph_o = O.phase_map(p.dims, p.cell, p.spheres)
    b_o = O.body_force(p.dims, p.bf_centre, p.bf_radius)
    with sfft.set_workers(os.cpu_count() or 1):
        r_ref = O.residual(ph_o, p.phases, e64.cpu().numpy(), O.fft3(b_o), O.wavevectors(p.dims))
    assert r_ref <= 1.05e-9, r_ref
    with api.Plan(p.dims, "mixed", cg=True) as plan:
        em, sm, _, im = plan.solve(ph, p.phases, p.c0, b, tol=1e-6, maxit=20000, want_u=False)
        am, hm, _ = plan.translate_average(ph, p.phases, p.c0, b, shifts, tol=1e-6, maxit=20000)
    assert im.status == _lib.OK and im.resid <= 1e-6
    assert torch.equal(hm, h64)
    err_e = rel(em.cpu().numpy(), e64.cpu().numpy())
    err_s = rel(sm.cpu().numpy(), s64.cpu().numpy())
    err_a = rel(am.cpu().numpy(), a64.cpu().numpy())
    assert max(err_e, err_s, err_a) < 1e-3, (err_e, err_s, err_a, im.iters, i64.iters)
    # Algorithm 3 with the G0 preconditioner inside the mixed ladder, same bound
    with api.Plan(p.dims, "mixed", cd="g0") as plan:
        ec, sc, _, ic = plan.solve(ph, p.phases, p.c0, b, tol=1e-6, maxit=20000, want_u=False)
    assert ic.status == _lib.OK and ic.resid <= 1e-6
    err_e = rel(ec.cpu().numpy(), e64.cpu().numpy())
    err_s = rel(sc.cpu().numpy(), s64.cpu().numpy())
    assert max(err_e, err_s) < 1e-3, (err_e, err_s, ic.iters)


def test_full_size_displacement_cg_iterates():
    """Algorithm 3 (G0-preconditioned, FP32) at 256^3 on the bench problem: three
    iterations against the oracle's iterates (strain, stress and displacement to
    1e-5 in relative L2, the residual history's last value to 1e-3)."""
    p = W.config_c2(contrast=10.0, seed=1)
    ph_o = O.phase_map(p.dims, p.cell, p.spheres)
    b_o = O.body_force(p.dims, p.bf_centre, p.bf_radius)
    with sfft.set_workers(os.cpu_count() or 1):
        ref = O.solve_cd(ph_o, p.phases, p.c0, b_o, tol=0.0, maxit=SWEEPS, precondition=True)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp32")
    with api.Plan(p.dims, "fp32", cd="g0") as plan:
        eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, tol=0.0, maxit=SWEEPS)
    assert info.iters == ref["iters"] == SWEEPS
    for got, key in ((eps, "eps"), (sig, "sig"), (u, "u")):
        err = rel(got.cpu().numpy(), ref[key])
        assert err < TOL["fp32"], (key, err)
    assert abs(info.resid - ref["resid"]) <= 1e-3 * ref["resid"]


def test_full_size_translated_averaging_c3():
    """C3 in the bench's launch configuration: 128^3 (8^3 cells of 16^3, one sphere
    per cell, contrast 10), the 4^3 shift lattice in batches of 16 members.

    (1) Three FP32 sweeps of a batch of 16 shifts: the first, a middle and the last
        member against the oracle's Algorithm 1 (Eqs. 5.7-5.10) on the translated
        phase map (Eq. 3.3) at the same sweep count.
    (2) bfcs_translate_average over the same 16 shifts at the same sweep count
        against the averages of Eqs. 3.4-3.6 written out here (FP64 sums of u, V u,
        eps, V eps, sigma, V sigma over the members' fields from (1)) and the
        inclusion hit counts.
    (3) The bench's converged form (mixed ladder to 1e-6) of the average over the
        first 16 shifts against an all-FP64 average to 1e-9: relative L2 below
        contrast x tol = 1e-5 per field group."""
    p = W.config_c3()
    shifts = W.c3_shifts()[:16]
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    ph_o = O.phase_map(p.dims, p.cell, p.spheres)
    assert np.array_equal(ph.cpu().numpy(), ph_o)
    b32 = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp32")
    b_o = O.body_force(p.dims, p.bf_centre, p.bf_radius)
    with api.Plan(p.dims, "fp32", max_batch=16) as plan:
        members = [dict(phase=ph, b=b32, shift=tuple(int(v) for v in chi)) for chi in shifts]
        members, infos = plan.solve_batched(members, p.phases, p.c0, tol=0.0, maxit=SWEEPS)
        assert all(i.iters == SWEEPS for i in infos)
        avg, hits, _ = plan.translate_average(ph, p.phases, p.c0, b32, shifts, tol=0.0, maxit=SWEEPS)
    for j in (0, 7, 15):
        pj = O.translate(ph_o, shifts[j])
        with sfft.set_workers(os.cpu_count() or 1):
            ref = O.solve(pj, p.phases, p.c0, b_o, tol=0.0, maxit=SWEEPS)
        for key, out in (("eps", "eps_out"), ("sig", "sig_out"), ("u", "u_out")):
            err = rel(members[j][out].cpu().numpy(), ref[key])
            assert err < TOL["fp32"], (j, key, err)
    acc = np.zeros((30,) + ph_o.shape)
    hit = np.zeros(ph_o.shape, dtype=np.int64)
    for chi, m in zip(shifts, members):
        v = (O.translate(ph_o, chi) != 0).astype(np.float64)
        u, e, s = (m[k].cpu().numpy().astype(np.float64) for k in ("u_out", "eps_out", "sig_out"))
        acc[0:3] += u
        acc[3:6] += v * u
        acc[6:12] += e
        acc[12:18] += v * e
        acc[18:24] += s
        acc[24:30] += v * s
        hit += v.astype(np.int64)
    acc /= len(shifts)
    assert np.array_equal(hits.cpu().numpy(), hit)
    got = avg.cpu().numpy()
    for lo, hi in ((0, 6), (6, 18), (18, 30)):
        assert rel(got[lo:hi], acc[lo:hi]) < 1e-12, (lo, rel(got[lo:hi], acc[lo:hi]))
    del members, avg, acc
    b64 = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp64")
    with api.Plan(p.dims, "fp64", max_batch=16) as plan:
        a64, h64, i64 = plan.translate_average(ph, p.phases, p.c0, b64, shifts, tol=1e-9, maxit=20000)
    assert all(i.status == _lib.OK for i in i64)
    with api.Plan(p.dims, "mixed", max_batch=16) as plan:
        am, hm, im = plan.translate_average(ph, p.phases, p.c0, b64, shifts, tol=p.tol, maxit=p.maxit)
    assert all(i.status == _lib.OK and i.resid <= p.tol for i in im)
    assert torch.equal(hm, h64)
    a64, am = a64.cpu().numpy(), am.cpu().numpy()
    for lo, hi in ((0, 6), (6, 18), (18, 30)):
        assert rel(am[lo:hi], a64[lo:hi]) < 1e-5, (lo, rel(am[lo:hi], a64[lo:hi]))
