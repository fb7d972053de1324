"""GPU parity of the displacement-based conjugate gradients (Algorithm 3, Eqs.
5.14-5.22, reading R18) against the FP64 oracle, through the C ABI.

Fixed iteration counts compare the CG iterates themselves (plain as printed and
G0-preconditioned): the strain, stress and displacement after j iterations match
the oracle's Algorithm 3 to 1e-10 (FP64) and 1e-5 (FP32) in relative L2.
Converged solves reach the fixed point of Algorithm 1 with the oracle's own
residual of the returned field at the tolerance.
"""
import numpy as np
import pytest
import torch

from oracle import bfcs_oracle as O
from paper_2601_00822_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def problem(name):
    if name == "c1_32cubed":
        return W.config_c1()
    if name == "ragged_48x24x96":
        return W.Problem(name="t", dims=(48, 24, 96), cell=(24, 12, 32),
                         spheres=np.asarray([[24, 12, 30, 90, 1], [3, 20, 60, 40, 2]], dtype=np.int32),
                         phases=[(1.0, 0.5), (6.0, 3.0), (0.5, 0.3)],
                         c0=W.reference_medium([(1.0, 0.5), (6.0, 3.0), (0.5, 0.3)]),
                         bf_centre=(24.0, 12.0, 48.0), bf_radius=7.0, mean_strain=(0.0,) * 6)
    # mean strain and a non-cubic grid
    return W.Problem(name="t", dims=(12, 32, 24), cell=(12, 16, 12),
                     spheres=np.asarray([[12, 16, 12, 49, 1]], dtype=np.int32),
                     phases=[(1.0, 0.5), (10.0, 5.0)], c0=W.reference_medium([(1.0, 0.5), (10.0, 5.0)]),
                     bf_centre=(6.0, 16.0, 12.0), bf_radius=4.5,
                     mean_strain=(0.01, -0.004, 0.002, 0.001, -0.003, 0.005))


def inputs(p, precision):
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, precision)
    return ph, b


def oracle_inputs(p):
    return O.phase_map(p.dims, p.cell, p.spheres), O.body_force(p.dims, p.bf_centre, p.bf_radius)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("cd", ["plain", "g0"])
@pytest.mark.parametrize("name", ["c1_32cubed", "ragged_48x24x96", "aniso_12x32x24"])
def test_cd_iterates_match_the_oracle(name, cd, precision):
    p = problem(name)
    ph_o, b_o = oracle_inputs(p)
    ph, b = inputs(p, precision)
    j = 5
    ref = O.solve_cd(ph_o, p.phases, p.c0, b_o, p.mean_strain, tol=0.0, maxit=j, precondition=cd == "g0")
    with api.Plan(p.dims, precision, cd=cd) as plan:
        eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, E=p.mean_strain, tol=0.0, maxit=j)
    assert info.iters == j == ref["iters"]
    bar = 1e-10 if precision == "fp64" else 1e-5
    for got, key in ((eps, "eps"), (sig, "sig"), (u, "u")):
        assert rel(got.cpu().numpy(), ref[key]) < bar, (key, rel(got.cpu().numpy(), ref[key]))
    assert abs(info.resid - ref["resid"]) <= 1e-3 * ref["resid"]


@pytest.mark.parametrize("cd", ["plain", "g0"])
def test_cd_converges_to_the_basic_scheme_fixed_point(cd):
    p = problem("c1_32cubed")
    ph_o, b_o = oracle_inputs(p)
    ref = O.solve(ph_o, p.phases, p.c0, b_o, tol=1e-12, maxit=4000)
    ph, b = inputs(p, "fp64")
    with api.Plan(p.dims, "fp64", cd=cd) as plan:
        eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, tol=1e-10, maxit=5000)
    assert info.status == _lib.OK and info.resid <= 1e-10
    r = O.residual(ph_o, p.phases, eps.cpu().numpy(), O.fft3(b_o), O.wavevectors(p.dims))
    assert r <= 1.05e-10 and abs(r - info.resid) <= 1e-3 * r
    for got, key in ((eps, "eps"), (sig, "sig"), (u, "u")):
        assert rel(got.cpu().numpy(), ref[key]) < 1e-8, (key, rel(got.cpu().numpy(), ref[key]))
    # the oracle's iteration count for the same tolerance (same algorithm, FP64 rounding apart)
    its = O.solve_cd(ph_o, p.phases, p.c0, b_o, tol=1e-10, maxit=5000, precondition=cd == "g0")["iters"]
    assert abs(info.iters - its) <= 2, (info.iters, its)


def test_cd_batched_members_equal_individual_solves():
    p = problem("aniso_12x32x24")
    ph, b = inputs(p, "fp32")
    shifts = [(0, 0, 0), (3, 5, 7), (11, 2, 9)]
    with api.Plan(p.dims, "fp32", max_batch=3, cd="g0") as plan, api.Plan(p.dims, "fp32", cd="g0") as one:
        members = [dict(phase=ph, b=b, E=p.mean_strain, shift=s) for s in shifts]
        members, infos = plan.solve_batched(members, p.phases, p.c0, tol=1e-5, maxit=500)
        for m, s, info in zip(members, shifts, infos):
            (mo,), (io,) = one.solve_batched([dict(phase=ph, b=b, E=p.mean_strain, shift=s)], p.phases, p.c0,
                                             tol=1e-5, maxit=500)
            assert info.status == io.status == _lib.OK and info.iters == io.iters
            for key in ("eps_out", "sig_out", "u_out"):
                assert torch.equal(m[key], mo[key]), (s, key)


def test_cd_in_the_mixed_ladder_meets_1e_9():
    """The ladder's FP32 solves driven by the preconditioned Algorithm 3, with
    float-float defect rounds: the oracle's residual of the returned FP64 strain."""
    p = problem("c1_32cubed")
    ph_o, b_o = oracle_inputs(p)
    ph, b = inputs(p, "fp64")
    with api.Plan(p.dims, "mixed", cd="g0") as plan:
        eps, _, _, info = plan.solve(ph, p.phases, p.c0, b, tol=1e-9, maxit=5000)
    assert info.status == _lib.OK and info.resid <= 1e-9
    r = O.residual(ph_o, p.phases, eps.cpu().numpy(), O.fft3(b_o), O.wavevectors(p.dims))
    assert r <= 1.05e-9


def test_cd_rejects_a_warm_start():
    p = problem("c1_32cubed")
    ph, b = inputs(p, "fp32")
    with api.Plan(p.dims, "fp32", cd="g0") as plan:
        eps, _, _, _ = plan.solve(ph, p.phases, p.c0, b, tol=1e-3, maxit=100)
        with pytest.raises(_lib.BfcsError):
            plan.solve(ph, p.phases, p.c0, b, tol=1e-3, maxit=100, eps_init=eps.clone())


# ---------------------------------------------------------------- degenerate cases
@pytest.mark.parametrize("precision", ["fp32", "fp64", "mixed"])
@pytest.mark.parametrize("cd", ["plain", "g0"])
def test_cd_no_load_and_no_mean_strain_give_the_zero_field(cd, precision):
    """b = 0 and E = 0: the right-hand side b^A vanishes, so the member stops at
    the initial step (no iteration) and every returned field is zero."""
    p = W.config_c1()
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    dt = torch.float32 if precision == "fp32" else torch.float64
    b = torch.zeros((3,) + ph.shape, dtype=dt, device="cuda")
    with api.Plan(p.dims, precision, cd=cd) as plan:
        eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, tol=1e-8, maxit=100)
    assert info.status == _lib.OK and info.iters == 0
    assert float(eps.abs().max()) == 0.0 and float(sig.abs().max()) == 0.0 and float(u.abs().max()) == 0.0


@pytest.mark.parametrize("cd", ["plain", "g0"])
def test_cd_homogeneous_medium_stops_at_the_reference_strain(cd):
    """Every voxel of one phase and C0 equal to it: L1 = 0, so b^A = 0 and the
    returned strain is the reference strain eps^{b(0)} + E of Eq. 2.8 itself, the
    oracle's converged field of the basic scheme, without an iteration."""
    dims = (16, 16, 16)
    phases = [(1.0, 0.5), (3.0, 1.2)]
    E = (0.004, -0.001, 0.002, 0.0, 0.001, -0.003)
    ph_o = np.ones(dims, dtype=np.int8)
    b_o = O.body_force(dims, (8.0, 8.0, 8.0), 4.0)
    ref = O.solve(ph_o, phases, phases[1], b_o, E, tol=1e-13, maxit=50)
    ph = torch.ones(dims, dtype=torch.int8, device="cuda")
    b = api.body_force(dims, (8.0, 8.0, 8.0), 4.0, "fp64")
    with api.Plan(dims, "fp64", cd=cd) as plan:
        eps, sig, u, info = plan.solve(ph, phases, phases[1], b, E=E, tol=1e-12, maxit=50)
    assert info.status == _lib.OK and info.iters == 0 and info.resid <= 1e-12
    for got, key in ((eps, "eps"), (sig, "sig"), (u, "u")):
        assert rel(got.cpu().numpy(), ref[key]) < 1e-12, (key, rel(got.cpu().numpy(), ref[key]))


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("fp32", 1e-5)])
@pytest.mark.parametrize("cd", ["plain", "g0"])
def test_cd_smallest_grid_against_the_oracle(cd, precision, bar):
    """The 4^3 grid (lines of 4 points on every axis, one 4-column tile) with a
    mean strain: three iterations against the oracle's Algorithm 3."""
    p = W.Problem(name="4cubed", dims=(4, 4, 4), cell=(4, 4, 4), spheres=np.asarray([[4, 4, 4, 4, 1]], np.int32),
                  phases=[(1.0, 0.5), (6.0, 3.0)], c0=(3.5, 1.75), bf_centre=(2.0, 2.0, 2.0), bf_radius=1.8,
                  mean_strain=(0.01, 0.0, -0.005, 0.0, 0.002, 0.0))
    ph_o, b_o = oracle_inputs(p)
    ref = O.solve_cd(ph_o, p.phases, p.c0, b_o, p.mean_strain, tol=0.0, maxit=3, precondition=cd == "g0")
    ph, b = inputs(p, precision)
    assert np.array_equal(ph.cpu().numpy(), ph_o)
    with api.Plan(p.dims, precision, cd=cd) as plan:
        eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, E=p.mean_strain, tol=0.0, maxit=3)
    assert info.iters == ref["iters"] >= 1, (info.iters, ref["iters"])
    for got, key in ((eps, "eps"), (sig, "sig"), (u, "u")):
        assert rel(got.cpu().numpy(), ref[key]) < bar, (key, rel(got.cpu().numpy(), ref[key]))


def test_cd_batch_with_a_member_that_stops_at_the_start():
    """One member without load or mean strain (done at the initial step, skipped by
    every later kernel) next to members that iterate: each equals its own solve."""
    p = problem("aniso_12x32x24")
    ph, b = inputs(p, "fp32")
    zero = torch.zeros_like(b)
    specs = [dict(phase=ph, b=b, E=p.mean_strain, shift=(0, 0, 0)),
             dict(phase=ph, b=zero, E=(0.0,) * 6, shift=(3, 5, 7)),
             dict(phase=ph, b=b, E=(0.0,) * 6, shift=(11, 2, 9))]
    with api.Plan(p.dims, "fp32", max_batch=3, cd="g0") as plan, api.Plan(p.dims, "fp32", cd="g0") as one:
        members, infos = plan.solve_batched([dict(s) for s in specs], p.phases, p.c0, tol=1e-5, maxit=500)
        assert infos[1].iters == 0 and float(members[1]["eps_out"].abs().max()) == 0.0
        for m, s, info in zip(members, specs, infos):
            (mo,), (io,) = one.solve_batched([dict(s)], p.phases, p.c0, tol=1e-5, maxit=500)
            assert info.status == io.status == _lib.OK and info.iters == io.iters
            for key in ("eps_out", "sig_out", "u_out"):
                assert torch.equal(m[key], mo[key]), (s["shift"], key)
