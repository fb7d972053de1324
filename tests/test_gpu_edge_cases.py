"""Degenerate and boundary cases of the solve against the oracle: no load and no
mean strain (the zero field), an empty batch, the smallest grid (4^3), a cell
that is all inclusion (a homogeneous medium other than the matrix: one sweep is
exact), and two members at the largest grid (256^3) batched against individual
solves."""
import numpy as np
import pytest
import torch

from oracle import bfcs_oracle as O
from paper_2601_00822_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("precision", ["fp32", "fp64", "mixed"])
def test_no_load_and_no_mean_strain_give_the_zero_field(precision):
    p = W.config_c1()
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    dt = torch.float32 if precision == "fp32" else torch.float64
    b = torch.zeros((3,) + ph.shape, dtype=dt, device="cuda")
    with api.Plan(p.dims, precision) as plan:
        eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, tol=1e-8, maxit=100)
    assert info.status == _lib.OK
    assert float(eps.abs().max()) == 0.0 and float(sig.abs().max()) == 0.0 and float(u.abs().max()) == 0.0


def test_empty_batch_is_a_no_op():
    with api.Plan((16, 16, 16), "fp32", max_batch=2) as plan:
        members, infos = plan.solve_batched([], [(1.0, 0.5)], (1.0, 0.5))
    assert members == [] and infos == []


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_smallest_grid_against_oracle(precision, bar):
    p = W.Problem(name="4cubed", dims=(4, 4, 4), cell=(4, 4, 4), spheres=np.asarray([[4, 4, 4, 4, 1]], np.int32),
                  phases=[(1.0, 0.5), (6.0, 3.0)], c0=(3.5, 1.75), bf_centre=(2.0, 2.0, 2.0), bf_radius=1.8,
                  mean_strain=(0.01, 0.0, -0.005, 0.0, 0.002, 0.0))
    ph_o = O.phase_map(p.dims, p.cell, p.spheres)
    b_o = O.body_force(p.dims, p.bf_centre, p.bf_radius)
    ref = O.solve(ph_o, p.phases, p.c0, b_o, p.mean_strain, tol=0, maxit=7)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    assert np.array_equal(ph.cpu().numpy(), ph_o)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, precision)
    with api.Plan(p.dims, precision) as plan:
        eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, p.mean_strain, tol=0, maxit=7)
    assert info.iters == 7
    for a, key in ((eps, "eps"), (sig, "sig"), (u, "u")):
        assert rel(a.cpu().numpy(), ref[key]) < bar, key


def test_all_inclusion_cell_is_solved_in_one_sweep():
    """Every voxel phase 1 and C0 equal to that phase: the polarization vanishes,
    so the first update is the exact solution (the reference strain of the
    homogeneous problem) and meets the oracle's converged field after one sweep."""
    dims = (16, 16, 16)
    phases = [(1.0, 0.5), (3.0, 1.2)]
    ph_o = np.ones((16, 16, 16), dtype=np.int8)
    b_o = O.body_force(dims, (8.0, 8.0, 8.0), 4.0)
    ref = O.solve(ph_o, phases, phases[1], b_o, tol=1e-13, maxit=50)     # C0 = L1: exact at once
    with api.Plan(dims, "fp64") as plan:
        ph = torch.ones((16, 16, 16), dtype=torch.int8, device="cuda")
        b = api.body_force(dims, (8.0, 8.0, 8.0), 4.0, "fp64")
        eps, _, _, info = plan.solve(ph, phases, phases[1], b, tol=0, maxit=1)
    assert rel(eps.cpu().numpy(), ref["eps"]) < 1e-12


def test_largest_grid_two_members_batched_equals_individual():
    p = W.config_c2(contrast=10.0, seed=1)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp32")
    specs = [((0, 0, 0), (0.0,) * 6), ((17, 5, 200), (0.001, 0.0, 0.0, 0.0, 0.0, -0.0005))]
    with api.Plan(p.dims, "fp32", max_batch=2) as plan:
        mem, infos = plan.solve_batched([dict(phase=ph, b=b, E=E, shift=sh, sig_out=None, u_out=None)
                                         for sh, E in specs], p.phases, p.c0, tol=0, maxit=12)
        assert [i.iters for i in infos] == [12, 12]
        for (sh, E), m in zip(specs, mem):
            (one,), _ = plan.solve_batched([dict(phase=ph, b=b, E=E, shift=sh, sig_out=None, u_out=None)],
                                           p.phases, p.c0, tol=0, maxit=12)
            assert torch.equal(one["eps_out"], m["eps_out"])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_largest_batch_and_more_members_than_the_batch(precision):
    """64 members (the most one launch carries) and 70 members on a plan of
    max_batch 64 (run as groups of at most 64): every member equals its own
    solve, and sampled members match the oracle at the same sweep count."""
    dims = (16, 16, 16)
    p = W.Problem(name="b64", dims=dims, cell=(8, 8, 8), spheres=np.asarray([[8, 8, 8, 30, 1]], np.int32),
                  phases=[(1.0, 0.5), (6.0, 3.0)], c0=(3.5, 1.75), bf_centre=(8.0, 8.0, 8.0), bf_radius=4.0)
    ph = api.voxelize(dims, p.cell, p.spheres)
    b = api.body_force(dims, p.bf_centre, p.bf_radius, precision)
    shifts = [(k % 16, (3 * k) % 16, (7 * k) % 16) for k in range(70)]
    sweeps = 6
    with api.Plan(dims, precision, max_batch=64, sparse_resid=True) as plan:
        for count in (64, 70):
            members = [dict(phase=ph, b=b, shift=s, sig_out=None, u_out=None) for s in shifts[:count]]
            members, infos = plan.solve_batched(members, p.phases, p.c0, tol=0, maxit=sweeps)
            assert len(infos) == count and all(i.iters == sweeps for i in infos)
            with api.Plan(dims, precision, sparse_resid=True) as one:
                for k in (0, 31, count - 1):
                    (m1,), _ = one.solve_batched([dict(phase=ph, b=b, shift=shifts[k], sig_out=None, u_out=None)],
                                                 p.phases, p.c0, tol=0, maxit=sweeps)
                    assert torch.equal(m1["eps_out"], members[k]["eps_out"]), (count, k)
    ph_o = O.phase_map(dims, p.cell, p.spheres)
    b_o = O.body_force(dims, p.bf_centre, p.bf_radius)
    bar = 1e-10 if precision == "fp64" else 1e-5
    for k in (5, 63):
        ref = O.solve(O.translate(ph_o, shifts[k]), p.phases, p.c0, b_o, tol=0, maxit=sweeps)
        assert rel(members[k]["eps_out"].cpu().numpy(), ref["eps"]) < bar, k
