"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars: bit-exact on integer work (phase maps); relative L2 <= 1e-10 for FP64
fields and <= 1e-5 for FP32 fields at the same sweep count (pure rounding).
"""
import numpy as np
import pytest
import torch

from oracle import bfcs_oracle as O
from paper_2601_00822_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    a = a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)
    b = b.astype(np.complex128) if np.iscomplexobj(b) else b.astype(np.float64)
    nb = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0)


def small_problem(dims, cell, sphere_rows, centre, a, phases=((1.0, 0.5), (10.0, 5.0)), E=(0.0,) * 6):
    return W.Problem(name="t", dims=dims, cell=cell, spheres=np.asarray(sphere_rows, dtype=np.int32),
                     phases=list(phases), c0=W.reference_medium(list(phases)), bf_centre=centre,
                     bf_radius=a, mean_strain=E)


def oracle_inputs(p):
    return O.phase_map(p.dims, p.cell, p.spheres), O.body_force(p.dims, p.bf_centre, p.bf_radius)


def gpu_inputs(p, precision):
    return api.voxelize(p.dims, p.cell, p.spheres), api.body_force(p.dims, p.bf_centre, p.bf_radius,
                                                                  precision)


CASES = {
    "c1_32cubed": W.config_c1(),
    "ragged_48x24x96": small_problem((48, 24, 96), (24, 12, 32), [[24, 12, 30, 90, 1], [3, 20, 60, 40, 2]],
                                     (24.0, 12.0, 48.0), 7.0,
                                     phases=((1.0, 0.5), (6.0, 3.0), (0.5, 0.3))),
    "aniso_12x32x24": small_problem((12, 32, 24), (12, 16, 12), [[12, 16, 12, 49, 1]], (6.0, 16.0, 12.0), 4.5,
                                    E=(0.01, -0.004, 0.002, 0.001, -0.003, 0.005)),
    # nz = 6 and 4: the z pass's 24 RMAX threads (72, 48) are rounded up to whole
    # warps, which its residual reduction needs; the history checks the residuals
    "thin_16x12x6": small_problem((16, 12, 6), (8, 12, 6), [[8, 12, 6, 16, 1]], (8.0, 6.0, 3.0), 2.5,
                                  E=(0.002, 0.0, -0.001, 0.0, 0.0, 0.003)),
    "thin_8x8x4": small_problem((8, 8, 4), (8, 8, 4), [[8, 8, 4, 12, 1]], (4.0, 4.0, 2.0), 1.8),
    # line lengths 128 (x), 6 (y) and 192 (z) in one solve
    "long_128x6x192": small_problem((128, 6, 192), (64, 6, 96), [[64, 6, 96, 36, 1], [10, 2, 40, 16, 1]],
                                    (64.0, 3.0, 96.0), 2.8, E=(0.0, 0.001, 0.0, 0.0, 0.002, 0.0)),
}


# ---------------------------------------------------------------- a1, a2
@pytest.mark.parametrize("name", sorted(CASES))
def test_phase_map_bit_exact(name):
    p = CASES[name]
    ph_gpu = api.voxelize(p.dims, p.cell, p.spheres).cpu().numpy()
    assert np.array_equal(ph_gpu, O.phase_map(p.dims, p.cell, p.spheres))


def test_phase_map_bit_exact_full_size_random_spheres():
    p = W.config_c2(contrast=10.0, seed=1)
    ph_gpu = api.voxelize(p.dims, p.cell, p.spheres).cpu().numpy()
    assert np.array_equal(ph_gpu, O.phase_map(p.dims, p.cell, p.spheres))
    assert 0.2 < (ph_gpu != 0).mean() < 0.3


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_body_force(name, precision):
    p = CASES[name]
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, precision).cpu().numpy()
    ref = O.body_force(p.dims, p.bf_centre, p.bf_radius)
    scale = np.abs(ref).max()
    assert np.abs(b - ref).max() <= (1e-15 if precision == "fp64" else 1e-7) * scale


# ---------------------------------------------------------------- a5, a7 transforms
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("dims", [(32, 32, 32), (48, 24, 96), (12, 32, 24), (256, 8, 6),
                                  (192, 6, 128), (6, 128, 192), (128, 192, 6)])
def test_fft3d_against_oracle_transform(dims, precision):
    nx, ny, nz = dims
    r = np.random.default_rng(5)
    x = r.standard_normal((5, nz, ny, nx))
    with api.Plan(dims, precision) as plan:
        xt = torch.tensor(x, dtype=plan.dtype, device="cuda")
        X = plan.fft3d(xt, -1).cpu().numpy()
        ref = O.fft3(x)[..., : nx // 2 + 1]
        t = 1e-6 if precision == "fp32" else 1e-13
        assert rel(X, ref) < t
        cdt = torch.complex128 if precision == "fp64" else torch.complex64
        back = plan.fft3d(torch.tensor(ref, device="cuda").to(cdt), +1).cpu().numpy()
        assert rel(back / (nx * ny * nz), x) < t


# ---------------------------------------------------------------- a3-a9, a11 the solve
def run_pair(p, precision, sweeps, tol=0.0):
    ph_o, b_o = oracle_inputs(p)
    ref = O.solve(ph_o, p.phases, p.c0, b_o, p.mean_strain, tol=tol, maxit=sweeps, history=True)
    ph, b = gpu_inputs(p, precision)
    with api.Plan(p.dims, precision) as plan:
        eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, p.mean_strain, tol=tol, maxit=sweeps)
        hist = plan.history()
    return ref, (eps.cpu().numpy(), sig.cpu().numpy(), u.cpu().numpy(), info, hist)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_fixed_sweeps_parity(name, precision):
    p = CASES[name]
    ref, (eps, sig, u, info, hist) = run_pair(p, precision, sweeps=12)
    assert info.iters == ref["sweeps"] == 12
    t = TOL[precision]
    assert rel(eps, ref["eps"]) < t, rel(eps, ref["eps"])
    assert rel(sig, ref["sig"]) < t
    assert rel(u, ref["u"]) < t
    assert abs(info.resid - ref["resid"]) <= 1e-3 * ref["resid"] + (1e-12 if precision == "fp64" else 1e-6)
    h_ref = np.array(ref["hist"])
    assert len(hist) == len(h_ref)
    assert np.all(np.abs(hist - h_ref) <= 1e-4 * h_ref + (1e-12 if precision == "fp64" else 1e-6))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("sweeps", [30, 45])
def test_sweep_count_stops_at_maxit_with_sweep_graphs(precision, sweeps):
    """A solve that ends at maxit runs exactly maxit sweeps when the sweeps are
    launched as 8-sweep CUDA graphs and maxit is not a multiple of 8 (the growing
    chunks of graph launches are cut at maxit), and matches the oracle there."""
    p = CASES["c1_32cubed"]
    ref, (eps, sig, u, info, hist) = run_pair(p, precision, sweeps=sweeps)
    assert info.iters == ref["sweeps"] == sweeps and len(hist) == sweeps
    t = TOL[precision]
    assert rel(eps, ref["eps"]) < t and rel(sig, ref["sig"]) < t and rel(u, ref["u"]) < t


def test_converged_fp64_config1():
    """Converged C1 in FP64 at the FP64 bar: the GPU solve stops at the tolerance
    after S sweeps; the oracle run for exactly S sweeps gives the same fields to
    1e-10 (pure rounding), and the oracle's own stopping rule ends within one
    sweep of S (the two residuals differ by rounding only near the threshold)."""
    p = W.config_c1()
    ref, (eps, sig, u, info, hist) = run_pair(p, "fp64", sweeps=p.maxit, tol=p.tol)
    assert info.status == _lib.OK and info.resid <= 10 * p.tol
    assert abs(info.iters - ref["sweeps"]) <= 1
    same = ref
    if ref["sweeps"] != info.iters:
        ph_o, b_o = oracle_inputs(p)
        same = O.solve(ph_o, p.phases, p.c0, b_o, tol=0.0, maxit=info.iters)
    for a, key in ((eps, "eps"), (sig, "sig"), (u, "u")):
        assert rel(a, same[key]) < TOL["fp64"], (key, rel(a, same[key]))


def test_fp32_converged_error_against_fp64():
    p = W.config_c1()
    ph, b = gpu_inputs(p, "fp32")
    ph_o, b_o = oracle_inputs(p)
    ref = O.solve(ph_o, p.phases, p.c0, b_o, tol=1e-12, maxit=4000)
    with api.Plan(p.dims, "fp32") as plan:
        eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, tol=1e-5, maxit=2000)
        assert info.status == _lib.OK and info.resid < 2e-5
        # error against the converged FP64 answer: iteration error ~ tol plus rounding
        assert rel(eps.cpu().numpy(), ref["eps"]) < 5e-5
        # below its rounding floor the FP32 iteration stalls and says so
        eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, tol=1e-9, maxit=3000)
        assert info.status == _lib.NOT_CONVERGED and info.stalled == 1 and info.iters < 3000


def test_homogeneous_medium_one_sweep_exact():
    p = small_problem((32, 24, 16), (32, 24, 16), [[20, 20, 20, 60, 1]], (10.0, 12.0, 8.0), 5.0,
                      phases=((2.0, 1.0), (2.0, 1.0)), E=(0.01, 0, 0, 0.002, 0, 0))
    ref, (eps, sig, u, info, hist) = run_pair(p, "fp64", sweeps=1)
    assert info.resid < 1e-13 and hist[0] < 1e-13
    assert rel(eps, ref["eps"]) < 1e-12


# ---------------------------------------------------------------- warm start, batching, averaging
def test_warm_start_from_converged_field():
    p = W.config_c1()
    ph, b = gpu_inputs(p, "fp64")
    with api.Plan(p.dims, "fp64") as plan:
        eps, _, _, info = plan.solve(ph, p.phases, p.c0, b, tol=1e-11, maxit=4000)
        eps2, _, _, info2 = plan.solve(ph, p.phases, p.c0, b, tol=1e-10, maxit=50, eps_init=eps.clone())
        hist = plan.history()
    assert info2.status == _lib.OK and info2.iters <= 2
    assert np.isinf(hist[0])
    assert rel(eps2.cpu().numpy(), eps.cpu().numpy()) < 1e-10


def test_batched_equals_individual_solves():
    p = CASES["aniso_12x32x24"]
    ph, b = gpu_inputs(p, "fp32")
    with api.Plan(p.dims, "fp32") as plan:
        shifts = [(0, 0, 0), (3, 5, 7), (11, 1, 2)]
        members = [dict(phase=ph, b=b, E=p.mean_strain, shift=s) for s in shifts]
        members, infos = plan.solve_batched(members, p.phases, p.c0, tol=0, maxit=9)
        ph_o, b_o = oracle_inputs(p)
        for mem, s in zip(members, shifts):
            ref = O.solve(O.translate(ph_o, s), p.phases, p.c0, b_o, p.mean_strain, tol=0, maxit=9)
            assert rel(mem["eps_out"].cpu().numpy(), ref["eps"]) < 1e-5
    assert all(i.iters == 9 for i in infos)


@pytest.mark.parametrize("max_batch", [1, 3])
def test_translate_average_parity(max_batch):
    dims = (16, 16, 16)
    p = small_problem(dims, (8, 8, 8), [[8, 8, 8, 36, 1]], (8.0, 8.0, 8.0), 4.0)
    shifts = [(0, 0, 0), (2, 0, 0), (0, 4, 2), (6, 6, 6), (1, 3, 5)]
    ph_o, b_o = oracle_inputs(p)
    avg_ref, hits_ref, _ = O.translate_average(ph_o, p.phases, p.c0, b_o, shifts, tol=0, maxit=10)
    ph, b = gpu_inputs(p, "fp64")
    with api.Plan(dims, "fp64", max_batch=max_batch) as plan:
        avg, hits, infos = plan.translate_average(ph, p.phases, p.c0, b, shifts, tol=0, maxit=10)
    assert np.array_equal(hits.cpu().numpy(), hits_ref)
    avg = avg.cpu().numpy()
    for a0, a1 in ((0, 3), (3, 6), (6, 12), (12, 18), (18, 24), (24, 30)):
        assert rel(avg[a0:a1], avg_ref[a0:a1]) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_members_advance_together(precision):
    """Members with different shifts, mean strains and a warm start, in one batch."""
    p = CASES["ragged_48x24x96"]
    ph, b = gpu_inputs(p, precision)
    ph_o, b_o = oracle_inputs(p)
    sweeps = 9
    init_ref = O.solve(ph_o, p.phases, p.c0, b_o, tol=0, maxit=3)["eps"]
    dt = torch.float64 if precision == "fp64" else torch.float32
    init = torch.tensor(init_ref, dtype=dt, device="cuda")
    specs = [((0, 0, 0), (0,) * 6, None), ((5, 3, 11), (0.01, 0, 0, 0, 0, 0.002), None),
             ((47, 23, 95), (0,) * 6, init), ((24, 12, 48), (0, -0.003, 0, 0.001, 0, 0), None)]
    with api.Plan(p.dims, precision, max_batch=4) as plan:
        members = [dict(phase=ph, b=b, E=E, shift=sh, eps_init=ei) for sh, E, ei in specs]
        members, infos = plan.solve_batched(members, p.phases, p.c0, tol=0, maxit=sweeps)
    for mem, (sh, E, ei), info in zip(members, specs, infos):
        ref = O.solve(O.translate(ph_o, sh), p.phases, p.c0, b_o, E, tol=0, maxit=sweeps,
                      eps_init=init_ref if ei is not None else None)
        assert info.iters == sweeps
        for key, k2 in (("eps_out", "eps"), ("sig_out", "sig"), ("u_out", "u")):
            assert rel(mem[key].cpu().numpy(), ref[k2]) < TOL[precision], (sh, key)


def test_graph_and_stream_sweeps_identical(monkeypatch):
    p = CASES["c1_32cubed"]
    ph, b = gpu_inputs(p, "fp32")
    out = []
    for g in ("0", "4"):
        monkeypatch.setenv("BFCS_GRAPH_SWEEPS", g)
        with api.Plan(p.dims, "fp32") as plan:
            eps, _, _, info = plan.solve(ph, p.phases, p.c0, b, tol=1e-5, maxit=500)
        out.append((eps.clone(), info.iters))
    assert out[0][1] == out[1][1]
    assert torch.equal(out[0][0], out[1][0])


# ---------------------------------------------------------------- a13 autotuned y-pass variants
TUNE_CASES = {
    "c1_32cubed": W.config_c1(),                                   # ny = 32 = 8 x 4
    "tall_16x96x12": small_problem((16, 96, 12), (16, 48, 12), [[16, 48, 12, 64, 1]], (8.0, 48.0, 6.0), 5.0),
}


@pytest.mark.parametrize("variant", range(8))
@pytest.mark.parametrize("name", sorted(TUNE_CASES))
def test_every_y_pass_variant_matches_oracle(name, variant, monkeypatch):
    """Each column tile / factor order / tensor-copy tile computes the same sweeps
    (FP32 rounding only)."""
    p = TUNE_CASES[name]
    monkeypatch.setenv("BFCS_COL_VARIANT", str(variant))
    ph, b = gpu_inputs(p, "fp32")
    ph_o, b_o = oracle_inputs(p)
    sweeps = 10
    with api.Plan(p.dims, "fp32") as plan:
        t = plan.tuning()
        eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, tol=0, maxit=sweeps)
    ref = O.solve(ph_o, p.phases, p.c0, b_o, tol=0, maxit=sweeps)
    ny = p.dims[1]
    valid = variant == 0 or (ny >= 32 and (variant < 3 or variant >= 6 or ny not in (64, 256)))
    assert t["variant"] == (variant if valid else 0)
    for a, key in ((eps, "eps"), (sig, "sig"), (u, "u")):
        assert rel(a.cpu().numpy(), ref[key]) < TOL["fp32"], (variant, key)


def test_autotuned_plan_reports_and_uses_its_choice(monkeypatch):
    p = W.config_c2(n=128, cell=32, bf_radius=12.0)
    ph, b = gpu_inputs(p, "fp32")
    monkeypatch.delenv("BFCS_COL_VARIANT", raising=False)
    with api.Plan(p.dims, "fp32", max_batch=2, autotune=True) as plan:
        t = plan.tuning()
        eps, _, _, info = plan.solve(ph, p.phases, p.c0, b, tol=0, maxit=6)
    assert 0 <= t["variant"] < 8 and t["variant_ms"][t["variant"]] > 0
    assert t["variant_ms"][6] > 0 and t["variant_ms"][7] > 0          # the tensor-copy tiles were timed
    assert t["variant_ms"][t["variant"]] == min(v for v in t["variant_ms"] if v > 0)
    assert t["tile"] in (8, 16, 32)
    monkeypatch.setenv("BFCS_COL_VARIANT", str(t["variant"]))
    with api.Plan(p.dims, "fp32") as plan:
        eps2, _, _, _ = plan.solve(ph, p.phases, p.c0, b, tol=0, maxit=6)
    assert torch.equal(eps, eps2)


# ---------------------------------------------------------------- a13 mixed grid sizes in one loop
GROUP = [("c1_32cubed", [((0, 0, 0), (0,) * 6), ((5, 3, 11), (0.01, 0, 0, 0, 0, 0.002))]),
         ("aniso_12x32x24", [((0, 0, 0), (0,) * 6), ((11, 31, 23), (0, -0.003, 0, 0.001, 0, 0))]),
         ("tall_16x96x12", [((3, 7, 1), (0,) * 6)])]     # all three share the phases and C0 of C1


def _group_case(name):
    return CASES[name] if name in CASES else TUNE_CASES[name]


@pytest.mark.parametrize("precision,tol,maxit", [("fp32", 0.0, 9), ("fp32", 1e-4, 400), ("fp64", 0.0, 7)])
def test_group_of_grids_equals_separate_batches(precision, tol, maxit):
    """Three grids advancing in one graph-launched loop give every member exactly
    what its own batched solve gives (same sweeps), and match the oracle."""
    cases = [(name, _group_case(name), specs) for name, specs in GROUP]
    p0 = cases[0][1]
    plans = [api.Plan(p.dims, precision, max_batch=len(specs)) for _, p, specs in cases]
    try:
        groups, inputs = [], []
        for plan, (name, p, specs) in zip(plans, cases):
            ph, b = gpu_inputs(p, precision)
            inputs.append((ph, b))
            groups.append((plan, [dict(phase=ph, b=b, E=E, shift=sh) for sh, E in specs]))
        out = api.solve_group(groups, p0.phases, p0.c0, tol=tol, maxit=maxit)
        for plan, (name, p, specs), (ph, b), (members, infos) in zip(plans, cases, inputs, out):
            ref_m, ref_i = plan.solve_batched([dict(phase=ph, b=b, E=E, shift=sh) for sh, E in specs],
                                              p0.phases, p0.c0, tol=tol, maxit=maxit)
            for mem, rm, inf, ri in zip(members, ref_m, infos, ref_i):
                assert inf.iters == ri.iters and inf.status == ri.status, name
                for key in ("eps_out", "sig_out", "u_out"):
                    assert torch.equal(mem[key], rm[key]), (name, key)
            if tol == 0.0:
                sh, E = specs[-1]
                ph_o, b_o = oracle_inputs(p)
                ref = O.solve(O.translate(ph_o, sh), p0.phases, p0.c0, b_o, E, tol=0, maxit=maxit)
                assert rel(members[-1]["eps_out"].cpu().numpy(), ref["eps"]) < TOL[precision], name
    finally:
        for plan in plans:
            plan.close()


@pytest.mark.parametrize("dims", [(64, 64, 64), (96, 128, 48)])
def test_persistent_z_pass_equals_one_tile_per_block(dims, monkeypatch):
    """The persistent, double-buffered z/Green pass computes every mode exactly as
    the one-tile-per-block form (bit-identical fields after fixed sweeps, batched
    members with one converging early); only the grouping of the residual
    partial sums differs."""
    nx, ny, nz = dims
    p = small_problem(dims, (nx // 2, ny // 2, nz // 2), [[nx // 2, ny // 2, nz // 2, 100, 1]],
                      (nx / 2, ny / 2, nz / 2), 6.0)
    ph, b = gpu_inputs(p, "fp32")
    out = {}
    for flag in ("0", "1"):
        monkeypatch.setenv("BFCS_ZGREEN_PERSISTENT", flag)
        with api.Plan(dims, "fp32", max_batch=3) as plan:
            members = [dict(phase=ph, b=b, shift=(k, 2 * k, 3 * k)) for k in range(3)]
            members, infos = plan.solve_batched(members, p.phases, p.c0, tol=0, maxit=12)
            hist = plan.history()
            eps, _, _, one = plan.solve(ph, p.phases, p.c0, b, tol=3e-3, maxit=500)
        out[flag] = ([m["eps_out"].clone() for m in members], hist, eps.clone(), one.iters)
    for a, b2 in zip(out["0"][0], out["1"][0]):
        assert torch.equal(a, b2)
    assert np.allclose(out["0"][1], out["1"][1], rtol=1e-9, atol=0)
    assert out["0"][3] == out["1"][3] and torch.equal(out["0"][2], out["1"][2])


# ---------------------------------------------------------------- errors
def test_error_statuses():
    p = CASES["aniso_12x32x24"]
    ph, b = gpu_inputs(p, "fp32")
    with api.Plan(p.dims, "fp32") as plan:
        bad_b = b.clone()
        bad_b[0] += 0.5                                    # not self-equilibrated (Eq. 2.5)
        with pytest.raises(_lib.BfcsError) as e:
            plan.solve(ph, p.phases, p.c0, bad_b, tol=1e-6, maxit=5)
        assert e.value.code == _lib.ERR_NONZERO_MEAN
        bad_ph = ph.clone()
        bad_ph[0, 0, 0] = 7                                # phase id beyond the table
        with pytest.raises(_lib.BfcsError) as e:
            plan.solve(bad_ph, p.phases, p.c0, b, tol=1e-6, maxit=5)
        assert e.value.code == _lib.ERR_INVALID_ARG
        with pytest.raises(_lib.BfcsError) as e:
            plan.solve(ph, p.phases, (1.0, -1.0), b, tol=1e-6, maxit=5)
        assert e.value.code == _lib.ERR_INVALID_ARG
        eps, _, _, info = plan.solve(ph, p.phases, p.c0, b, tol=1e-30, maxit=3)
        assert info.status == _lib.NOT_CONVERGED and info.iters == 3
        # the plan is still usable after the errors
        eps2, _, _, info2 = plan.solve(ph, p.phases, p.c0, b, tol=0, maxit=3)
        assert torch.equal(eps, eps2)


# ---------------------------------------------------------------- a12 precision ladder
def test_mixed_ladder_goes_below_the_fp32_floor():
    p = W.config_c1()
    ph_o, b_o = oracle_inputs(p)
    ref = O.solve(ph_o, p.phases, p.c0, b_o, tol=1e-12, maxit=4000)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp64")
    with api.Plan(p.dims, "mixed") as plan:
        eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, tol=1e-9, maxit=4000)
        assert info.status == _lib.OK and info.resid <= 1e-9 and info.precision_path == 2
        for a, key in ((eps, "eps"), (sig, "sig"), (u, "u")):
            assert rel(a.cpu().numpy(), ref[key]) < 1e-8, (key, rel(a.cpu().numpy(), ref[key]))
        # the returned FP64 field's residual, evaluated by the oracle
        r = O.residual(ph_o, p.phases, eps.cpu().numpy(), O.fft3(b_o), O.wavevectors(p.dims))
        assert r <= 2e-9
        # a warm start from the converged field enters the FP32 phase already
        # converged there; one correction below the FP32 floor remains
        eps2, _, u2, info2 = plan.solve(ph, p.phases, p.c0, b, tol=1e-9, maxit=4000, eps_init=eps.clone())
        assert info2.status == _lib.OK and info2.resid <= 1e-9
        assert info2.iters < 0.5 * info.iters, (info2.iters, info.iters)
        assert rel(eps2.cpu().numpy(), eps.cpu().numpy()) < 1e-8
        # the displacement agrees up to its rounding-level mean (gauge) component
        assert rel(u2.cpu().numpy(), u.cpu().numpy()) < 1e-8


def test_mixed_ladder_defect_reaches_1e_12():
    """The defect passes compute in float-float (~48 bits): tight enough for a
    residual of 1e-12, confirmed by the oracle's FP64 residual of the field."""
    p = W.config_c1()
    ph_o, b_o = oracle_inputs(p)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp64")
    with api.Plan(p.dims, "mixed") as plan:
        eps, _, _, info = plan.solve(ph, p.phases, p.c0, b, tol=1e-12, maxit=6000, want_sig=False, want_u=False)
    assert info.status == _lib.OK and info.resid <= 1e-12
    r = O.residual(ph_o, p.phases, eps.cpu().numpy(), O.fft3(b_o), O.wavevectors(p.dims))
    assert r <= 2e-12, r


@pytest.mark.parametrize("tol", [1e-6, 1e-9])
@pytest.mark.parametrize("name", ["c1_32cubed", "aniso_12x32x24"])
def test_mixed_strain_increments_keep_the_strain_compatible(name, tol):
    """At tolerances of 1e-9 and above, the ladder's rounds after the first carry
    the FP64 strain forward by each correction's FP32 strain instead of re-forming
    it from the displacement.  The returned strain must still equal E + sym grad u
    of the returned displacement (spectral, Eq. 2.3 with Eq. 4.8, through the
    oracle's transforms) to 1e-9 of its norm.  It must meet the tolerance by the
    oracle's own residual, and info.resid must be that residual (up to the
    float-float arithmetic): the defect is still evaluated from the returned field."""
    p = CASES[name]
    ph_o, b_o = oracle_inputs(p)
    ph, _ = gpu_inputs(p, "fp32")
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp64")
    with api.Plan(p.dims, "mixed") as plan:
        eps, _, u, info = plan.solve(ph, p.phases, p.c0, b, E=p.mean_strain, tol=tol, maxit=6000)
    assert info.status == _lib.OK and info.resid <= tol and info.precision_path == 2
    e, uu = eps.cpu().numpy(), u.cpu().numpy()
    xi = O.wavevectors(p.dims)
    e_ref = np.real(O.ifft3(O.sym_grad_hat(O.fft3(uu), xi)))
    e_ref += np.asarray(p.mean_strain, dtype=np.float64).reshape(6, 1, 1, 1)
    assert rel(e, e_ref) < 1e-9, rel(e, e_ref)
    r = O.residual(ph_o, p.phases, e, O.fft3(b_o), xi)
    # float-float defect passes: ~48 bits relative to the stress scale, ~1e-15 of D absolute
    assert r <= 1.05 * tol and abs(r - info.resid) <= 1e-4 * r + 1e-14, (r, info.resid)


def test_mixed_batched_equals_individual_and_meets_tolerance():
    """The batched ladder (FP32 sweeps of all members in one launch per pass,
    FP64 defects per member) gives each member exactly the individual result;
    every returned field meets the tolerance by the oracle's own residual."""
    p = W.config_c1()
    ph_o, b_o = oracle_inputs(p)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp64")
    init = torch.tensor(O.solve(ph_o, p.phases, p.c0, b_o, tol=0, maxit=5)["eps"], device="cuda")
    specs = [((0, 0, 0), (0,) * 6, None), ((5, 3, 11), (0.01, 0, 0, 0, 0, 0.002), None),
             ((0, 0, 0), (0,) * 6, init), ((31, 16, 2), (0, -0.003, 0, 0.001, 0, 0), None),
             ((7, 7, 7), (0,) * 6, init)]
    tol = 1e-9
    with api.Plan(p.dims, "mixed", max_batch=3) as plan, api.Plan(p.dims, "mixed") as single:
        members = [dict(phase=ph, b=b, E=E, shift=sh, eps_init=ei) for sh, E, ei in specs]
        members, infos = plan.solve_batched(members, p.phases, p.c0, tol=tol, maxit=4000)
        for mem, (sh, E, ei), info in zip(members, specs, infos):
            assert info.status == _lib.OK and info.resid <= tol and info.precision_path == 2
            (one_m,), (one,) = single.solve_batched([dict(phase=ph, b=b, E=E, shift=sh, eps_init=ei)],
                                                    p.phases, p.c0, tol=tol, maxit=4000)
            assert one.iters == info.iters and one.resid == info.resid
            for key in ("eps_out", "sig_out", "u_out"):
                assert torch.equal(one_m[key], mem[key]), (sh, key)
            r = O.residual(O.translate(ph_o, sh), p.phases, mem["eps_out"].cpu().numpy(), O.fft3(b_o),
                           O.wavevectors(p.dims))
            assert r <= 2 * tol, (sh, r)


def test_mixed_translate_average_against_oracle():
    dims = (16, 16, 16)
    p = small_problem(dims, (8, 8, 8), [[8, 8, 8, 36, 1]], (8.0, 8.0, 8.0), 4.0)
    shifts = [(0, 0, 0), (3, 1, 4), (7, 7, 0)]
    ph_o, b_o = oracle_inputs(p)
    avg_ref, hits_ref, _ = O.translate_average(ph_o, p.phases, p.c0, b_o, shifts, tol=1e-12, maxit=4000)
    ph = api.voxelize(dims, p.cell, p.spheres)
    b = api.body_force(dims, p.bf_centre, p.bf_radius, "fp64")
    with api.Plan(dims, "mixed") as plan:
        avg, hits, infos = plan.translate_average(ph, p.phases, p.c0, b, shifts, tol=1e-10, maxit=4000)
    assert all(i.status == _lib.OK for i in infos)
    assert np.array_equal(hits.cpu().numpy(), hits_ref)
    avg = avg.cpu().numpy()
    for a0, a1 in ((0, 3), (3, 6), (6, 12), (12, 18), (18, 24), (24, 30)):
        assert rel(avg[a0:a1], avg_ref[a0:a1]) < 1e-8


# ---------------------------------------------------------------- C4: stiff inclusions, contrast 1000
def test_precision_study_contrast_1000():
    """C4's microstructure (RSA vf 0.3, Young contrast 1000) at 32^3: FP32 and FP64
    sweeps match the oracle at a fixed sweep count, and the converged mixed ladder
    agrees with an all-FP64 GPU solve to within what the tolerances allow."""
    p = W.config_c2(contrast=1000.0, seed=1, n=32, cell=32, vf=0.3, bf_radius=6.0)
    ph_o, b_o = oracle_inputs(p)
    ref = O.solve(ph_o, p.phases, p.c0, b_o, tol=0, maxit=15)
    for precision in ("fp32", "fp64"):
        ph, b = gpu_inputs(p, precision)
        with api.Plan(p.dims, precision) as plan:
            eps, sig, _, _ = plan.solve(ph, p.phases, p.c0, b, tol=0, maxit=15)
        assert rel(eps.cpu().numpy(), ref["eps"]) < TOL[precision], precision
        assert rel(sig.cpu().numpy(), ref["sig"]) < TOL[precision], precision
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp64")
    with api.Plan(p.dims, "fp64") as plan:
        e64, s64, _, i64 = plan.solve(ph, p.phases, p.c0, b, tol=1e-9, maxit=200000)
    with api.Plan(p.dims, "mixed") as plan:
        em, sm, _, im = plan.solve(ph, p.phases, p.c0, b, tol=1e-7, maxit=200000)
    assert i64.status == _lib.OK and im.status == _lib.OK and im.resid <= 1e-7
    assert i64.iters > 1000            # the slow fixed point of a stiff, high-contrast composite
    err_e = rel(em.cpu().numpy(), e64.cpu().numpy())
    err_s = rel(sm.cpu().numpy(), s64.cpu().numpy())
    assert err_e < 1e-4 and err_s < 1e-4, (err_e, err_s, im.iters, i64.iters)


# ---------------------------------------------------------------- conjugate gradients (Algorithm 2)
def test_cg_converges_to_the_oracle_fixed_point_in_fewer_applications():
    p = W.config_c1()
    ph_o, b_o = oracle_inputs(p)
    ref = O.solve(ph_o, p.phases, p.c0, b_o, tol=1e-12, maxit=4000)
    ph, b = gpu_inputs(p, "fp64")
    with api.Plan(p.dims, "fp64", cg=True) as plan:
        eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, tol=1e-10, maxit=4000)
    with api.Plan(p.dims, "fp64") as plan:
        _, _, _, basic = plan.solve(ph, p.phases, p.c0, b, tol=1e-10, maxit=4000)
    assert info.status == _lib.OK and info.resid <= 1e-10
    for a, key in ((eps, "eps"), (sig, "sig"), (u, "u")):
        assert rel(a.cpu().numpy(), ref[key]) < 1e-8, key
    r = O.residual(ph_o, p.phases, eps.cpu().numpy(), O.fft3(b_o), O.wavevectors(p.dims))
    assert r <= 2e-10
    assert info.iters < basic.iters, (info.iters, basic.iters)


def test_cg_at_contrast_1000_against_plain_sweeps():
    """Stiff inclusions (C4's microstructure at 32^3): CG reaches the same field
    as the plain scheme with a small fraction of its operator applications."""
    p = W.config_c2(contrast=1000.0, seed=1, n=32, cell=32, vf=0.3, bf_radius=6.0)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp64")
    with api.Plan(p.dims, "fp64") as plan:
        e0, s0, _, i0 = plan.solve(ph, p.phases, p.c0, b, tol=1e-9, maxit=200000)
    with api.Plan(p.dims, "fp64", cg=True) as plan:
        e1, s1, _, i1 = plan.solve(ph, p.phases, p.c0, b, tol=1e-9, maxit=200000)
    assert i0.status == _lib.OK and i1.status == _lib.OK and i1.resid <= 1e-9
    assert rel(e1.cpu().numpy(), e0.cpu().numpy()) < 1e-6
    assert i1.iters * 5 < i0.iters, (i1.iters, i0.iters)


@pytest.mark.parametrize("variant", [0, 1, 6, 7])
def test_cg_operator_under_every_y_pass_variant(variant, monkeypatch):
    """The operator's y passes run on the CG vectors, not on the plan's spectrum.
    Under every y-pass variant (the tensor-copy tiles included, whose tensor maps
    address the spectrum), a fixed number of operator applications (the first
    sweep, 6 CG iterations, 2 verifying sweeps) gives the FP64 plan's iterate
    (FP64 plans have no tensor-copy tiles)."""
    p = W.config_c1()
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    monkeypatch.setenv("BFCS_COL_VARIANT", str(variant))
    with api.Plan(p.dims, "fp32", cg=True) as plan:
        assert plan.tuning()["variant"] == variant
        b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp32")
        eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, tol=1e-12, maxit=8)
    monkeypatch.delenv("BFCS_COL_VARIANT")
    with api.Plan(p.dims, "fp64", cg=True) as plan:
        b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp64")
        e64, s64, u64, i64 = plan.solve(ph, p.phases, p.c0, b, tol=1e-12, maxit=8)
    assert info.iters == i64.iters == 9, (info.iters, i64.iters)
    for a, r, key in ((eps, e64, "eps"), (sig, s64, "sig"), (u, u64, "u")):
        assert rel(a.cpu().numpy(), r.cpu().numpy()) < 1e-4, (variant, key, rel(a.cpu().numpy(), r.cpu().numpy()))


def test_cg_inside_the_mixed_ladder_and_batched_equals_individual():
    p = W.config_c1()
    ph_o, b_o = oracle_inputs(p)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp64")
    specs = [((0, 0, 0), (0,) * 6), ((5, 3, 11), (0.01, 0, 0, 0, 0, 0.002)), ((31, 16, 2), (0,) * 6)]
    with api.Plan(p.dims, "mixed", max_batch=3, cg=True) as plan, api.Plan(p.dims, "mixed", cg=True) as one:
        members, infos = plan.solve_batched([dict(phase=ph, b=b, E=E, shift=sh) for sh, E in specs],
                                            p.phases, p.c0, tol=1e-9, maxit=4000)
        for mem, (sh, E), info in zip(members, specs, infos):
            assert info.status == _lib.OK and info.resid <= 1e-9
            (m1,), (i1,) = one.solve_batched([dict(phase=ph, b=b, E=E, shift=sh)], p.phases, p.c0, tol=1e-9,
                                             maxit=4000)
            assert i1.iters == info.iters and torch.equal(m1["eps_out"], mem["eps_out"])
            r = O.residual(O.translate(ph_o, sh), p.phases, mem["eps_out"].cpu().numpy(), O.fft3(b_o),
                           O.wavevectors(p.dims))
            assert r <= 2e-9, (sh, r)


# ---------------------------------------------------------------- full size (256^3, the benchmarked launch)
def test_full_size_solve_meets_tolerance_independently_checked():
    p = W.config_c2(contrast=10.0, seed=1)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp64")
    with api.Plan(p.dims, "mixed") as plan:
        eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, tol=p.tol, maxit=4000)
    assert info.status == _lib.OK and info.resid <= p.tol
    # independent check by the oracle's residual (Eq. 5.11 reading) on the returned field
    ph_o = O.phase_map(p.dims, p.cell, p.spheres)
    assert np.array_equal(ph.cpu().numpy(), ph_o)
    b_o = O.body_force(p.dims, p.bf_centre, p.bf_radius)
    e = eps.cpu().numpy()
    r = O.residual(ph_o, p.phases, e, O.fft3(b_o), O.wavevectors(p.dims))
    assert r <= 1.05 * p.tol, r
    assert abs(r - info.resid) <= 1e-3 * r
    # sigma = L(x) eps voxel by voxel on a sample
    s = sig.cpu().numpy()
    rng = np.random.default_rng(0)
    idx = tuple(rng.integers(0, 256, size=(3, 4000)))
    sref = O.apply_local(ph_o[idx], p.phases, e[(slice(None),) + idx])
    assert np.allclose(s[(slice(None),) + idx], sref, rtol=1e-13, atol=1e-15)
    # the FP32-only path stops at its rounding floor and says so
    b32 = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp32")
    with api.Plan(p.dims, "fp32") as plan:
        _, _, _, info32 = plan.solve(ph, p.phases, p.c0, b32, tol=p.tol, maxit=4000)
    assert info32.status == _lib.NOT_CONVERGED and info32.stalled == 1 and info32.resid < 1e-4


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_phase_map_at_an_unaligned_address(precision):
    """A phase map passed as a view one byte into a larger buffer (the x pass then
    reads it directly instead of staging 16-byte pieces) gives the same fields as
    the same map at an aligned address; both match the oracle at a fixed sweep count."""
    p = CASES["c1_32cubed"]
    ph, b = gpu_inputs(p, precision)
    big = torch.zeros(ph.numel() + 1, dtype=torch.int8, device="cuda")
    big[1:].copy_(ph.view(-1))
    ph_off = big[1:].view(ph.shape)
    assert ph_off.data_ptr() % 16 == 1
    with api.Plan(p.dims, precision) as plan:
        e0, s0, u0, _ = plan.solve(ph, p.phases, p.c0, b, tol=0, maxit=6)
        e1, s1, u1, _ = plan.solve(ph_off, p.phases, p.c0, b, tol=0, maxit=6)
    assert torch.equal(e0, e1) and torch.equal(s0, s1) and torch.equal(u0, u1)
    ph_o, b_o = oracle_inputs(p)
    ref = O.solve(ph_o, p.phases, p.c0, b_o, tol=0, maxit=6)
    assert rel(e1.cpu().numpy(), ref["eps"]) < TOL[precision] * 10


# ---------------------------------------------------------------- sparse residual evaluation
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["c1_32cubed", "ragged_48x24x96"])
def test_sparse_residual_same_fields_fixed_sweeps(name, precision):
    """With BFCS_SPARSE_RESID every sweep computes the same fields (the residual
    does not enter the iteration) and the residuals it does evaluate (every 8th
    sweep with tol = 0) are those of the dense evaluation; the final residual
    and the oracle's fields after the same sweeps agree."""
    p = CASES[name]
    ph, b = gpu_inputs(p, precision)
    sweeps = 20
    out = {}
    for sparse in (False, True):
        with api.Plan(p.dims, precision, sparse_resid=sparse) as plan:
            eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, p.mean_strain, tol=0.0, maxit=sweeps)
            out[sparse] = (eps.clone(), sig.clone(), u.clone(), info, plan.history())
    e0, s0, u0, i0, h0 = out[False]
    e1, s1, u1, i1, h1 = out[True]
    assert torch.equal(e0, e1) and torch.equal(s0, s1) and torch.equal(u0, u1)
    assert i1.iters == i0.iters == sweeps and i1.resid == i0.resid
    evaluated = ~np.isnan(h1)
    assert list(np.nonzero(evaluated)[0]) == [0, 8, 16]
    assert np.array_equal(h1[evaluated], h0[evaluated])
    ph_o, b_o = oracle_inputs(p)
    ref = O.solve(ph_o, p.phases, p.c0, b_o, p.mean_strain, tol=0.0, maxit=sweeps)
    assert rel(e1.cpu().numpy(), ref["eps"]) < TOL[precision]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-5)])
def test_sparse_residual_converged_solve(precision, tol):
    """A converged solve with sparse evaluation meets the tolerance, stops at
    most two sweeps after the dense evaluation would, and its fields equal the
    oracle's after the same number of sweeps (batched members with different
    shifts, mean strains and a warm start included)."""
    p = CASES["ragged_48x24x96"]
    ph, b = gpu_inputs(p, precision)
    ph_o, b_o = oracle_inputs(p)
    init_ref = O.solve(ph_o, p.phases, p.c0, b_o, tol=0, maxit=3)["eps"]
    dt = torch.float64 if precision == "fp64" else torch.float32
    init = torch.tensor(init_ref, dtype=dt, device="cuda")
    specs = [((0, 0, 0), (0,) * 6, None), ((5, 3, 11), (0.01, 0, 0, 0, 0, 0.002), None),
             ((47, 23, 95), (0,) * 6, init)]
    res = {}
    for sparse in (False, True):
        with api.Plan(p.dims, precision, max_batch=3, sparse_resid=sparse) as plan:
            members = [dict(phase=ph, b=b, E=E, shift=sh, eps_init=ei) for sh, E, ei in specs]
            members, infos = plan.solve_batched(members, p.phases, p.c0, tol=tol, maxit=4000)
        res[sparse] = (members, infos)
    for k, (sh, E, ei) in enumerate(specs):
        dense, sparse = res[False][1][k], res[True][1][k]
        assert sparse.status == _lib.OK and sparse.resid <= tol
        assert dense.iters <= sparse.iters <= dense.iters + 2, (k, dense.iters, sparse.iters)
        ref = O.solve(O.translate(ph_o, sh), p.phases, p.c0, b_o, E, tol=0.0, maxit=sparse.iters,
                      eps_init=init_ref if ei is not None else None)
        for key, k2 in (("eps_out", "eps"), ("sig_out", "sig"), ("u_out", "u")):
            assert rel(res[True][0][k][key].cpu().numpy(), ref[k2]) < TOL[precision], (k, key)


def test_sparse_residual_in_the_mixed_ladder():
    """The bench's configuration (mixed ladder, autotuned, sparse evaluation) on C1
    reaches 1e-9 by the oracle's own residual of the returned field."""
    p = W.config_c1()
    ph_o, b_o = oracle_inputs(p)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp64")
    with api.Plan(p.dims, "mixed", autotune=True, sparse_resid=True) as plan:
        eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, tol=1e-9, maxit=4000)
    assert info.status == _lib.OK and info.resid <= 1e-9
    r = O.residual(ph_o, p.phases, eps.cpu().numpy(), O.fft3(b_o), O.wavevectors(p.dims))
    assert r <= 2e-9, r


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("comps", [(1,), (2,), (0, 2), (0, 1, 2)])
def test_loads_with_vanishing_components(comps, precision):
    """The z pass neither stages nor reads load components that vanish identically;
    loads along other axes and with several components match the oracle at a fixed
    sweep count (dense and sparse residual evaluation)."""
    p = CASES["ragged_48x24x96"]
    ph_o, b_o = oracle_inputs(p)
    b3 = np.zeros_like(b_o)
    for k, c in enumerate(comps):
        b3[c] = np.roll(b_o[0], 5 * k, axis=2)           # mean-free profiles in the chosen components
    ref = O.solve(ph_o, p.phases, p.c0, b3, p.mean_strain, tol=0.0, maxit=9, history=True)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    dt = torch.float64 if precision == "fp64" else torch.float32
    b = torch.tensor(b3, dtype=dt, device="cuda")
    for sparse in (False, True):
        with api.Plan(p.dims, precision, sparse_resid=sparse) as plan:
            eps, sig, u, info = plan.solve(ph, p.phases, p.c0, b, p.mean_strain, tol=0.0, maxit=9)
            hist = plan.history()
        for got, key in ((eps, "eps"), (sig, "sig"), (u, "u")):
            assert rel(got.cpu().numpy(), ref[key]) < TOL[precision], (comps, sparse, key)
        ev = ~np.isnan(hist)
        h_ref = np.array(ref["hist"])
        assert np.all(np.abs(hist[ev] - h_ref[ev]) <= 1e-4 * h_ref[ev] + (1e-12 if precision == "fp64" else 1e-6))
