"""The comparison sweeps around a library FFT (libfft_sweeps: bfcs_polarize and
bfcs_green_apply with torch.fft's transforms) against the FP64 oracle at a fixed
sweep count (Algorithm 1, Eqs. 5.7-5.10), and the residual numerator of
Eq. 5.11 (reading R4) from bfcs_green_apply against the oracle's residual."""
import numpy as np
import pytest
import torch

from oracle import bfcs_oracle as O
from paper_2601_00822_gb300 import api, workloads as W
from paper_2601_00822_gb300.libfft_sweeps import LibFftSweeps

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a, np.float64) - b).ravel()) / np.linalg.norm(b.ravel()))


def _case(name):
    if name == "c1_32cubed":
        return W.config_c1()
    return W.Problem(name="ragged", dims=(48, 24, 96), cell=(24, 12, 32),
                     spheres=np.asarray([[24, 12, 30, 90, 1], [3, 20, 60, 40, 2]], dtype=np.int32),
                     phases=[(1.0, 0.5), (6.0, 3.0), (0.5, 0.3)],
                     c0=W.reference_medium([(1.0, 0.5), (6.0, 3.0), (0.5, 0.3)]),
                     bf_centre=(24.0, 12.0, 48.0), bf_radius=7.0, mean_strain=(0.01, 0, -0.002, 0, 0.003, 0))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["c1_32cubed", "ragged_48x24x96"])
def test_library_fft_sweeps_match_the_oracle(name, precision):
    p = _case(name)
    sweeps = 7
    ph_o = O.phase_map(p.dims, p.cell, p.spheres)
    b_o = O.body_force(p.dims, p.bf_centre, p.bf_radius)
    ref = O.solve(ph_o, p.phases, p.c0, b_o, p.mean_strain, tol=0.0, maxit=sweeps, history=True)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, precision)
    with api.Plan(p.dims, precision) as plan:
        s = LibFftSweeps(plan, ph, p.phases, p.c0, b, p.mean_strain)
        nums = []
        for _ in range(sweeps):
            s.sweep()
            nums.append(float(s.num.item()))
        eps = s.eps.cpu().numpy()
    assert rel(eps, ref["eps"]) < TOL[precision]
    # residual of eps^s (Eq. 5.11, reading R4): numerator from the Green step,
    # denominator ||b_hat|| + xi_min |sigma_hat(0)| evaluated here from the oracle's fields
    xi = O.wavevectors(p.dims)
    b_hat = O.fft3(b_o)
    act = (xi[0] ** 2 + xi[1] ** 2 + xi[2] ** 2) > 0
    bden = np.sqrt(np.sum(np.abs(b_hat[:, np.broadcast_to(act, b_hat.shape[1:])]) ** 2))
    eps_s = O.solve(ph_o, p.phases, p.c0, b_o, p.mean_strain, tol=0.0, maxit=0)["eps"]
    for k in range(sweeps):
        s0 = O.fft3(O.apply_local(ph_o, p.phases, eps_s))[:, 0, 0, 0]
        s0n = np.sqrt(np.sum(np.abs(s0[:3]) ** 2) + 2 * np.sum(np.abs(s0[3:]) ** 2))
        r = np.sqrt(nums[k]) / (bden + 2 * np.pi / max(p.dims) * s0n)
        t = 1e-4 if precision == "fp32" else 1e-9
        assert abs(r - ref["hist"][k]) <= t * ref["hist"][k] + (1e-6 if precision == "fp32" else 1e-13), k
        eps_s = O.solve(ph_o, p.phases, p.c0, b_o, p.mean_strain, tol=0.0, maxit=k + 1)["eps"]


def test_library_fft_sweeps_equal_fused_sweeps_at_256():
    """At the benchmarked size the comparison sweeps and the fused sweeps give the
    same strain after five sweeps (FP32 rounding only)."""
    p = W.config_c2(contrast=10.0, seed=1)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp32")
    with api.Plan(p.dims, "fp32") as plan:
        eps, _, _, _ = plan.solve(ph, p.phases, p.c0, b, tol=0.0, maxit=5, want_sig=False, want_u=False)
        s = LibFftSweeps(plan, ph, p.phases, p.c0, b)
        for _ in range(5):
            s.sweep()
        err = float(torch.linalg.vector_norm(s.eps - eps) / torch.linalg.vector_norm(eps))
    assert err < 1e-5, err
