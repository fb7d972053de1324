"""GPU parity of the nonlocal kernel regression (Eqs. 6.5-6.6, displacement
operator Gamma = -b): bfcs_kernel_apply against the oracle's direct sums over
the horizon; bfcs_kernel_fit against the oracle's Gram matrix, right-hand side,
exact minimiser and Adam iterate; end to end on a translated-averaging dataset
that each side computes itself; and at 256^3 the recovery of a planted kernel
and the agreement of the fitted loss with a direct evaluation."""
import numpy as np
import pytest
import torch

from oracle import bfcs_oracle as O
from paper_2601_00822_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(6056)


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("delta,coef", [(3.5, [0.4, -1.1, 0.3, 2.2, -0.7, 1.0]), (2.0, [1.0, 0.5])])
def test_apply_against_direct_sums(precision, delta, coef):
    dims = (24, 16, 32)
    u = RNG.standard_normal((3, dims[2], dims[1], dims[0]))
    ref = O.kernel_operator(u, coef, delta)
    with api.Plan(dims, precision) as plan:
        out = plan.kernel_apply(coef, delta, torch.tensor(u, device="cuda")).cpu().numpy()
    assert rel(out, ref) < 1e-12


def test_fit_against_oracle():
    dims = (16, 16, 16)
    us = [RNG.standard_normal((3, 16, 16, 16)) for _ in range(2)]
    gs = [RNG.standard_normal((3, 16, 16, 16)) + O.kernel_operator(u, [1.0, -0.5, 0.8, 0.2, -1.0], 3.0)
          for u in us]
    ref = O.kernel_fit(us, gs, 3.0, 4, lam=1e-2, iters=500, lr=0.02)
    with api.Plan(dims, "fp64") as plan:
        fit = plan.kernel_fit([torch.tensor(u, device="cuda") for u in us],
                              [torch.tensor(g, device="cuda") for g in gs], 3.0, 4, lam=1e-2, iters=500, lr=0.02)
    assert rel(fit["G"], ref["G"]) < 1e-12 and rel(fit["g"], ref["g"]) < 1e-12
    assert rel(fit["exact"], ref["exact"]) < 1e-8
    assert rel(fit["coef"], ref["coef"]) < 1e-8
    assert abs(fit["loss"] - ref["loss"]) <= 1e-9 * ref["s"]
    assert fit["exact_loss"] <= fit["loss"] * (1 + 1e-12)


def test_end_to_end_on_translated_averages():
    """D^p of two BFCS loads (C1's microstructure at 16^3: one 16^3 cell, R = 5
    sphere, contrast 10; a = 4 and a = 5.5 about the centre), 4 shifts each,
    computed by each side; Gamma_k = -b_k; degree 5, horizon 4."""
    p = W.config_c1()
    dims, cell = (16, 16, 16), (16, 16, 16)
    shifts = [(0, 0, 0), (4, 0, 0), (0, 8, 4), (12, 4, 8)]
    loads = [((8.0, 8.0, 8.0), 4.0), ((8.0, 8.0, 8.0), 5.5)]
    ph_o = O.phase_map(dims, cell, p.spheres)
    us_o, gs_o = [], []
    for c, a in loads:
        b = O.body_force(dims, c, a)
        avg, _, _ = O.translate_average(ph_o, p.phases, p.c0, b, shifts, tol=1e-12, maxit=4000)
        us_o.append(avg[0:3])
        gs_o.append(-b)
    ref = O.kernel_fit(us_o, gs_o, 4.0, 5, lam=1e-6, iters=2000, lr=0.05)
    ph = api.voxelize(dims, cell, p.spheres)
    us, gs = [], []
    with api.Plan(dims, "fp64", max_batch=4) as plan:
        for c, a in loads:
            b = api.body_force(dims, c, a, "fp64")
            avg, _, infos = plan.translate_average(ph, p.phases, p.c0, b, shifts, tol=1e-11, maxit=4000)
            assert all(i.status == _lib.OK for i in infos)
            us.append(avg[0:3].contiguous())
            gs.append((-b).contiguous())
        fit = plan.kernel_fit(us, gs, 4.0, 5, lam=1e-6, iters=2000, lr=0.05)
    assert rel(fit["G"], ref["G"]) < 1e-8 and rel(fit["g"], ref["g"]) < 1e-8
    assert rel(fit["exact"], ref["exact"]) < 1e-5
    assert fit["exact_loss"] < 0.9 * ref["s"]            # the kernel explains part of the load


def test_full_size_planted_kernel_and_loss():
    n = 256
    c_true = [0.9, -0.4, 1.3, 0.1, -0.6]
    gen = torch.Generator(device="cuda").manual_seed(11)
    with api.Plan((n, n, n), "fp64") as plan:
        us = [torch.randn((3, n, n, n), dtype=torch.float64, device="cuda", generator=gen) for _ in range(2)]
        gs = [plan.kernel_apply(c_true, 3.0, u) for u in us]
        fit = plan.kernel_fit(us, gs, 3.0, 4, lam=0.0, iters=200, lr=0.02)
        assert np.allclose(fit["exact"], c_true, rtol=1e-6, atol=1e-8)
        # the Parseval loss of the Adam iterate against a direct evaluation through the operator
        direct = sum(float(((plan.kernel_apply(fit["coef"], 3.0, u) - g) ** 2).sum()) for u, g in zip(us, gs))
        assert abs(direct - fit["loss"]) <= 1e-8 * sum(float((g * g).sum()) for g in gs)


def test_kernel_fit_argument_errors():
    u = torch.zeros((3, 16, 16, 16), dtype=torch.float64, device="cuda")
    with api.Plan((16, 16, 16), "fp32") as plan:                # FP32 plans have no FP64 transforms
        with pytest.raises(RuntimeError):
            plan.kernel_apply([1.0, 1.0], 2.0, u)
    with api.Plan((16, 16, 16), "fp64") as plan:
        with pytest.raises(RuntimeError):
            plan.kernel_apply([1.0, 1.0], 8.0, u)                # 2 delta must stay below the grid
        with pytest.raises(RuntimeError):
            plan.kernel_fit([u], [u], 2.0, 8)                    # degree above 7
        out = plan.kernel_apply([1.0, -2.0, 0.5], 2.5, u)        # zero field -> zero operator
        assert float(out.abs().max()) == 0.0
