"""GPU parity of the ensemble dataset D^d (Eq. 3.8) through bfcs_ensemble_average:
against the FP64 oracle on three unrelated 32^3 configurations (fixed sweep
counts in FP64 and FP32, ragged batches, and converged through the mixed
ladder); against the translated average for translated copies; and at 256^3
the exact mirror symmetry of a configuration pair about the load plane."""
import numpy as np
import pytest
import torch

from oracle import bfcs_oracle as O
from paper_2601_00822_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu

PHASES = [(1.0, 0.5), (8.0, 4.0), (0.3, 0.15)]
C0 = W.reference_medium(PHASES)
DIMS = (32, 32, 32)
CENTRE, A = (16.0, 16.0, 16.0), 7.0


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0)


def configs_np():
    out = []
    for seed, ph_id in ((11, 1), (12, 2), (13, 1)):
        sph = W.rsa_spheres((32, 32, 32), 0.2, 3.0, 5.0, seed, max_tries=2000, phase=ph_id)
        out.append(O.phase_map(DIMS, (32, 32, 32), sph))
    planes = (out[2] == 0) & (np.arange(32)[None, None, :] % 7 == 0)
    out[2][planes] = 2                       # a third phase in thin planes of the matrix
    return out


@pytest.mark.parametrize("precision,max_batch,bar", [("fp64", 2, 1e-10), ("fp64", 3, 1e-10), ("fp32", 2, 1e-5)])
def test_fixed_sweeps_against_oracle(precision, max_batch, bar):
    cfg = configs_np()
    b_o = O.body_force(DIMS, CENTRE, A)
    ref, hits_ref, _ = O.ensemble_average(cfg, PHASES, C0, b_o, tol=0, maxit=12)
    confs = [torch.from_numpy(c).cuda() for c in cfg]
    b = api.body_force(DIMS, CENTRE, A, precision)
    with api.Plan(DIMS, precision, max_batch=max_batch) as plan:
        avg, hits, infos = plan.ensemble_average(confs, PHASES, C0, b, tol=0, maxit=12)
    assert [i.iters for i in infos] == [12, 12, 12]
    assert np.array_equal(hits.cpu().numpy(), hits_ref)
    avg = avg.cpu().numpy()
    for a0, a1 in ((0, 3), (3, 6), (6, 12), (12, 18), (18, 24), (24, 30)):
        assert rel(avg[a0:a1], ref[a0:a1]) < bar, (a0, a1)


def test_converged_mixed_against_oracle():
    cfg = configs_np()
    b_o = O.body_force(DIMS, CENTRE, A)
    ref, _, _ = O.ensemble_average(cfg, PHASES, C0, b_o, tol=1e-12, maxit=4000)
    confs = [torch.from_numpy(c).cuda() for c in cfg]
    b = api.body_force(DIMS, CENTRE, A, "fp64")
    with api.Plan(DIMS, "mixed", max_batch=3) as plan:
        avg, _, infos = plan.ensemble_average(confs, PHASES, C0, b, tol=1e-10, maxit=4000)
    assert all(i.status == _lib.OK and i.resid <= 1e-10 for i in infos)
    avg = avg.cpu().numpy()
    for a0, a1 in ((0, 3), (3, 6), (6, 12), (12, 18), (18, 24), (24, 30)):
        assert rel(avg[a0:a1], ref[a0:a1]) < 1e-8, (a0, a1)


def test_translated_copies_equal_the_translated_average():
    p = W.config_c1()
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp32")
    shifts = [(0, 0, 0), (5, 1, 3), (9, 12, 2), (15, 15, 15)]
    confs = [torch.roll(ph, shifts=(s[2], s[1], s[0]), dims=(0, 1, 2)).contiguous() for s in shifts]
    with api.Plan(p.dims, "fp32", max_batch=4) as plan:
        avg_t, hits_t, _ = plan.translate_average(ph, p.phases, p.c0, b, shifts, tol=0, maxit=15)
        avg_e, hits_e, _ = plan.ensemble_average(confs, p.phases, p.c0, b, tol=0, maxit=15)
    assert torch.equal(hits_t, hits_e)
    assert rel(avg_e.cpu().numpy(), avg_t.cpu().numpy()) < 1e-14


def test_full_size_mirror_pair_is_symmetric():
    """C2's 256^3 microstructure X and its mirror image about the load plane
    x = 128, mixed ladder to residual 1e-8: the pair's averages are symmetric
    under the reflection (vectors: x component odd; tensors: xz, xy odd)."""
    p = W.config_c2(contrast=10.0, seed=1)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    ph[:, :, 160:] = 0                       # no inclusions at x >= 160: X itself is not symmetric
    refl = torch.flip(ph, dims=[2]).contiguous()
    b = api.body_force(p.dims, p.bf_centre, p.bf_radius, "fp64")
    with api.Plan(p.dims, "mixed", max_batch=2) as plan:
        avg, hits, infos = plan.ensemble_average([ph, refl], p.phases, p.c0, b, tol=1e-8, maxit=20000)
    assert all(i.status == _lib.OK for i in infos)
    assert torch.equal(hits, torch.flip(hits, dims=[2]))
    vec = torch.tensor([-1.0, 1.0, 1.0], dtype=torch.float64, device="cuda")[:, None, None, None]
    ten = torch.tensor([1.0, 1.0, 1.0, 1.0, -1.0, -1.0], dtype=torch.float64, device="cuda")[:, None, None, None]
    for lo, sign in ((0, vec), (3, vec), (6, ten), (12, ten), (18, ten), (24, ten)):
        f = avg[lo:lo + sign.shape[0]]
        err = (torch.flip(f, dims=[3]) - sign * f).abs().max().item()
        assert err <= 1e-6 * f.abs().max().item(), lo
