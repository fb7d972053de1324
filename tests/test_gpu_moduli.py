"""GPU parity of the effective stiffness L* (Eqs. 6.1-6.3) and the inclusion
strain concentration A* (Eq. 3.2) through bfcs_effective_stiffness.

Against the FP64 oracle on config C1 (32^3, contrast 10); against the closed
forms of a laminate; and, at 256^3, against properties that hold at any size:
symmetry and positive definiteness of L*, the Voigt and Reuss bounds, and the
two-phase identity <sigma> = L_m E + f (L_i - L_m) <eps>_i.
"""
import functools

import numpy as np
import pytest
import torch

from oracle import bfcs_oracle as O
from paper_2601_00822_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu

VOIGT = np.diag([1.0, 1.0, 1.0, 0.5, 0.5, 0.5])   # tensorial response -> symmetric (Voigt) form


def stiffness_matrix(lam, mu):
    M = np.zeros((6, 6))
    M[:3, :3] = lam
    for i in range(3):
        M[i, i] = lam + 2 * mu
    for i in range(3, 6):
        M[i, i] = 2 * mu
    return M


@functools.lru_cache(maxsize=None)
def oracle_c1():
    p = W.config_c1()
    ph = O.phase_map(p.dims, p.cell, p.spheres)
    return O.effective_moduli(ph, p.phases, p.c0, tol=1e-12)


def gpu_moduli(p, precision, tol, max_batch=6, maxit=20000, phase=None, cg=False):
    ph = api.voxelize(p.dims, p.cell, p.spheres) if phase is None else phase
    plan = api.Plan(p.dims, precision=precision, max_batch=max_batch, cg=cg)
    try:
        return plan.effective_stiffness(ph, p.phases, p.c0, tol=tol, maxit=maxit)
    finally:
        plan.close()


@pytest.mark.parametrize("precision,tol,bar", [("fp64", 1e-11, 1e-8), ("mixed", 1e-11, 1e-8),
                                               ("fp32", 1e-5, 2e-4)])
def test_c1_against_oracle(precision, tol, bar):
    Lo, Ao = oracle_c1()
    Ls, As, infos = gpu_moduli(W.config_c1(), precision, tol)
    assert all(i.status == _lib.OK for i in infos)
    assert np.abs(Ls - Lo).max() <= bar * np.abs(Lo).max()
    assert np.abs(As - Ao).max() <= bar * np.abs(Ao).max()


def test_c1_chunks_and_cg_agree():
    Lo, Ao = oracle_c1()
    p = W.config_c1()
    L6, A6, _ = gpu_moduli(p, "fp64", 1e-11, max_batch=6)
    L4, A4, _ = gpu_moduli(p, "fp64", 1e-11, max_batch=4)      # chunks of 4 + 2 members
    assert np.abs(L4 - L6).max() <= 1e-13 * np.abs(L6).max()
    assert np.abs(A4 - A6).max() <= 1e-13 * np.abs(A6).max()
    Lc, Ac, infos = gpu_moduli(p, "fp64", 1e-11, cg=True)
    assert all(i.status == _lib.OK for i in infos)
    assert np.abs(Lc - Lo).max() <= 1e-8 * np.abs(Lo).max()
    assert np.abs(Ac - Ao).max() <= 1e-8 * np.abs(Ao).max()


def _laminate_uniaxial(comp, target):
    n = comp.size
    alt = (-1.0) ** np.arange(n)
    A = np.array([[comp.sum(), (alt * comp).sum()], [(alt * comp).sum(), (alt * alt * comp).sum()]])
    c0, c1 = np.linalg.solve(A, np.array([n * target, 0.0]))
    return c0 + c1 * alt


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-9), ("fp32", 1e-5)])
def test_laminate_closed_forms(precision, bar):
    layers = np.array([0, 1, 1, 0, 0, 0, 1, 0, 1, 1, 1, 0], dtype=np.int8)
    nx, ny, nz = layers.size, 4, 4
    lam_ph, mu_ph = np.array([1.0, 8.0]), np.array([0.6, 4.0])
    phase = torch.from_numpy(np.broadcast_to(layers[None, None, :], (nz, ny, nx)).copy()).cuda()
    p = W.Problem(name="laminate", dims=(nx, ny, nz), cell=(nx, ny, nz), spheres=np.zeros((0, 5), np.int32),
                  phases=list(zip(lam_ph, mu_ph)), c0=(4.5, 2.3), bf_centre=(0.0, 0.0, 0.0), bf_radius=1.0)
    tol = 1e-12 if precision == "fp64" else 1e-6
    Ls, As, infos = gpu_moduli(p, precision, tol, phase=phase)
    lam, mu = lam_ph[layers], mu_ph[layers]
    incl = layers != 0
    s_xx = _laminate_uniaxial(1.0 / (lam + 2 * mu), 1.0)
    e_xx = s_xx / (lam + 2 * mu)
    s_xy = _laminate_uniaxial(1.0 / (2 * mu), 1.0)
    scale = np.abs(Ls).max()
    assert abs(Ls[0, 0] - s_xx.mean()) <= bar * scale
    assert abs(Ls[1, 0] - (lam * e_xx).mean()) <= bar * scale
    assert abs(Ls[3, 3] - 2 * mu.mean()) <= bar * scale
    assert abs(Ls[5, 5] - s_xy.mean()) <= bar * scale
    assert abs(As[0, 0] - e_xx[incl].mean()) <= bar
    assert abs(As[3, 3] - 1.0) <= bar
    assert abs(As[5, 5] - (s_xy / (2 * mu))[incl].mean()) <= bar


def test_homogeneous_cell_without_inclusions():
    p = W.Problem(name="hom", dims=(16, 16, 16), cell=(16, 16, 16), spheres=np.zeros((0, 5), np.int32),
                  phases=[(1.7, 0.9), (5.0, 2.0)], c0=(3.0, 1.5), bf_centre=(0.0, 0.0, 0.0), bf_radius=1.0)
    phase = torch.zeros((16, 16, 16), dtype=torch.int8, device="cuda")
    Ls, As, _ = gpu_moduli(p, "fp64", 1e-12, phase=phase)
    assert np.abs(Ls - stiffness_matrix(1.7, 0.9)).max() <= 1e-12
    assert np.isnan(As).all()


def test_full_size_c2_properties():
    """256^3 RSA microstructure at contrast 10 (mixed precision, tol 1e-6)."""
    p = W.config_c2(contrast=10.0, seed=1)
    ph = api.voxelize(p.dims, p.cell, p.spheres)
    Ls, As, infos = gpu_moduli(p, "mixed", 1e-6, phase=ph)
    assert all(i.status == _lib.OK and i.resid <= 1e-6 for i in infos)
    S = Ls @ VOIGT
    assert np.abs(S - S.T).max() <= 1e-4 * np.abs(S).max()
    S = 0.5 * (S + S.T)
    assert np.linalg.eigvalsh(S).min() > 0
    f = float((ph != 0).double().mean())
    L0, L1 = stiffness_matrix(*p.phases[0]), stiffness_matrix(*p.phases[1])
    voigt = ((1 - f) * L0 + f * L1) @ VOIGT
    reuss = np.linalg.inv((1 - f) * np.linalg.inv(L0 @ VOIGT) + f * np.linalg.inv(L1 @ VOIGT))
    assert np.linalg.eigvalsh(voigt - S).min() > 0
    assert np.linalg.eigvalsh(S - reuss).min() > 0
    assert np.abs(Ls - (L0 + f * (L1 - L0) @ As)).max() <= 1e-10 * np.abs(Ls).max()
    # cubic symmetry of the cell average is only statistical; the isotropic parts are close
    assert np.std(np.diag(Ls)[:3]) <= 0.05 * np.mean(np.diag(Ls)[:3])
