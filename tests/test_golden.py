"""Hand-derived values under tests/golden/, each fixture citing the equations it
evaluates: the oracle (CPU) and the CUDA path (GPU) against the same numbers.

* bfcs_field_4cubed_a2.txt - the BFCS load of Eq. 2.5 at voxel centres, exact
  binary fractions (both sides must reproduce them bit for bit);
* green_u0_isotropic.txt - U0 = -Gamma0 of Eqs. 2.16-2.18 on unit polarizations
  at two wavevector directions and two reference media;
* laminate_two_phase_e11.txt - the exact solution of a two-phase laminate under a
  prescribed mean strain (Eqs. 2.1-2.3, 2.24).
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import bfcs_oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
COMPS = ("xx", "yy", "zz", "yz", "xz", "xy")


def rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [line.split() for line in f if line.strip() and not line.startswith("#")]


def num(tok):
    return float(Fraction(tok))


def golden_field():
    b = np.zeros((3, 4, 4, 4))
    for x, y, z, v in rows("bfcs_field_4cubed_a2.txt"):
        b[0, int(z), int(y), int(x)] = int(v) / 1024.0
    return b


LAMINATE_DIMS = (8, 4, 4)
LAMINATE_E = (0.011, 0.0, 0.0, 0.0, 0.0, 0.0)


def laminate():
    """Phase ids (A = 0 on x = 0..3, B = 1 on x = 4..7), the phase table and the
    expected per-phase strain and stress (6 components each)."""
    nx, ny, nz = LAMINATE_DIMS
    layers = np.array([0] * 4 + [1] * 4, dtype=np.int8)
    phase = np.broadcast_to(layers[None, None, :], (nz, ny, nx)).copy()
    table, eps, sig = [], [], []
    for r in rows("laminate_two_phase_e11.txt"):
        table.append((num(r[1]), num(r[2])))
        eps.append([num(r[3]), num(r[4]), num(r[5]), 0.0, 0.0, 0.0])
        sig.append([num(r[6]), num(r[7]), num(r[8]), 0.0, 0.0, 0.0])
    eps, sig = np.array(eps).T, np.array(sig).T        # (6 components, 2 phases)
    return phase, table, eps[:, layers][:, None, None, :], sig[:, layers][:, None, None, :]


# ------------------------------------------------------------------ oracle (CPU)
def test_golden_files_are_complete():
    assert len(rows("bfcs_field_4cubed_a2.txt")) == 32
    assert len(rows("green_u0_isotropic.txt")) == 13
    assert len(rows("laminate_two_phase_e11.txt")) == 2


def test_oracle_bfcs_field_is_the_hand_evaluation_of_eq_2_5():
    b = O.body_force((4, 4, 4), (2.0, 2.0, 2.0), 2.0)
    assert np.array_equal(b, golden_field())


def test_oracle_bfcs_field_wraps_periodically():
    """The same load centred at the grid corner: every offset beyond half a
    period wraps to its minimum image, so the field is the fixture rolled by two
    voxels along each axis (voxel i sits where voxel (i + 2) mod 4 sat)."""
    b = O.body_force((4, 4, 4), (0.0, 0.0, 0.0), 2.0)
    assert np.array_equal(b, np.roll(golden_field(), 2, axis=(1, 2, 3)))


def test_oracle_u0_is_the_hand_evaluation_of_eqs_2_16_2_18():
    for r in rows("green_u0_isotropic.txt"):
        lam0, mu0 = num(r[0]), num(r[1])
        xi = tuple(np.array([[[num(v)]]]) for v in r[2:5])
        tau = np.zeros((6, 1, 1, 1), dtype=complex)
        tau[COMPS.index(r[5])] = 1.0          # tensorial: tau_ij = tau_ji = 1
        out = O.u0_apply(tau, xi, lam0, mu0)[:, 0, 0, 0]
        want = np.array([num(v) for v in r[6:12]])
        assert np.allclose(out.real, want, rtol=0, atol=1e-15), (r, out.real)
        assert np.all(out.imag == 0)


def test_oracle_laminate_is_the_exact_solution():
    phase, table, eps, sig = laminate()
    nx, ny, nz = LAMINATE_DIMS
    res = O.solve(phase, table, (5.5, 2.75), np.zeros((3, nz, ny, nx)), LAMINATE_E, tol=1e-14, maxit=5000)
    assert res["resid"] < 1e-14
    assert np.allclose(res["eps"], np.broadcast_to(eps, res["eps"].shape), rtol=0, atol=1e-14)
    assert np.allclose(res["sig"], np.broadcast_to(sig, res["sig"].shape), rtol=0, atol=1e-14)


# ------------------------------------------------------------------ CUDA path (GPU)
@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gpu_bfcs_field_is_the_hand_evaluation_of_eq_2_5(precision):
    from paper_2601_00822_gb300 import api
    b = api.body_force((4, 4, 4), (2.0, 2.0, 2.0), 2.0, precision).cpu().numpy()
    want = golden_field()
    if precision == "fp64":
        assert np.array_equal(b, want)
    else:       # k/1024 with |k| < 2^10 is exact in binary32 too
        assert np.array_equal(b.astype(np.float64), want)
    # centred at the grid corner: the minimum images wrap around the period
    bc = api.body_force((4, 4, 4), (0.0, 0.0, 0.0), 2.0, precision).cpu().numpy().astype(np.float64)
    assert np.array_equal(bc, np.roll(want, 2, axis=(1, 2, 3)))


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol,bar", [("fp64", 1e-13, 1e-12), ("mixed", 1e-12, 1e-11),
                                               ("fp32", 1e-5, 1e-4)])
def test_gpu_laminate_is_the_exact_solution(precision, tol, bar):
    """Solved to the residual `tol`; in this layered medium the relative error of
    the axial stress is bounded by the residual (its fluctuation is what Eq. 5.11
    measures), so `bar` = 10 tol relative to the field values (0.02 and 0.04)."""
    import torch
    from paper_2601_00822_gb300 import _lib, api
    phase, table, eps, sig = laminate()
    nx, ny, nz = LAMINATE_DIMS
    ph = torch.tensor(phase, device="cuda")
    dt = torch.float32 if precision == "fp32" else torch.float64
    b = torch.zeros((3, nz, ny, nx), dtype=dt, device="cuda")
    with api.Plan(LAMINATE_DIMS, precision) as plan:
        e, s, _, info = plan.solve(ph, table, (5.5, 2.75), b, LAMINATE_E, tol=tol, maxit=5000)
    assert info.status == _lib.OK
    e, s = e.cpu().numpy().astype(np.float64), s.cpu().numpy().astype(np.float64)
    assert np.allclose(e, np.broadcast_to(eps, e.shape), rtol=0, atol=bar * 0.02)
    assert np.allclose(s, np.broadcast_to(sig, s.shape), rtol=0, atol=bar * 0.04)
