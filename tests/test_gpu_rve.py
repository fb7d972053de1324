"""GPU parity of the RVE diagnostic and the RVE-size loop (Def. 2.2, Sec. 5):
bfcs_radial_profile against the oracle's shell maxima on seeded fields
(bit-exact shell counts), bfcs_rve_size against the oracle's loop on the two
cases its pins fix (a loop that rejects then accepts, and one the annulus
decides), and at full size the loop's decisions against its own profiles and
the stabilisation of the strain inside the accepted RVE on a 256^3 grid."""
import numpy as np
import pytest
import torch

from oracle import bfcs_oracle as O
from paper_2601_00822_gb300 import _lib, api, workloads as W

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(20261203)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("ncomp", [3, 6])
def test_radial_profile_against_oracle(precision, ncomp):
    dims = (48, 24, 96)
    centre = (24.5, 12.0, 40.0)
    f = RNG.standard_normal((ncomp, dims[2], dims[1], dims[0]))
    dt = torch.float32 if precision == "fp32" else torch.float64
    ft = torch.tensor(f, dtype=dt, device="cuda")
    ref, cnt = O.radial_profile(ft.double().cpu().numpy(), centre, 30)
    with api.Plan(dims, precision) as plan:
        prof, counts = plan.radial_profile(ft, centre, 30)
    assert np.array_equal(counts, cnt)
    assert np.allclose(prof, ref, rtol=1e-15, atol=0)


SMALL = dict(cell=(8, 8, 8), spheres=np.asarray([[8, 8, 8, 25, 1]], np.int32), phases=[(1.0, 0.5), (6.0, 3.0)],
             c0=(3.5, 1.75))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-10)])
@pytest.mark.parametrize("a,tol_f,sizes", [(3.0, 0.05, (16, 24, 32)), (4.0, 0.048, (24, 32))])
def test_rve_loop_against_oracle(precision, tol, a, tol_f, sizes):
    ref = O.rve_size(SMALL["cell"], SMALL["spheres"], SMALL["phases"], SMALL["c0"], a, sizes, tol=1e-12,
                     tol_f=tol_f)
    recs, prof, acc = api.rve_size(SMALL["cell"], SMALL["spheres"], SMALL["phases"], SMALL["c0"], a, sizes,
                                   precision=precision, tol=tol, maxit=4000, tol_f=tol_f)
    assert [(r["n"], r["r_rve"], r["contained"]) for r in recs] == \
        [(r["n"], r["r_rve"], r["contained"]) for r in ref]
    assert acc == len(ref) - 1 and ref[-1]["contained"]
    for i, (g, o) in enumerate(zip(recs, ref)):
        assert g["centre"] == o["centre"] and g["status"] == _lib.OK
        m = g["n"] // 2
        assert np.abs(prof[i, 0, :m] - o["prof_eps"]).max() <= 1e-8 * o["prof_eps"].max()
        assert np.abs(prof[i, 1, :m] - o["prof_sig"]).max() <= 1e-8 * o["prof_sig"].max()


def test_full_size_loop_decisions_and_stabilisation():
    """C2's microstructure (32^3 cells, RSA vf 0.25, contrast 10), support
    radius a = 8, field tolerance 5%, grids 64, 128, 256 (mixed ladder to 1e-6):
    each step's radius follows from its own profiles, the loop stops at the
    first grid that holds RVE + a/2, and the strain inside that RVE agrees with
    the 256^3 solution within the field tolerance."""
    p = W.config_c2(contrast=10.0, seed=1)
    a, tol_f, sizes = 8.0, 0.05, (64, 128, 256)
    recs, prof, acc = api.rve_size(p.cell, p.spheres, p.phases, p.c0, a, sizes, precision="mixed", tol=1e-6,
                                   tol_f=tol_f)
    assert acc >= 0 and acc == len(recs) - 1
    for i, r in enumerate(recs):
        m = r["n"] // 2
        rr = O.rve_radius([prof[i, 0, :m], prof[i, 1, :m]], tol_f, m)      # the rule, applied to the GPU's profiles
        assert r["r_rve"] == rr and r["status"] == _lib.OK
        assert r["contained"] == (rr is not None and rr + a / 2 <= m)
        assert r["contained"] == (i == acc)
    n, r = recs[acc]["n"], recs[acc]["r_rve"]
    assert n < 256, "the RVE should fit below the largest grid"

    def strain(nn):
        ph = api.voxelize((nn,) * 3, p.cell, p.spheres)
        c = recs[acc]["centre"] if nn == n else tuple(float(k * np.floor(nn / (2.0 * k) + 0.5)) for k in p.cell)
        b = api.body_force((nn,) * 3, c, a, "fp64")
        with api.Plan((nn,) * 3, "mixed") as plan:
            eps, _, _, info = plan.solve(ph, p.phases, p.c0, b, tol=1e-6, maxit=20000, want_sig=False, want_u=False)
        assert info.status == _lib.OK
        return eps, int(c[0])

    (ea, ca), (eb, cb) = strain(n), strain(256)
    g = torch.arange(-r, r, device="cuda")
    ball = ((g[:, None, None] + 0.5) ** 2 + (g[None, :, None] + 0.5) ** 2 + (g[None, None, :] + 0.5) ** 2) < r * r

    def window(e, c, nn):
        idx = (c + g) % nn
        return e[:, idx][:, :, idx][:, :, :, idx]

    diff = (window(ea, ca, n) - window(eb, cb, 256)).abs()[:, ball].max().item()
    assert diff <= tol_f * ea.abs().max().item(), diff


def test_radial_profile_argument_errors():
    with api.Plan((16, 16, 16), "fp64") as plan:
        f = torch.zeros((6, 16, 16, 16), dtype=torch.float64, device="cuda")
        with pytest.raises(RuntimeError):
            plan.radial_profile(f, (8.25, 8.0, 8.0), 8)        # not on the half-voxel lattice
        with pytest.raises(RuntimeError):
            plan.radial_profile(f, (8.0, 8.0, 8.0), 0)         # no shells
        with pytest.raises(RuntimeError):
            plan.radial_profile(f, (8.0, 8.0, 8.0), 4096)      # more shells than the kernel keeps
        prof, counts = plan.radial_profile(f, (-8.0, 24.0, 8.5), 8)   # centres wrap periodically
        assert np.all(prof == 0) and counts.sum() > 0
