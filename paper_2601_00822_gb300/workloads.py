"""Seeded synthetic inputs for the BFCS solver.

This module holds no arithmetic of the solution method: it only draws and
describes inputs (sphere lists in a periodic unit cell, per-phase Lame
constants, the reference medium, the body-force centre and radius).  Both the
CUDA path and the FP64 oracle consume what it returns; each side turns it into
a phase map and a body-force field with its own code.

Sphere encoding (integer, so that voxelisation is exact on both sides):
  row = (X, Y, Z, T, phase) with X = 2*cx, Y = 2*cy, Z = 2*cz the doubled
  centre in cell coordinates (half-voxel resolution) and T = floor((2R)^2) the
  squared doubled radius.  Voxel centres sit at i + 0.5, i.e. doubled 2i + 1.

The random generator is SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), a public-domain counter-based
mixer; its output is mapped to [0, 1) with the top 53 bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream: state += golden gamma, then two xor-shift-multiply rounds."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


def lame_from_young(young: float, nu: float) -> tuple[float, float]:
    """Isotropic Lame constants (lambda, mu) from Young's modulus and Poisson's ratio."""
    lam = young * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = young / (2.0 * (1.0 + nu))
    return lam, mu


def reference_medium(phases: list[tuple[float, float]]) -> tuple[float, float]:
    """C0 = (Cmin + Cmax)/2 taken componentwise on (lambda, mu)."""
    lams = [p[0] for p in phases]
    mus = [p[1] for p in phases]
    return 0.5 * (min(lams) + max(lams)), 0.5 * (min(mus) + max(mus))


def sphere_row(cx: float, cy: float, cz: float, radius: float, phase: int = 1) -> list[int]:
    """Encode one sphere; the centre is rounded to the nearest half voxel."""
    return [int(round(2 * cx)), int(round(2 * cy)), int(round(2 * cz)),
            int(math.floor(4.0 * radius * radius)), int(phase)]


def rsa_spheres(cell: tuple[int, int, int], vf: float, rmin: float, rmax: float,
                seed: int, max_tries: int = 200000, phase: int = 1) -> np.ndarray:
    """Random sequential addition of non-overlapping spheres in a periodic cell.

    Radii are uniform in [rmin, rmax], centres uniform in the cell (rounded to
    half voxels).  Overlap uses the periodic minimum image on the doubled
    integer grid with a gap of one voxel.  Addition stops once the continuous
    volume fraction sum(4/3 pi R^3)/|cell| reaches vf.
    """
    rng = SplitMix64(seed)
    cx, cy, cz = cell
    vol = float(cx * cy * cz)
    rows: list[list[int]] = []
    radii: list[float] = []
    filled = 0.0
    tries = 0
    while filled < vf and tries < max_tries:
        tries += 1
        r = rmin + (rmax - rmin) * rng.uniform()
        r = round(2.0 * r) / 2.0
        c = (rng.uniform() * cx, rng.uniform() * cy, rng.uniform() * cz)
        row = sphere_row(c[0], c[1], c[2], r, phase)
        ok = True
        for other, ro in zip(rows, radii):
            d2 = 0
            for ax, n in enumerate(cell):
                d = (row[ax] - other[ax]) % (2 * n)
                if d >= n:
                    d -= 2 * n
                d2 += d * d
            gap = 2.0 * (r + ro + 1.0)
            if d2 < gap * gap:
                ok = False
                break
        if ok:
            rows.append(row)
            radii.append(r)
            filled += 4.0 / 3.0 * math.pi * r ** 3 / vol
    return np.asarray(rows, dtype=np.int32).reshape(-1, 5)


@dataclass
class Problem:
    """One BFCS problem instance (dims are (nx, ny, nz); arrays are z-major, x fastest)."""
    name: str
    dims: tuple[int, int, int]
    cell: tuple[int, int, int]
    spheres: np.ndarray                      # (n, 5) int32, see module docstring
    phases: list[tuple[float, float]]        # (lambda, mu) per phase id; id 0 = matrix
    c0: tuple[float, float]                  # reference medium (lambda0, mu0)
    bf_centre: tuple[float, float, float]    # BFCS centre (voxel units)
    bf_radius: float                         # BFCS radius a (voxel units)
    mean_strain: tuple[float, ...] = (0.0,) * 6   # E: xx yy zz yz xz xy (tensorial)
    tol: float = 1e-6
    maxit: int = 2000
    extra: dict = field(default_factory=dict)


def config_c1() -> Problem:
    """32^3 = 2^3 cells of 16^3, one centred sphere R = 5 per cell, contrast 10."""
    phases = [(1.0, 0.5), (10.0, 5.0)]
    return Problem(
        name="c1_32cubed_fp64", dims=(32, 32, 32), cell=(16, 16, 16),
        spheres=np.asarray([sphere_row(8, 8, 8, 5.0)], dtype=np.int32),
        phases=phases, c0=reference_medium(phases),
        bf_centre=(16.0, 16.0, 16.0), bf_radius=6.0, tol=1e-10, maxit=4000)


def config_c2(contrast: float = 10.0, seed: int = 1, n: int = 256, cell: int = 32,
              vf: float = 0.25, bf_radius: float = 24.0) -> Problem:
    """n^3 = (n/cell)^3 cells of cell^3, RSA spheres vf 0.25 radii 4..6; Young contrast."""
    spheres = rsa_spheres((cell,) * 3, vf, 4.0, 6.0, seed)
    phases = [lame_from_young(1.0, 0.3), lame_from_young(contrast, 0.2)]
    c = n // 2
    return Problem(
        name=f"c2_{n}cubed_contrast{int(contrast)}_seed{seed}", dims=(n, n, n),
        cell=(cell,) * 3, spheres=spheres, phases=phases, c0=reference_medium(phases),
        bf_centre=(float(c), float(c), float(c)), bf_radius=bf_radius, tol=1e-6,
        maxit=20000, extra={"contrast": contrast, "seed": seed, "vf": vf})


def config_c3(n: int = 128) -> Problem:
    """n^3 = (n/16)^3 cells of 16^3, one centred sphere R = 5.8 (vf ~0.2), contrast 10."""
    phases = [lame_from_young(1.0, 0.3), lame_from_young(10.0, 0.2)]
    c = n // 2
    return Problem(
        name=f"c3_{n}cubed_translated", dims=(n, n, n), cell=(16, 16, 16),
        spheres=np.asarray([sphere_row(8, 8, 8, 5.8)], dtype=np.int32),
        phases=phases, c0=reference_medium(phases),
        bf_centre=(float(c), float(c), float(c)), bf_radius=6.0, tol=1e-6, maxit=20000)


def c3_shifts(stride: int = 4, cell: int = 16) -> np.ndarray:
    """Integer translation lattice chi in one unit cell (4^3 = 64 shifts for stride 4)."""
    ax = np.arange(0, cell, stride)
    g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    return g.astype(np.int32)


def config_c4(seed: int = 1, n: int = 256) -> Problem:
    """n^3, RSA vf 0.3 in 32^3 cells, stiff inclusions at Young contrast 1000."""
    p = config_c2(contrast=1000.0, seed=seed, n=n, vf=0.3)
    p.name = f"c4_{n}cubed_contrast1000_seed{seed}"
    return p


def config_c5_sample(seed: int, n: int = 64) -> Problem:
    """One training sample: one 16^3-cell RSA microstructure of vf ~U[0.1, 0.3]
    (addition stops at vf or after 4000 tries: the one-voxel gap jams the
    packing near vf 0.25), contrast 10, BFCS radius a ~ U[4, 12] at a uniform
    random voxel corner."""
    rng = SplitMix64(0xC5C5 ^ (seed * 0x9E3779B1))
    vf = 0.1 + 0.2 * rng.uniform()
    a = 4.0 + 8.0 * rng.uniform()
    centre = tuple(float(int(rng.uniform() * n)) for _ in range(3))
    spheres = rsa_spheres((16, 16, 16), vf, 2.0, 4.0, seed ^ 0x5EED, max_tries=4000)
    phases = [lame_from_young(1.0, 0.3), lame_from_young(10.0, 0.2)]
    return Problem(
        name=f"c5_{n}cubed_seed{seed}", dims=(n, n, n), cell=(16, 16, 16),
        spheres=spheres, phases=phases, c0=reference_medium(phases),
        bf_centre=centre, bf_radius=a, tol=1e-6, maxit=20000,
        extra={"vf": vf, "seed": seed})
