"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a direct
DFT sum, an operator identity, a closed-form solution, a dense brute-force
solve, an energy or reciprocity identity, or an exact symmetry.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import bfcs_oracle as O

RNG = np.random.default_rng(20260103)
WEIGHT = np.array([1, 1, 1, 2, 2, 2], dtype=float)   # shear components count twice


def rand_sym(shape=()):
    return RNG.standard_normal((6,) + shape)


def mean_free(b):
    return b - b.mean(axis=(-3, -2, -1), keepdims=True)


def drop_xi_zero(b):
    """Remove the load content on modes where xi = 0 (k = 0 and Nyquist corners)."""
    nz, ny, nx = b.shape[-3:]
    bh = O.fft3(b)
    xi = O.wavevectors((nx, ny, nz))
    q = xi[0] ** 2 + xi[1] ** 2 + xi[2] ** 2
    bh = bh * (q > 0)
    return np.real(O.ifft3(bh))


# ------------------------------------------------------------ DFT (Eqs. 4.3-4.5, 4.10-4.15)
@pytest.mark.parametrize("shape", [(4, 6, 2), (2, 4, 6), (3, 2, 4)])
def test_fft_matches_direct_dft(shape):
    f = RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)
    nz, ny, nx = shape
    direct = np.zeros(shape, dtype=complex)
    inv = np.zeros(shape, dtype=complex)
    pts = list(itertools.product(range(nz), range(ny), range(nx)))
    for k in pts:
        acc = 0j
        acc_i = 0j
        for n in pts:
            ph = 2 * math.pi * sum(k[a] * n[a] / shape[a] for a in range(3))
            acc += f[n] * complex(math.cos(ph), -math.sin(ph))      # omega^{-kn}
            acc_i += f[n] * complex(math.cos(ph), math.sin(ph))     # omega^{+kn}
        direct[k] = acc
        inv[k] = acc_i / (nz * ny * nx)
    assert np.allclose(O.fft3(f), direct, rtol=0, atol=1e-12)
    assert np.allclose(O.ifft3(f), inv, rtol=0, atol=1e-12)
    assert np.allclose(O.ifft3(O.fft3(f)), f, atol=1e-13)             # Eq. 4.9


def test_convolution_theorem_1d_and_3d():
    n = 12
    f, g = RNG.standard_normal(n), RNG.standard_normal(n)
    s = np.array([sum(f[m] * g[(k - m) % n] for m in range(n)) for k in range(n)])   # Eq. 4.14
    assert np.allclose(np.fft.fft(s), np.fft.fft(f) * np.fft.fft(g), atol=1e-11)
    shape = (4, 2, 6)
    f3, g3 = RNG.standard_normal(shape), RNG.standard_normal(shape)
    conv = np.zeros(shape)
    for k in itertools.product(*(range(d) for d in shape)):
        for j in itertools.product(*(range(d) for d in shape)):
            conv[k] += f3[tuple((k[a] - j[a]) % shape[a] for a in range(3))] * g3[j]  # Eq. 4.11
    assert np.allclose(O.fft3(conv), O.fft3(f3) * O.fft3(g3), atol=1e-10)          # Eq. 4.10


def test_wavevector_nyquist_and_hermitian():
    dims = (8, 6, 4)
    xi = O.wavevectors(dims)
    for a, n in enumerate(dims):
        v = xi[a].ravel()
        assert v[n // 2] == 0.0
        for k in range(n):
            assert v[(-k) % n] == -v[k]
        assert v[1] == pytest.approx(2 * math.pi / n)


def test_spectral_derivative_exact_on_trig_polynomial():
    dims = (16, 8, 4)
    nx, ny, nz = dims
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    xi = O.wavevectors(dims)
    for m in (1, 3, 7):
        f = np.sin(2 * math.pi * m * x / nx) * np.cos(2 * math.pi * 2 * y / ny) + 0 * np.zeros((nz, 1, 1))
        df = np.real(O.ifft3(1j * xi[0] * O.fft3(f)))
        exact = (2 * math.pi * m / nx) * np.cos(2 * math.pi * m * x / nx) * np.cos(2 * math.pi * 2 * y / ny)
        assert np.allclose(df, exact + 0 * df, atol=1e-12)
    # Nyquist content has zero derivative under reading R1
    f = np.cos(math.pi * x) + 0 * np.zeros((nz, ny, 1))
    assert np.allclose(np.real(O.ifft3(1j * xi[0] * O.fft3(f))), 0, atol=1e-12)


# ------------------------------------------------------------ Green operators (Eqs. 2.16-2.18, 2.27)
def u0_tensor(xi_vec, lam0, mu0):
    """U0_ijkl at one wavevector, recovered from u0_apply on symmetric basis tensors."""
    xi = tuple(np.array([[[v]]]) for v in xi_vec)
    U = np.zeros((3, 3, 3, 3))
    for b, (k, l) in enumerate(O.COMP):
        basis = np.zeros((6, 1, 1, 1), dtype=complex)
        basis[b] = 1.0 if k == l else 0.5     # E^{kl} = (e_k e_l + e_l e_k)/2
        out = O.u0_apply(basis, xi, lam0, mu0)[:, 0, 0, 0].real
        for a, (i, j) in enumerate(O.COMP):
            for (p, q) in {(i, j), (j, i)}:
                for (r, s) in {(k, l), (l, k)}:
                    U[p, q, r, s] = out[a]
    return U


def sym6(t):
    """3x3 -> 6 components."""
    return np.array([t[i, j] for (i, j) in O.COMP])


def full3(v):
    return np.array([[v[O.IDX[i, j]] for j in range(3)] for i in range(3)])


@pytest.mark.parametrize("seed", range(5))
def test_u0_symmetries_evenness_homogeneity(seed):
    r = np.random.default_rng(seed)
    xi = r.standard_normal(3)
    lam0, mu0 = 1.0 + r.random(), 0.5 + r.random()
    U = u0_tensor(xi, lam0, mu0)
    assert np.allclose(U, U.transpose(1, 0, 2, 3), atol=1e-14)
    assert np.allclose(U, U.transpose(0, 1, 3, 2), atol=1e-14)
    assert np.allclose(U, U.transpose(2, 3, 0, 1), atol=1e-14)
    assert np.allclose(U, u0_tensor(-xi, lam0, mu0), atol=1e-14)
    assert np.allclose(U, u0_tensor(3.7 * xi, lam0, mu0), atol=1e-13)


@pytest.mark.parametrize("seed", range(5))
def test_projection_identities(seed):
    r = np.random.default_rng(100 + seed)
    xi = r.standard_normal(3)
    lam0, mu0 = 0.5 + r.random(), 0.3 + r.random()
    U = u0_tensor(xi, lam0, mu0)
    G = -U                                         # Gamma0 = -U0
    C = O.stiffness(lam0, mu0)
    GCG = np.einsum("ijmn,mnpq,pqkl->ijkl", G, C, G)
    assert np.allclose(GCG, G, atol=1e-13)         # Gamma0 C0 Gamma0 = Gamma0
    v = r.standard_normal(3)
    e = 0.5 * (np.outer(xi, v) + np.outer(v, xi))  # compatible (zero-mean) strain mode
    assert np.allclose(np.einsum("ijkl,kl->ij", U, np.einsum("klmn,mn->kl", C, e)), -e,
                       atol=1e-13)                 # Eq. 2.27 on k != 0
    tau = full3(r.standard_normal(6))
    lhs = np.einsum("ijkl,kl->ij", C, np.einsum("ijkl,kl->ij", G, tau)) @ xi
    assert np.allclose(lhs, tau @ xi, atol=1e-13)  # xi.C0.Gamma0 tau = xi.tau


def test_reference_strain_equilibrates_load():
    r = np.random.default_rng(7)
    lam0, mu0 = 2.0, 0.7
    xi = tuple(r.standard_normal((1, 1, 5)) for _ in range(3))
    bh = r.standard_normal((3, 1, 1, 5)) + 1j * r.standard_normal((3, 1, 1, 5))
    e = O.eps_b0_hat(bh, xi, lam0, mu0)
    s = e.copy()
    tr = e[0] + e[1] + e[2]
    s = 2 * mu0 * e
    s[:3] += lam0 * tr
    assert np.allclose(O.div_hat(s, xi) + bh, 0, atol=1e-12)   # i xi.(C0 eps^{b0}) + b = 0


# ------------------------------------------------------------ closed forms
def navier_inverse(xi, lam, mu):
    """Closed-form inverse of the isotropic acoustic tensor (textbook)."""
    q = xi @ xi
    return (np.eye(3) - (lam + mu) / (lam + 2 * mu) * np.outer(xi, xi) / q) / (mu * q)


def test_plane_wave_load_homogeneous_closed_form():
    dims = (8, 6, 4)
    nx, ny, nz = dims
    lam, mu = 1.3, 0.8
    m = np.array([1, 2, 1])
    xi = 2 * math.pi * m / np.array(dims)
    B = np.array([0.3, -0.2, 0.5])
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    z = np.arange(nz)[:, None, None]
    ph = xi[0] * x + xi[1] * y + xi[2] * z
    b = np.stack([B[i] * np.cos(ph) for i in range(3)])
    a = navier_inverse(xi, lam, mu) @ B                 # u = a cos(xi.x)
    phase = np.zeros((nz, ny, nx), dtype=np.int8)
    res = O.solve(phase, [(lam, mu)], (lam, mu), b, tol=0, maxit=1)
    u_exact = np.stack([a[i] * np.cos(ph) for i in range(3)])
    e_exact = np.stack([-0.5 * (xi[i] * a[j] + xi[j] * a[i]) * np.sin(ph) for (i, j) in O.COMP])
    assert np.allclose(res["u"], u_exact, atol=1e-13)
    assert np.allclose(res["eps"], e_exact, atol=1e-13)
    assert res["resid"] < 1e-13


def test_homogeneous_case_one_sweep_exact():
    dims = (6, 8, 4)
    nx, ny, nz = dims
    c0 = (1.7, 0.9)
    phase = RNG.integers(0, 3, size=(nz, ny, nx)).astype(np.int8)
    table = [c0, c0, c0]                                  # C(x) = C0 everywhere
    b = drop_xi_zero(RNG.standard_normal((3, nz, ny, nx)))
    E = tuple(0.01 * RNG.standard_normal(6))
    res = O.solve(phase, table, c0, b, E, tol=0, maxit=1, history=True)
    xi = O.wavevectors(dims)
    e0h = O.eps_b0_hat(O.fft3(b), xi, *c0)
    e0h[:, 0, 0, 0] = nx * ny * nz * np.array(E)
    assert np.allclose(res["eps"], np.real(O.ifft3(e0h)), atol=1e-13)
    assert res["hist"][0] < 1e-13 and res["resid"] < 1e-13
    assert np.allclose(res["eps"].mean(axis=(1, 2, 3)), E, atol=1e-14)


def laminate_exact(lam, mu, b1, e11):
    """Exact discrete solution of the 1D laminate d/dx sigma11 + b1 = 0 under reading R1."""
    n = b1.size
    k = np.fft.fftfreq(n, d=1.0 / n)
    k[n // 2] = 0
    xi = 2 * math.pi * k / n
    bh = np.fft.fft(b1)
    s0h = np.zeros(n, dtype=complex)
    nzm = xi != 0
    s0h[nzm] = 1j * bh[nzm] / xi[nzm]
    s0 = np.real(np.fft.ifft(s0h))
    comp = 1.0 / (lam + 2 * mu)                   # compliance along the stack
    alt = (-1.0) ** np.arange(n)
    A = np.array([[comp.sum(), (alt * comp).sum()], [(alt * comp).sum(), comp.sum()]])
    rhs = np.array([n * e11 - (comp * s0).sum(), -(alt * comp * s0).sum()])
    c0, c1 = np.linalg.solve(A, rhs)
    sig11 = s0 + c0 + c1 * alt
    return comp * sig11, sig11


def test_laminate_closed_form():
    nx, ny, nz = 16, 2, 2
    lam_ph = [1.0, 10.0]
    mu_ph = [0.5, 5.0]
    layers = np.array([0, 0, 1, 1, 1, 0, 0, 0, 1, 0, 1, 1, 0, 0, 1, 0], dtype=np.int8)
    phase = np.broadcast_to(layers[None, None, :], (nz, ny, nx)).copy()
    b1 = RNG.standard_normal(nx)
    bh = np.fft.fft(b1)
    bh[0] = 0
    bh[nx // 2] = 0
    b1 = np.real(np.fft.ifft(bh))
    b = np.zeros((3, nz, ny, nx))
    b[0] = b1[None, None, :]
    E = (0.02, 0, 0, 0, 0, 0)
    table = list(zip(lam_ph, mu_ph))
    c0 = (5.5, 2.75)
    res = O.solve(phase, table, c0, b, E, tol=1e-14, maxit=5000)
    e11, s11 = laminate_exact(np.array(lam_ph)[layers], np.array(mu_ph)[layers], b1, E[0])
    assert res["resid"] < 1e-13
    assert np.allclose(res["eps"][0], e11[None, None, :], atol=1e-12)
    assert np.allclose(res["eps"][1:], 0, atol=1e-12)
    assert np.allclose(res["sig"][0], s11[None, None, :], atol=1e-11)


# ------------------------------------------------------------ dense brute force
def _operators(dims):
    """Real matrices of the spectral symmetric gradient D_s (3N -> 6N) and of the
    divergence (6N -> 3N), assembled column by column from unit vectors."""
    nx, ny, nz = dims
    n = nx * ny * nz
    xi = O.wavevectors(dims)
    Ds = np.zeros((6 * n, 3 * n))
    for c in range(3 * n):
        u = np.zeros(3 * n)
        u[c] = 1.0
        uh = O.fft3(u.reshape(3, nz, ny, nx))
        Ds[:, c] = np.real(O.ifft3(O.sym_grad_hat(uh, xi))).ravel()
    Dv = np.zeros((3 * n, 6 * n))
    for c in range(6 * n):
        s = np.zeros(6 * n)
        s[c] = 1.0
        sh = O.fft3(s.reshape(6, nz, ny, nx))
        Dv[:, c] = np.real(O.ifft3(O.div_hat(sh, xi))).ravel()
    return Ds, Dv


@pytest.mark.parametrize("dims", [(4, 4, 4), (6, 4, 2)])
def test_dense_bruteforce_solve(dims):
    nx, ny, nz = dims
    n = nx * ny * nz
    r = np.random.default_rng(sum(dims))
    phase = r.integers(0, 2, size=(nz, ny, nx)).astype(np.int8)
    table = [(1.0, 0.5), (4.0, 2.0)]
    c0 = (2.5, 1.25)
    b = mean_free(r.standard_normal((3, nz, ny, nx)))
    E = tuple(0.05 * r.standard_normal(6))
    Ds, Dv = _operators(dims)
    lam = np.array([t[0] for t in table])[phase].ravel()
    mu = np.array([t[1] for t in table])[phase].ravel()

    def Lmat():
        L = np.zeros((6 * n, 6 * n))
        for a in range(6):
            for p in range(n):
                L[a * n + p, a * n + p] += 2 * mu[p]
                if a < 3:
                    for c in range(3):
                        L[a * n + p, c * n + p] += lam[p]
        return L

    L = Lmat()
    Evec = np.concatenate([np.full(n, E[a]) for a in range(6)])
    A = -Dv @ L @ Ds
    rhs = b.ravel() + Dv @ (L @ Evec)
    u = np.linalg.lstsq(A, rhs, rcond=1e-12)[0]
    eps_direct = (Evec + Ds @ u).reshape(6, nz, ny, nx)
    res = O.solve(phase, table, c0, b, E, tol=1e-14, maxit=5000)
    assert res["resid"] < 1e-13
    assert np.allclose(res["eps"], eps_direct, atol=1e-10)


# ------------------------------------------------------------ energy, reciprocity, translation
def _c1_small():
    dims = (16, 16, 16)
    spheres = np.array([[16, 16, 16, 100, 1]], dtype=np.int32)
    phase = O.phase_map(dims, (16, 16, 16), spheres)
    table = [(1.0, 0.5), (10.0, 5.0)]
    return dims, phase, table, (5.5, 2.75)


def test_energy_identity_fixes_displacement_scale():
    dims, phase, table, c0 = _c1_small()
    b = O.body_force(dims, (8.0, 8.0, 8.0), 5.0)
    res = O.solve(phase, table, c0, b, tol=1e-12, maxit=3000)
    work = np.sum(b * res["u"])
    energy = np.sum(WEIGHT[:, None, None, None] * res["sig"] * res["eps"])
    assert work > 0
    assert work == pytest.approx(energy, rel=1e-9)


def test_betti_reciprocity():
    dims, phase, table, c0 = _c1_small()
    bA = O.body_force(dims, (8.0, 8.0, 8.0), 5.0)
    bB = O.body_force(dims, (4.0, 10.0, 6.0), 4.0)
    bB = np.stack([bB[0] * 0, bB[0], bB[0] * 0])      # a load along x2 this time
    uA = O.solve(phase, table, c0, bA, tol=1e-12, maxit=3000)["u"]
    uB = O.solve(phase, table, c0, bB, tol=1e-12, maxit=3000)["u"]
    lhs, rhs = np.sum(bA * uB), np.sum(bB * uA)
    assert abs(lhs - rhs) <= 1e-9 * max(abs(lhs), abs(rhs), 1e-30)
    assert abs(lhs) > 1e-8


def test_translation_equivariance():
    dims = (12, 8, 8)
    nx, ny, nz = dims
    spheres = np.array([[6, 7, 8, 12, 1]], dtype=np.int32)
    phase0 = O.phase_map(dims, (12, 8, 8), spheres)
    table = [(1.0, 0.5), (6.0, 3.0)]
    c0 = (3.5, 1.75)
    b = O.body_force(dims, (6.0, 4.0, 4.0), 3.5)
    chi = (5, 3, 2)
    a = O.solve(O.translate(phase0, chi), table, c0, b, tol=0, maxit=25)
    bs = O.translate(b, tuple(-c for c in chi))
    c = O.solve(phase0, table, c0, bs, tol=0, maxit=25)
    for key in ("eps", "sig", "u"):
        assert np.allclose(a[key], O.translate(c[key], chi), atol=1e-13)


def test_neumann_partial_sums():
    dims = (8, 8, 8)
    nx, ny, nz = dims
    r = np.random.default_rng(3)
    phase = r.integers(0, 2, size=(nz, ny, nx)).astype(np.int8)
    table = [(1.0, 0.5), (3.0, 1.5)]
    c0 = (2.0, 1.0)
    b = mean_free(r.standard_normal((3, nz, ny, nx)))
    xi = O.wavevectors(dims)
    e0 = np.real(O.ifft3(O.eps_b0_hat(O.fft3(b), xi, *c0)))
    t1 = [(l - c0[0], m - c0[1]) for l, m in table]

    def B(e):   # B^U = F^-1 U0 F L1  (Eq. 5.5)
        return np.real(O.ifft3(O.u0_apply(O.fft3(O.apply_local(phase, t1, e)), xi, *c0)))

    term, total = e0, e0.copy()
    for j in range(1, 6):
        term = B(term)
        total = total + term
        res = O.solve(phase, table, c0, b, tol=0, maxit=j)
        assert np.allclose(res["eps"], total, atol=1e-13)   # Eq. 5.6


# ------------------------------------------------------------ inputs: phase map and body force
def test_phase_map_bruteforce():
    dims, cell = (12, 10, 8), (6, 10, 4)
    spheres = np.array([[3, 9, 4, 9, 1], [11, 1, 7, 6, 2], [0, 19, 0, 4, 3]], dtype=np.int32)
    ph = O.phase_map(dims, cell, spheres)
    nx, ny, nz = dims
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                want = 0
                for (X, Y, Z, T, p) in spheres:
                    d2 = 0
                    for (i, c, n) in ((x % cell[0], X, cell[0]), (y % cell[1], Y, cell[1]),
                                      (z % cell[2], Z, cell[2])):
                        best = min(abs(2 * i + 1 - c + 2 * n * s) for s in (-1, 0, 1))
                        d2 += best * best
                    if d2 <= T:
                        want = p
                assert ph[z, y, x] == want


def test_centred_sphere_voxel_count():
    # lattice points (i+1/2, j+1/2, k+1/2) - 8 with squared distance <= 25, counted by loops
    count = sum(1 for i in range(16) for j in range(16) for k in range(16)
                if (i + 0.5 - 8) ** 2 + (j + 0.5 - 8) ** 2 + (k + 0.5 - 8) ** 2 <= 25)
    ph = O.phase_map((16, 16, 16), (16, 16, 16), np.array([[16, 16, 16, 100, 1]]))
    assert int((ph == 1).sum()) == count == 552


def test_body_force_form():
    dims = (24, 20, 16)
    centre, a = (10.0, 9.5, 8.0), 6.0
    b = O.body_force(dims, centre, a)
    assert abs(b[0].sum()) < 1e-12 and np.all(b[1:] == 0)
    raw = b[0] - b[0][0, 0, 0]           # the far field equals minus the removed mean
    nx, ny, nz = dims
    h = 1e-5
    for (x, y, z) in [(12, 9, 8), (7, 11, 6), (10, 14, 9)]:
        p = np.array([x + 0.5, y + 0.5, z + 0.5]) - np.array(centre)

        def phi(q):
            r2 = q @ q
            return (1 - r2 / a ** 2) ** 3 if r2 < a * a else 0.0
        fd = (phi(p + [h, 0, 0]) - phi(p - [h, 0, 0])) / (2 * h)
        assert raw[z, y, x] == pytest.approx(fd, abs=1e-8)
    # voxel centres at integer + 1/2 about an integer centre: odd in x1, sum exactly ~0
    b2 = O.body_force((16, 16, 16), (8.0, 8.0, 8.0), 5.0)[0]
    assert np.allclose(b2, -b2[:, :, ::-1], atol=1e-15)


# ------------------------------------------------------------ translated averaging
def test_translate_average_invariants():
    dims = (8, 8, 8)
    cell = (4, 4, 4)
    spheres = np.array([[4, 4, 4, 6, 1]], dtype=np.int32)
    phase0 = O.phase_map(dims, cell, spheres)
    table = [(1.0, 0.5), (5.0, 2.5)]
    c0 = (3.0, 1.5)
    b = O.body_force(dims, (4.0, 4.0, 4.0), 2.5)
    # single shift chi = 0 reproduces the plain solve
    avg, hits, _ = O.translate_average(phase0, table, c0, b, [(0, 0, 0)], tol=0, maxit=10)
    one = O.solve(phase0, table, c0, b, tol=0, maxit=10)
    assert np.allclose(avg[6:12], one["eps"]) and np.allclose(avg[0:3], one["u"])
    v = (phase0 != 0)
    assert np.allclose(avg[24:30], v * one["sig"]) and np.array_equal(hits, v)
    # the full stride-1 lattice of shifts in one cell: every voxel is hit by as many
    # shifts as the cell has inclusion voxels
    shifts = [(i, j, k) for i in range(4) for j in range(4) for k in range(4)]
    per_cell = int((O.phase_map(cell, cell, spheres) != 0).sum())
    _, hits, _ = O.translate_average(phase0, table, c0, b, shifts, tol=0, maxit=0)
    assert np.all(hits == per_cell)
    # shifting by a whole cell period leaves every member unchanged
    avg2, _, _ = O.translate_average(phase0, table, c0, b, [(4, 0, 0), (0, 4, 4)], tol=0, maxit=6)
    one = O.solve(phase0, table, c0, b, tol=0, maxit=6)
    assert np.allclose(avg2[18:24], one["sig"], atol=1e-14)


def test_residual_normaliser_closed_form():
    """Reading R4 of Eq. 5.11 on a field whose residual is known by hand: a
    homogeneous medium (mu = 1/2) under the uniform pure shear eps_xy = 0.05, so
    sigma_xy = 0.05 everywhere and its divergence vanishes, with the load
    b_x = cos(2 pi x / nx).  On the 8 x 4 x 2 grid (N = 64) the numerator is
    |b_hat| = N / sqrt(2) (two modes of modulus N / 2); the normaliser adds
    xi_min |sigma_hat(0)|_F with xi_min = 2 pi / 8 (the largest edge) and
    |sigma_hat(0)|_F = N 0.05 sqrt(2) (the shear counted in both off-diagonal
    entries).  Hence r = 1 / (1 + pi / 40)."""
    dims = (8, 4, 2)
    nx, ny, nz = dims
    phase = np.zeros((nz, ny, nx), dtype=np.int8)
    eps = np.zeros((6, nz, ny, nx))
    eps[5] = 0.05
    b = np.zeros((3, nz, ny, nx))
    b[0] = np.cos(2 * np.pi * np.arange(nx) / nx)[None, None, :]
    r = O.residual(phase, [(1.0, 0.5)], eps, O.fft3(b), O.wavevectors(dims))
    assert r == pytest.approx(1.0 / (1.0 + math.pi / 40.0), rel=1e-14)


def test_residual_decreases_and_parseval():
    dims, phase, table, c0 = _c1_small()
    b = O.body_force(dims, (8.0, 8.0, 8.0), 5.0)
    res = O.solve(phase, table, c0, b, tol=1e-9, maxit=500, history=True)
    h = res["hist"]
    assert h[-1] < h[0] * 1e-6
    assert all(h[i + 1] < h[i] for i in range(5, len(h) - 1))
    # real-space equilibrium error of the returned field matches the spectral numerator
    nx, ny, nz = dims
    xi = O.wavevectors(dims)
    sh = O.fft3(res["sig"])
    bh = O.fft3(b)
    q = xi[0] ** 2 + xi[1] ** 2 + xi[2] ** 2
    d = (O.div_hat(sh, xi) + bh) * (q > 0)
    real_space = np.real(O.ifft3(d))
    assert np.sum(np.abs(d) ** 2) == pytest.approx(nx * ny * nz * np.sum(real_space ** 2), rel=1e-10)


def test_translation_direction_by_index():
    """Eq. 3.3: L(x, chi) = L0(x - chi), checked element by element."""
    f = RNG.integers(0, 100, size=(5, 6, 7))
    chi = (2, 4, 1)   # (x, y, z)
    g = O.translate(f, chi)
    for z in range(5):
        for y in range(6):
            for x in range(7):
                assert g[z, y, x] == f[(z - chi[2]) % 5, (y - chi[1]) % 6, (x - chi[0]) % 7]


# ------------------------------------------------------------ effective moduli (Eqs. 6.1-6.3, 3.2)
def _stiffness_matrix(lam, mu):
    """Response <sigma>_I to unit tensorial E_J of a homogeneous isotropic medium."""
    M = np.zeros((6, 6))
    M[:3, :3] = lam
    for i in range(3):
        M[i, i] = lam + 2 * mu
    for i in range(3, 6):
        M[i, i] = 2 * mu
    return M


def _laminate_uniaxial(comp, target):
    """1D laminate along x under reading R1: the stress sigma = c0 + c1 (-1)^x is
    in equilibrium, the strain comp * sigma must have mean `target` and no
    Nyquist component.  Returns the stress."""
    n = comp.size
    alt = (-1.0) ** np.arange(n)
    A = np.array([[comp.sum(), (alt * comp).sum()], [(alt * comp).sum(), (alt * alt * comp).sum()]])
    c0, c1 = np.linalg.solve(A, np.array([n * target, 0.0]))
    return c0 + c1 * alt


def test_effective_moduli_homogeneous_and_identical_phases():
    phase = np.zeros((4, 4, 6), dtype=np.int8)
    phase[1:3, 1:3, 2:4] = 1
    table = [(2.0, 1.5), (2.0, 1.5)]
    Ls, As = O.effective_moduli(phase, table, (1.0, 1.0), tol=1e-13)
    assert np.allclose(Ls, _stiffness_matrix(2.0, 1.5), atol=1e-11)
    assert np.allclose(As, np.eye(6), atol=1e-11)


def test_effective_moduli_laminate_closed_forms():
    nx, ny, nz = 12, 2, 2
    layers = np.array([0, 1, 1, 0, 0, 0, 1, 0, 1, 1, 1, 0], dtype=np.int8)
    lam_ph, mu_ph = np.array([1.0, 8.0]), np.array([0.6, 4.0])
    phase = np.broadcast_to(layers[None, None, :], (nz, ny, nx)).copy()
    table = list(zip(lam_ph, mu_ph))
    Ls, As = O.effective_moduli(phase, table, (4.5, 2.3), tol=1e-13, maxit=8000)
    lam, mu = lam_ph[layers], mu_ph[layers]
    incl = layers != 0
    # E = e_xx: sigma_xx uniform up to the Nyquist mode, eps_xx = sigma_xx / (lam + 2 mu)
    s_xx = _laminate_uniaxial(1.0 / (lam + 2 * mu), 1.0)
    e_xx = s_xx / (lam + 2 * mu)
    assert abs(Ls[0, 0] - s_xx.mean()) < 1e-10
    assert abs(Ls[1, 0] - (lam * e_xx).mean()) < 1e-10 and abs(Ls[2, 0] - Ls[1, 0]) < 1e-10
    assert abs(As[0, 0] - e_xx[incl].mean()) < 1e-10
    # E = e_yz (in-plane shear): strain uniform, <sigma_yz> = 2 <mu>
    assert abs(Ls[3, 3] - 2 * mu.mean()) < 1e-10 and abs(As[3, 3] - 1.0) < 1e-10
    # E = e_xy (shear across the layers): sigma_xy as in the uniaxial case with compliance 1 / (2 mu)
    s_xy = _laminate_uniaxial(1.0 / (2 * mu), 1.0)
    assert abs(Ls[5, 5] - s_xy.mean()) < 1e-10
    assert abs(As[5, 5] - (s_xy / (2 * mu))[incl].mean()) < 1e-10


def test_effective_stiffness_is_symmetric_positive_definite():
    phases = [(1.0, 0.5), (10.0, 5.0)]                   # contrast 10, C0 = mean of the extremes
    phase = O.phase_map((8, 8, 8), (8, 8, 8), np.asarray([[8, 8, 8, 27, 1]], dtype=np.int32))
    Ls, As = O.effective_moduli(phase, phases, (5.5, 2.75), tol=1e-12)
    S = Ls @ np.diag([1, 1, 1, 0.5, 0.5, 0.5])     # Voigt-symmetric form of the tensorial response
    assert np.allclose(S, S.T, atol=1e-9 * abs(S).max())
    assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > 0
    # between the phases' stiffnesses (Voigt / Reuss-type ordering of the bulk response)
    k = S[:3, :3].sum() / 9
    assert phases[0][0] + 2 / 3 * phases[0][1] < k < phases[1][0] + 2 / 3 * phases[1][1]
    # sigma = L(x) eps voxel by voxel, so for two phases <sigma> = L_m E + f (L_i - L_m) <eps>_i
    f = (phase != 0).mean()
    L0, L1 = _stiffness_matrix(*phases[0]), _stiffness_matrix(*phases[1])
    assert np.allclose(Ls, L0 + f * (L1 - L0) @ As, atol=1e-12 * abs(Ls).max())


# ------------------------------------------------------------ ensemble dataset D^d (Eq. 3.8)
def _ensemble_case():
    nx, ny, nz = 8, 6, 4
    ph = (RNG.random((nz, ny, nx)) < 0.3).astype(np.int8)
    ph[RNG.random((nz, ny, nx)) < 0.15] = 2
    table = [(1.0, 0.5), (6.0, 3.0), (0.4, 0.2)]
    b = O.body_force((nx, ny, nz), (4.0, 3.0, 2.0), 2.5)
    return ph, table, (3.2, 1.6), b


def test_ensemble_of_one_configuration_is_its_solution():
    ph, table, c0, b = _ensemble_case()
    avg, hits, _ = O.ensemble_average([ph, ph, ph], table, c0, b, tol=1e-12)
    res = O.solve(ph, table, c0, b, tol=1e-12)
    v = (ph != 0)
    assert np.allclose(avg[0:3], res["u"], atol=1e-13) and np.allclose(avg[3:6], v * res["u"], atol=1e-13)
    assert np.allclose(avg[6:12], res["eps"], atol=1e-13) and np.allclose(avg[24:30], v * res["sig"], atol=1e-13)
    assert np.array_equal(hits, 3 * v)


def test_ensemble_of_mirror_pair_is_mirror_symmetric():
    """X and its reflection x -> 2c - x about the load centre plane c = 4: b_x is
    odd, so the averaged fields of the pair are symmetric under the reflection
    (vectors: x component odd; symmetric tensors: xz, xy odd), the inclusion
    weighted ones included."""
    ph, table, c0, b = _ensemble_case()
    refl = ph[:, :, ::-1].copy()                 # voxel i -> 2c - 1 - i = 7 - i for c = 4
    assert np.allclose(b[0][:, :, ::-1], -b[0], atol=1e-15)
    avg, hits, _ = O.ensemble_average([ph, refl], table, c0, b, tol=1e-13, maxit=4000)
    vec_sign = np.array([-1, 1, 1])[:, None, None, None]
    ten_sign = np.array([1, 1, 1, 1, -1, -1])[:, None, None, None]
    for lo, sign in ((0, vec_sign), (3, vec_sign), (6, ten_sign), (12, ten_sign), (18, ten_sign), (24, ten_sign)):
        f = avg[lo:lo + sign.shape[0]]
        assert np.abs(f[..., ::-1] - sign * f).max() <= 1e-11 * np.abs(f).max(), lo
    assert np.array_equal(hits, hits[:, :, ::-1])
    # a single configuration is not symmetric, so the pair's symmetry is not trivial
    one, _, _ = O.ensemble_average([ph], table, c0, b, tol=1e-13, maxit=4000)
    assert np.abs(one[12:18][..., ::-1] - ten_sign * one[12:18]).max() > 1e-3 * np.abs(one[12:18]).max()


def test_ensemble_of_all_translations_is_the_translated_average():
    """Eq. 3.8 is the dataset of Eq. 3.7 with configurations in place of
    translations: the ensemble of the translated copies of one cell gives the
    translated average."""
    ph, table, c0, b = _ensemble_case()
    shifts = [(0, 0, 0), (3, 1, 0), (5, 4, 2), (1, 5, 3)]
    configs = [O.translate(ph, np.asarray(s)) for s in shifts]
    avg_e, hits_e, _ = O.ensemble_average(configs, table, c0, b, tol=1e-12)
    avg_t, hits_t, _ = O.translate_average(ph, table, c0, b, shifts, tol=1e-12)
    assert np.allclose(avg_e, avg_t, atol=1e-14) and np.array_equal(hits_e, hits_t)


# ------------------------------------------------------------ RVE size (Def. 2.2, Sec. 5)
def test_radial_profile_against_brute_force_loops():
    nx, ny, nz = 6, 4, 5
    centre = (3.0, 2.0, 2.5)
    f6 = RNG.standard_normal((6, nz, ny, nx))
    f3 = RNG.standard_normal((3, nz, ny, nx))
    for f, w in ((f6, (1, 1, 1, 2, 2, 2)), (f3, (1, 1, 1))):
        prof, counts = O.radial_profile(f, centre, 5)
        ref = np.zeros(5)
        cnt = np.zeros(5, dtype=int)
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    d2 = 0.0
                    for pos, c, n in ((x, centre[0], nx), (y, centre[1], ny), (z, centre[2], nz)):
                        d = pos + 0.5 - c
                        d = min(abs(d - n * k) for k in (-1, 0, 1))
                        d2 += d * d
                    k = int(math.floor(math.sqrt(d2)))
                    if k < 5:
                        v = math.sqrt(sum(wc * f[c, z, y, x] ** 2 for c, wc in enumerate(w)))
                        ref[k] = max(ref[k], v)
                        cnt[k] += 1
        assert np.array_equal(counts, cnt)
        assert np.allclose(prof, ref, rtol=1e-15, atol=0)


def test_radial_profile_of_the_distance_itself():
    """A field equal to the distance from the centre: shell k holds values in [k, k + 1);
    about a voxel corner the innermost shell is the 8 voxels at sqrt(3) / 2."""
    n = 8
    c = (4.0, 4.0, 4.0)
    g = np.arange(n) + 0.5 - 4.0
    d = np.sqrt(g[None, None, :] ** 2 + g[None, :, None] ** 2 + g[:, None, None] ** 2)
    f = np.stack([d, np.zeros_like(d), np.zeros_like(d)])
    prof, counts = O.radial_profile(f, c, 4)
    assert counts[0] == 8 and abs(prof[0] - math.sqrt(3) / 2) < 1e-15
    for k in range(4):
        assert counts[k] > 0 and k <= prof[k] < k + 1


def test_rve_radius_rule():
    p1 = np.array([1.0, 0.5, 0.1, 1e-4, 1e-5, 0.0])
    p2 = np.array([2.0, 1.0, 0.05, 0.01, 1e-6, 0.0])
    assert O.rve_radius([p1], 1e-3, 6) == 3
    assert O.rve_radius([p2], 1e-3, 6) == 4
    assert O.rve_radius([p1, p2], 1e-3, 6) == 4
    assert O.rve_radius([p1], 1e-3, 3) is None          # the outermost shell considered is still above
    assert O.rve_radius([np.array([1.0, 0.0, 0.0])], 1e-3, 3) == 1


def test_rve_size_loop_accepts_the_first_cell_holding_the_rve_and_fields_stabilise():
    """Cell 8^3 with one sphere, support radius a = 3, field tolerance 5%: the
    16^3 cell holds no RVE, 24^3 does (r + a/2 <= 12) and ends the loop; the
    strain inside that RVE then changes by less than the tolerance when the
    cell is enlarged to 40^3 (Sec. 5: further enlargement leaves it unaffected)."""
    cell = (8, 8, 8)
    sph = np.asarray([[8, 8, 8, 25, 1]], np.int32)
    table, c0, a, tol_f = [(1.0, 0.5), (6.0, 3.0)], (3.5, 1.75), 3.0, 0.05
    recs = O.rve_size(cell, sph, table, c0, a, sizes=(16, 24, 32), tol=1e-11, tol_f=tol_f)
    assert [r["n"] for r in recs] == [16, 24]
    assert recs[0]["r_rve"] is None and not recs[0]["contained"]
    r = recs[1]["r_rve"]
    assert recs[1]["contained"] and r + a / 2 <= 12
    pe = recs[1]["prof_eps"]
    assert pe[r - 1] > tol_f * pe.max() and np.all(pe[r:12] <= tol_f * pe.max())

    def solve(n):
        ph = O.phase_map((n,) * 3, cell, sph)
        cen = tuple(float(k * int(np.floor(n / (2.0 * k) + 0.5))) for k in cell)
        return O.solve(ph, table, c0, O.body_force((n,) * 3, cen, a), tol=1e-11, maxit=4000)["eps"], int(cen[0])

    (ea, ca), (eb, cb) = solve(24), solve(40)
    g = np.arange(-r, r)
    ball = (g[:, None, None] + 0.5) ** 2 + (g[None, :, None] + 0.5) ** 2 + (g[None, None, :] + 0.5) ** 2 < r * r
    wa = ea[:, (ca + g)[:, None, None] % 24, (ca + g)[None, :, None] % 24, (ca + g)[None, None, :] % 24]
    wb = eb[:, (cb + g)[:, None, None] % 40, (cb + g)[None, :, None] % 40, (cb + g)[None, None, :] % 40]
    assert np.abs(wa - wb)[:, ball].max() <= tol_f * np.abs(ea).max()


def test_rve_size_loop_needs_the_annulus_inside_the_cell():
    """a = 4, field tolerance 4.8%: at 24^3 the fields fall below the tolerance
    from r = 11 on, but r + a/2 = 13 > 12 leaves no room for the annulus of
    half the support radius, so the loop goes on to 32^3 (r = 10 fits)."""
    recs = O.rve_size((8, 8, 8), np.asarray([[8, 8, 8, 25, 1]], np.int32), [(1.0, 0.5), (6.0, 3.0)], (3.5, 1.75),
                      4.0, sizes=(24, 32), tol=1e-11, tol_f=0.048)
    assert [(r["n"], r["r_rve"], r["contained"]) for r in recs] == [(24, 11, False), (32, 10, True)]


# ------------------------------------------------------------ nonlocal kernel regression (Eqs. 6.5-6.6)
def test_bernstein_basis_partition_of_unity_and_endpoints():
    t = np.linspace(0, 1, 11)
    for M in (0, 1, 3, 6):
        B = O.bernstein(M, t)
        assert np.allclose(B.sum(axis=0), 1.0, atol=1e-14)        # binomial theorem
        assert B[0, 0] == 1.0 and B[M, -1] == 1.0 and np.all(B >= 0)


@pytest.mark.parametrize("delta", [2.5, 2.0])     # 2.0: lattice points on the horizon are outside (r < delta)
def test_kernel_operator_on_plane_waves(delta):
    """cos(q . x) is an eigenfunction: L[u] = (sum_xi K(|xi|) (cos(q . xi) - 1)) u."""
    nx, ny, nz = 8, 6, 10
    coef = np.array([0.3, -1.2, 0.7, 2.0])
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    z = np.arange(nz)[:, None, None]
    q = (2 * math.pi * 1 / nx, 2 * math.pi * 2 / ny, 2 * math.pi * 3 / nz)
    wave = np.cos(q[0] * x + q[1] * y + q[2] * z) * np.ones((nz, ny, nx))
    u = np.stack([wave, 2 * wave, -wave])
    mult = 0.0
    r = 2
    for ox in range(-r, r + 1):
        for oy in range(-r, r + 1):
            for oz in range(-r, r + 1):
                d = math.sqrt(ox * ox + oy * oy + oz * oz)
                if 0 < d < delta:
                    t = d / delta
                    K = sum(c * math.comb(3, m) * t ** m * (1 - t) ** (3 - m) for m, c in enumerate(coef))
                    mult += K * (math.cos(q[0] * ox + q[1] * oy + q[2] * oz) - 1)
    assert np.allclose(O.kernel_operator(u, coef, delta), mult * u, atol=1e-12)
    assert np.allclose(O.kernel_operator(np.ones((3, nz, ny, nx)), coef, delta), 0.0, atol=1e-13)


def test_kernel_operator_with_unit_kernel_against_loops():
    """All Bernstein coefficients 1 give K = 1 inside the horizon (partition of unity)."""
    nx, ny, nz = 5, 4, 6
    u = RNG.standard_normal((3, nz, ny, nx))
    delta = 1.8
    out = O.kernel_operator(u, np.ones(4), delta)
    ref = np.zeros_like(u)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for ox in (-1, 0, 1):
                    for oy in (-1, 0, 1):
                        for oz in (-1, 0, 1):
                            d = math.sqrt(ox * ox + oy * oy + oz * oz)
                            if 0 < d < delta:
                                ref[:, z, y, x] += u[:, (z + oz) % nz, (y + oy) % ny, (x + ox) % nx] - u[:, z, y, x]
    assert np.allclose(out, ref, atol=1e-12)


def test_kernel_fit_recovers_a_planted_kernel_and_shrinks_with_tikhonov():
    nx, ny, nz = 8, 8, 8
    delta, M = 3.0, 4
    c_true = np.array([1.5, -0.5, 0.8, 0.2, -1.0])
    us = [RNG.standard_normal((3, nz, ny, nx)) for _ in range(2)]
    gammas = [O.kernel_operator(u, c_true, delta) for u in us]
    fit = O.kernel_fit(us, gammas, delta, M, lam=0.0, iters=3000, lr=0.02)
    assert np.allclose(fit["exact"], c_true, rtol=1e-8, atol=1e-10)
    assert fit["loss"] < 1e-3 * fit["s"]      # Adam from c = 0 (J = s there) gets close; G is ill-conditioned
    norms = [np.linalg.norm(O.kernel_fit(us, gammas, delta, M, lam=lam, iters=1)["exact"])
             for lam in (0.0, 1e2, 1e4, 1e6)]
    assert all(a > b for a, b in zip(norms, norms[1:]))           # Tikhonov shrinks the coefficients


def test_kernel_fit_loss_is_the_direct_sum_and_adam_reaches_the_tikhonov_minimiser():
    """Eq. 6.6 with Tikhonov weight lam > 0: the reported J equals the sum
    |L_c[u] - Gamma|^2 + lam |c|^2 evaluated directly with the operator (not
    through G, g and s), and Adam ends at the minimiser (G + lam I)^-1 g of that
    regularised J (lam = the mean eigenvalue of G keeps the problem well
    conditioned)."""
    nx, ny, nz = 6, 6, 6
    delta, M = 2.5, 2
    u = RNG.standard_normal((3, nz, ny, nx))
    gam = RNG.standard_normal((3, nz, ny, nx))
    G = O.kernel_fit([u], [gam], delta, M, lam=0.0, iters=1)["G"]
    lam = float(np.trace(G)) / G.shape[0]
    fit = O.kernel_fit([u], [gam], delta, M, lam=lam, iters=2000, lr=0.05)
    c = fit["coef"]
    direct = float(((O.kernel_operator(u, c, delta) - gam) ** 2).sum()) + lam * float(c @ c)
    assert fit["loss"] == pytest.approx(direct, rel=1e-12)
    assert np.allclose(c, fit["exact"], rtol=1e-8, atol=0)


def test_kernel_fit_first_adam_step_is_minus_lr_sign_gradient():
    nx, ny, nz = 6, 6, 6
    u = RNG.standard_normal((3, nz, ny, nx))
    gam = RNG.standard_normal((3, nz, ny, nx))
    fit = O.kernel_fit([u], [gam], 2.0, 2, lam=0.5, iters=1, lr=0.1)
    grad0 = -2.0 * fit["g"]                                       # gradient at c = 0
    assert np.allclose(fit["coef"], -0.1 * np.sign(grad0), atol=1e-6)


# ------------------------------------------------------------ Algorithm 3 (displacement-based CG)
def test_cd_homogeneous_medium_is_the_reference_solution():
    """L = L0 everywhere: b^A = div L1 eps^{b(0)} vanishes, so u1 = 0 and eps = eps^{b(0)}
    (+ E) with no iteration, for the plain and the preconditioned forms."""
    dims = (6, 8, 4)
    nx, ny, nz = dims
    c0 = (1.7, 0.9)
    phase = RNG.integers(0, 2, size=(nz, ny, nx)).astype(np.int8)
    b = drop_xi_zero(RNG.standard_normal((3, nz, ny, nx)))
    E = tuple(0.01 * RNG.standard_normal(6))
    xi = O.wavevectors(dims)
    e0h = O.eps_b0_hat(O.fft3(b), xi, *c0)
    e0h[:, 0, 0, 0] = nx * ny * nz * np.array(E)
    for pc in (False, True):
        res = O.solve_cd(phase, [c0, c0], c0, b, E, tol=1e-13, maxit=10, precondition=pc)
        assert res["iters"] == 0 and res["resid"] < 1e-13
        assert np.allclose(res["eps"], np.real(O.ifft3(e0h)), atol=1e-13)


def test_cd_operator_on_a_plane_wave_is_the_navier_acoustic_tensor():
    """Homogeneous (lam, mu): A(u) = -div L grad^s u of u = a cos(xi.x) is K(xi) a cos(xi.x)
    with the acoustic tensor K_ik = mu |xi|^2 d_ik + (lam + mu) xi_i xi_k."""
    dims = (8, 6, 4)
    nx, ny, nz = dims
    lam, mu = 1.3, 0.8
    m = np.array([1, 2, 1])
    xv = 2 * math.pi * m / np.array(dims)
    a = np.array([0.4, -0.1, 0.7])
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny)[None, :, None]
    z = np.arange(nz)[:, None, None]
    ph = xv[0] * x + xv[1] * y + xv[2] * z
    u = np.stack([a[i] * np.cos(ph) for i in range(3)])
    K = mu * (xv @ xv) * np.eye(3) + (lam + mu) * np.outer(xv, xv)
    phase = np.zeros((nz, ny, nx), dtype=np.int8)
    Au = np.real(O.ifft3(O.disp_operator(phase, [(lam, mu)], O.fft3(u), O.wavevectors(dims))))
    Ka = K @ a
    assert np.allclose(Au, np.stack([Ka[i] * np.cos(ph) for i in range(3)]), atol=1e-12)


def _dense_system(dims, phase, table, c0, b, E):
    """The displacement-based system of Algorithm 3 assembled from dense matrices of
    the spectral gradient and divergence (unit-vector columns), independently of
    the oracle's matrix-free operator: A = -Dv L Ds, u^b solving -Dv L0 Ds u^b = b,
    eps^b = E + Ds u^b, b^A = Dv (L - L0) eps^b, and M = (-Dv L0 Ds)^+."""
    nx, ny, nz = dims
    n = nx * ny * nz
    Ds, Dv = _operators(dims)

    def Lmat(lam, mu):
        L = np.zeros((6 * n, 6 * n))
        for c in range(6):
            for p in range(n):
                L[c * n + p, c * n + p] += 2 * mu[p]
                if c < 3:
                    for d in range(3):
                        L[c * n + p, d * n + p] += lam[p]
        return L

    lam = np.array([t[0] for t in table])[phase].ravel()
    mu = np.array([t[1] for t in table])[phase].ravel()
    L = Lmat(lam, mu)
    L0 = Lmat(np.full(n, c0[0]), np.full(n, c0[1]))
    A = -Dv @ L @ Ds
    A0 = -Dv @ L0 @ Ds
    A0p = np.linalg.pinv(A0, rcond=1e-12)
    ub = A0p @ b.ravel()
    eb = np.concatenate([np.full(n, E[c]) for c in range(6)]) + Ds @ ub
    bA = Dv @ ((L - L0) @ eb)
    return A, A0p, bA, eb, Ds


@pytest.mark.parametrize("precondition", [False, True])
def test_cd_iterates_are_textbook_cg_on_the_dense_system(precondition):
    """The oracle's Algorithm 3 after j iterations equals j steps of textbook (P)CG
    from u1 = 0 on the dense system (the same inner product up to the DFT's factor
    |N|, which cancels in alpha and beta): a wrong step length, sign, update order
    or preconditioner changes the iterates at once."""
    dims = (4, 4, 2)
    nx, ny, nz = dims
    r = np.random.default_rng(7)
    phase = r.integers(0, 2, size=(nz, ny, nx)).astype(np.int8)
    table = [(1.0, 0.5), (6.0, 3.0)]
    c0 = (3.5, 1.75)
    b = drop_xi_zero(r.standard_normal((3, nz, ny, nx)))
    E = tuple(0.05 * r.standard_normal(6))
    A, A0p, bA, eb, Ds = _dense_system(dims, phase, table, c0, b, E)
    M = A0p if precondition else np.eye(A.shape[0])
    u = np.zeros_like(bA)
    res_ = bA.copy()
    z = M @ res_
    p = z.copy()
    rz = res_ @ z
    for j in range(1, 7):
        q = A @ p
        al = rz / (p @ q)
        u = u + al * p
        res_ = res_ - al * q
        z = M @ res_
        rz_new = res_ @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        got = O.solve_cd(phase, table, c0, b, E, tol=0.0, maxit=j, precondition=precondition)
        assert got["iters"] == j
        want = (eb + Ds @ u).reshape(6, nz, ny, nx)
        assert np.allclose(got["eps"], want, atol=1e-10 * np.abs(want).max()), (j, precondition)


@pytest.mark.parametrize("precondition", [False, True])
def test_cd_converges_to_the_laminate_closed_form(precondition):
    nx, ny, nz = 16, 2, 2
    lam_ph = [1.0, 10.0]
    mu_ph = [0.5, 5.0]
    layers = np.array([0, 0, 1, 1, 1, 0, 0, 0, 1, 0, 1, 1, 0, 0, 1, 0], dtype=np.int8)
    phase = np.broadcast_to(layers[None, None, :], (nz, ny, nx)).copy()
    b1 = np.random.default_rng(3).standard_normal(nx)
    bh = np.fft.fft(b1)
    bh[0] = 0
    bh[nx // 2] = 0
    b1 = np.real(np.fft.ifft(bh))
    b = np.zeros((3, nz, ny, nx))
    b[0] = b1[None, None, :]
    E = (0.02, 0, 0, 0, 0, 0)
    table = list(zip(lam_ph, mu_ph))
    res = O.solve_cd(phase, table, (5.5, 2.75), b, E, tol=1e-14, maxit=5000, precondition=precondition)
    e11, s11 = laminate_exact(np.array(lam_ph)[layers], np.array(mu_ph)[layers], b1, E[0])
    assert res["resid"] < 1e-13
    assert np.allclose(res["eps"][0], e11[None, None, :], atol=1e-12)
    assert np.allclose(res["eps"][1:], 0, atol=1e-12)
    assert np.allclose(res["sig"][0], s11[None, None, :], atol=1e-11)


def test_cd_residual_is_the_equilibrium_residual_and_matches_the_basic_scheme():
    """The CG residual b^A - A(u1) is i xi . sigma_hat + b_hat (reading R18): its
    history ends at the Eq. 5.11 residual of the returned field; both forms reach
    the fixed point of Algorithm 1, the preconditioned one in far fewer iterations."""
    dims, phase, table, c0 = _c1_small()
    b = O.body_force(dims, (8.0, 8.0, 8.0), 5.0)
    ref = O.solve(phase, table, c0, b, tol=1e-12, maxit=3000)
    its = {}
    for pc in (False, True):
        res = O.solve_cd(phase, table, c0, b, tol=1e-12, maxit=5000, precondition=pc, history=True)
        # (the recursive residual drifts from the true one by rounding: ~1e-16 of D per iteration)
        assert res["resid"] <= 1.01e-12 and abs(res["hist"][-1] - res["resid"]) <= 1e-4 * res["resid"] + 1e-15
        assert np.linalg.norm(res["eps"] - ref["eps"]) <= 1e-9 * np.linalg.norm(ref["eps"])
        assert np.allclose(res["u"], ref["u"], atol=1e-9 * np.abs(ref["u"]).max())
        its[pc] = res["iters"]
    assert its[True] < ref["sweeps"] < its[False]
    # with a mean shear strain the normaliser's sigma_hat(0) has shear parts
    r = np.random.default_rng(11)
    dims = (8, 6, 4)
    phase = r.integers(0, 2, size=(4, 6, 8)).astype(np.int8)
    b = drop_xi_zero(r.standard_normal((3, 4, 6, 8)))
    E = (0.01, -0.002, 0.0, 0.004, -0.003, 0.006)
    res = O.solve_cd(phase, [(1.0, 0.5), (5.0, 2.5)], (3.0, 1.5), b, E, tol=1e-11, maxit=500, precondition=True,
                     history=True)
    assert res["resid"] <= 1.01e-11 and abs(res["hist"][-1] - res["resid"]) <= 1e-4 * res["resid"] + 1e-15
