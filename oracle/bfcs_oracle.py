"""FP64 CPU oracle for the BFCS FFT solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
module: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg
(and its --impl reference arm) use it.  It shares no code with the CUDA path.

It is a plain, slow, obviously-correct restatement of the paper's method
(Buryachenko, "New RVE concept and FFT methods in micromechanics of composites
subjected to body force with compact support"):

  * DFT conventions, Eqs. 4.3-4.5 (forward omega^{-kn}, inverse with 1/|N|),
    evaluated with scipy's FFT (single thread) as the library primitive.
  * Strain Green operator U0 in Fourier space, Eqs. 2.16-2.18, contracted as a
    full fourth-order tensor.
  * Modified Lippmann-Schwinger equation, Eqs. 2.14 / 5.3-5.4, solved by the
    modified basic scheme, Algorithm 1 (Eqs. 5.7-5.10).
  * Reference displacement u^{b(0)} = G0 * b, Eqs. 2.8-2.9, with G0 the inverse
    of the isotropic acoustic tensor.
  * Equilibrium residual, Eq. 5.11 (normalisation read as stated below).
  * Microstructure translation and translated averaging, Eqs. 3.3-3.7.
  * Displacement-based conjugate gradients, Algorithm 3 (Eqs. 5.14-5.22), plain
    as printed and with the reference medium's Green operator as preconditioner.

Readings taken where the paper is silent or garbled (each is listed in the
design notes of the repository):
  R1  wavevector xi_a = 2 pi k_a / N_a with signed index k_a in (-N_a/2, N_a/2)
      and xi_a = 0 on the Nyquist index k_a = N_a/2 (spectral differentiation
      for even N); every operator (U0, G0, divergence) uses this xi, which keeps
      them Hermitian-consistent so that all fields stay real.
  R2  U0 = -Gamma0 (Moulinec-Suquet); the index "h" of Eq. 2.17 is read as l.
  R3  k = 0 mode of the strain = the prescribed mean strain E (DFT scale N*E);
      on the other modes with xi = 0 (Nyquist corners) the strain update is 0
      and the load b is not felt there.
  R4  residual r = ||i xi.sigma_hat + b_hat|| / D over modes with xi != 0,
      D = ||b_hat|| + xi_min |sigma_hat(0)|, xi_min = 2 pi / max N_a.
  R5  stray superscript "^L" in Eq. 5.9 ignored.
  R6  translated averages divide by the number of shifts (Eqs. 3.5-3.6 as
      printed), inclusion-weighted ones included; the hit count is returned.
  R7  translation: L(x, chi) = L0(x - chi) with b fixed (Eq. 3.3).
  R18 Algorithm 3: the right-hand side of Eq. 5.14 is read with L1 = L - L0
      (div L grad^s u1 = -div L1 eps^{b(0)}), the form that follows from Eqs.
      2.10-2.13 and whose solution is that of Eq. 5.3 (with L it would drop the
      body force); the operator is taken with the sign that makes it positive,
      A(u) = -div L grad^s u, and b^A = div L1 eps^{b(0)}; the first iterate is
      u1 = 0 (the printed u1 = b^A is a force, not a displacement); the CG
      residual b^A - A(u1) is then exactly i xi . sigma_hat + b_hat, so the stop
      test is the residual of Eq. 5.11 (reading R4), checked after each update.

Loop convention shared with the GPU path: sweep s forms tau^s = L1 eps^s, its
transform, the residual r(eps^s) and eps^{s+1}.  The solve stops after the
first sweep with r(eps^s) <= tol or after maxit sweeps and returns eps^S
(S = sweeps run) with sigma^S, u^S and r(eps^S).

Layouts: fields are numpy arrays indexed [component][z][y][x]; symmetric
tensors use 6 components (xx, yy, zz, yz, xz, xy), tensorial (not
engineering) shears.

Parity: pinned by the -m "not gpu" tests (direct DFT, Green-operator
identities, homogeneous closed form, plane-wave Navier solution, laminate
closed form, dense brute-force solve, energy identity, Betti reciprocity,
translation equivariance, averaging invariants).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft

# (i, j) of each stored component, Voigt-like order xx yy zz yz xz xy
COMP = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
# stored component index of each (i, j)
IDX = np.array([[0, 5, 4], [5, 1, 3], [4, 3, 2]])


def to_full(v6):
    """(6, ...) symmetric storage -> nested 3x3 list of arrays (views)."""
    return [[v6[IDX[i, j]] for j in range(3)] for i in range(3)]


# ---------------------------------------------------------------- a1 phase map
def phase_map(dims, cell, spheres):
    """Integer voxelisation of spheres in a periodic unit cell (Eqs. 2.21, 3.3).

    dims = (nx, ny, nz) must be multiples of cell = (cx, cy, cz).  A voxel with
    doubled centre 2i+1 lies in a sphere (X, Y, Z, T, phase) when the squared
    periodic minimum-image distance on the doubled grid is <= T.  Later spheres
    overwrite earlier ones; voxels in no sphere are phase 0 (matrix).
    Returns int8 array [z][y][x].
    """
    nx, ny, nz = dims
    cx, cy, cz = cell
    if nx % cx or ny % cy or nz % cz:
        raise ValueError("grid is not a whole number of unit cells")
    ph = np.zeros((cz, cy, cx), dtype=np.int8)

    def dd(n, c):
        d = (2 * np.arange(n, dtype=np.int64) + 1 - c) % (2 * n)
        return np.where(d >= n, d - 2 * n, d)

    for X, Y, Z, T, p in np.asarray(spheres, dtype=np.int64).reshape(-1, 5):
        dx, dy, dz = dd(cx, X), dd(cy, Y), dd(cz, Z)
        d2 = dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2
        ph[d2 <= T] = p
    return np.tile(ph, (nz // cz, ny // cy, nx // cx))


def translate(field, shift):
    """f(x, chi) = f0(x - chi) on the periodic grid (Eq. 3.3); shift = (sx, sy, sz)."""
    sx, sy, sz = (int(s) for s in shift)
    return np.roll(field, (sz, sy, sx), axis=(-3, -2, -1))


# ---------------------------------------------------------------- a2 body force
def body_force(dims, centre, a):
    """BFCS of Eq. 2.5 in the form b = (d phi / d x1, 0, 0), phi = (1 - r^2/a^2)^3
    for r < a, evaluated at voxel centres i + 0.5 with the periodic minimum image
    about `centre`, then made mean-free in FP64.  Returns (3, nz, ny, nx)."""
    nx, ny, nz = dims

    def rel(n, c):
        d = np.arange(n, dtype=np.float64) + 0.5 - c
        return d - n * np.round(d / n)

    x = rel(nx, centre[0])[None, None, :]
    y = rel(ny, centre[1])[None, :, None]
    z = rel(nz, centre[2])[:, None, None]
    r2 = x * x + y * y + z * z
    s = 1.0 - r2 / (a * a)
    b1 = np.where(r2 < a * a, -6.0 * x * s * s / (a * a), 0.0)
    b1 = b1 - b1.mean()
    b = np.zeros((3, nz, ny, nx))
    b[0] = b1
    return b


# ---------------------------------------------------------------- transforms
def fft3(f):
    """Eq. 4.3 on the last three axes (library FFT as the primitive)."""
    return sfft.fftn(f, axes=(-3, -2, -1))


def ifft3(fh):
    """Eq. 4.4 on the last three axes, including 1/|N|."""
    return sfft.ifftn(fh, axes=(-3, -2, -1))


def wavevectors(dims):
    """Reading R1: xi_a = 2 pi k_a / N_a (h = 1), zero on the Nyquist index.
    Returns (xi_x, xi_y, xi_z) shaped to broadcast on [z][y][x]."""
    out = []
    for n in dims:
        k = np.fft.fftfreq(n, d=1.0 / n)          # 0..n/2-1, -n/2..-1
        k[n // 2] = 0.0                            # Nyquist index -> 0
        out.append(2.0 * np.pi * k / n)
    nx, ny, nz = dims
    return (out[0].reshape(1, 1, nx), out[1].reshape(1, ny, 1), out[2].reshape(nz, 1, 1))


# ---------------------------------------------------------------- constitutive
def stiffness(lam, mu):
    """Isotropic L_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk) (P. 2, L = 3k N1 + 2 mu N2)."""
    d = np.eye(3)
    return (lam * np.einsum("ij,kl->ijkl", d, d)
            + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))


def apply_local(phase, table, eps):
    """sigma = L(x) eps pointwise for isotropic phases; table[p] = (lam, mu)."""
    lam = np.asarray([t[0] for t in table])[phase]
    mu = np.asarray([t[1] for t in table])[phase]
    tr = eps[0] + eps[1] + eps[2]
    out = 2.0 * mu * eps
    out[:3] += lam * tr
    return out


# ---------------------------------------------------------------- Green operators
def u0_apply(tau_hat, xi, lam0, mu0):
    """eps_hat_ij = sum_kl U0_ijkl(xi) tau_hat_kl, Eqs. 2.16-2.18, all 81 terms.

    U0 = U1/(4 mu0) + (lam0+mu0)/(mu0 (lam0+2 mu0)) U2,
    U1_ijkl = -(d_ki xi_l xi_j + d_li xi_k xi_j + d_kj xi_l xi_i + d_lj xi_k xi_i)/|xi|^2,
    U2_ijkl = xi_i xi_j xi_k xi_l / |xi|^4.   Modes with xi = 0 give 0.
    With P_ab = xi_a xi_b / |xi|^2 this reads U1_ijkl = -(d_ki P_lj + d_li P_kj
    + d_kj P_li + d_lj P_ki) and U2_ijkl = P_ij P_kl.
    """
    q = xi[0] ** 2 + xi[1] ** 2 + xi[2] ** 2
    nz = q > 0
    iq = np.where(nz, 1.0 / np.where(nz, q, 1.0), 0.0)
    P = [[xi[a] * xi[b] * iq for b in range(3)] for a in range(3)]
    c1 = 1.0 / (4.0 * mu0)
    c2 = (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0))
    t = to_full(tau_hat)
    d = np.eye(3)
    out = np.zeros_like(tau_hat)
    for a, (i, j) in enumerate(COMP):
        acc = 0.0
        for k in range(3):
            for l in range(3):
                u1 = 0.0
                for (delta, pp) in ((d[k, i], P[l][j]), (d[l, i], P[k][j]),
                                    (d[k, j], P[l][i]), (d[l, j], P[k][i])):
                    if delta:
                        u1 = u1 - delta * pp
                u2 = P[i][j] * P[k][l]
                acc = acc + (c1 * u1 + c2 * u2) * t[k][l]
        out[a] = acc
    return out


def g0_apply(v_hat, xi, lam0, mu0):
    """w = G0(xi) v, G0 = K0^{-1} the inverse of the isotropic acoustic tensor
    K0_ik = mu0 |xi|^2 d_ik + (lam0+mu0) xi_i xi_k of the Navier operator
    (Eqs. 2.6, 2.8): G0 = [d_ik - (lam0+mu0)/(lam0+2 mu0) xi_i xi_k/|xi|^2]/(mu0 |xi|^2).
    Modes with xi = 0 give 0."""
    q = xi[0] ** 2 + xi[1] ** 2 + xi[2] ** 2
    nz = q > 0
    iq = np.where(nz, 1.0 / np.where(nz, q, 1.0), 0.0)
    c = (lam0 + mu0) / (lam0 + 2.0 * mu0)
    xv = xi[0] * v_hat[0] + xi[1] * v_hat[1] + xi[2] * v_hat[2]
    return np.stack([(v_hat[i] - c * xi[i] * xv * iq) * iq / mu0 for i in range(3)])


def sym_grad_hat(u_hat, xi):
    """eps_hat = sym(i xi (x) u_hat) in 6-component storage (Eq. 2.3 with Eq. 4.8)."""
    out = np.empty((6,) + np.broadcast_shapes(u_hat[0].shape, xi[0].shape), dtype=complex)
    for a, (i, j) in enumerate(COMP):
        out[a] = 0.5j * (xi[j] * u_hat[i] + xi[i] * u_hat[j])
    return out


def div_hat(s_hat, xi):
    """(i xi . sigma_hat)_i = i sum_j xi_j sigma_hat_ij (Eq. 2.1 with Eq. 4.8)."""
    s = to_full(s_hat)
    return np.stack([1j * (xi[0] * s[i][0] + xi[1] * s[i][1] + xi[2] * s[i][2])
                     for i in range(3)])


def eps_b0_hat(b_hat, xi, lam0, mu0):
    """Reference strain eps^{b(0)} = sym grad (G0 * b), Eqs. 2.8-2.9 and 2.14."""
    return sym_grad_hat(g0_apply(b_hat, xi, lam0, mu0), xi)


# ---------------------------------------------------------------- residual
def residual(phase, table, eps, b_hat, xi):
    """Reading R4 of Eq. 5.11, from sigma = L eps formed in real space."""
    sig_hat = fft3(apply_local(phase, table, eps))
    q = xi[0] ** 2 + xi[1] ** 2 + xi[2] ** 2
    act = np.broadcast_to(q > 0, sig_hat.shape[1:])
    div = div_hat(sig_hat, xi) + b_hat
    num = np.sqrt(np.sum(np.abs(div[:, act]) ** 2))
    s0 = sig_hat[:, 0, 0, 0]
    s0n = np.sqrt(np.sum(np.abs(s0[:3]) ** 2) + 2.0 * np.sum(np.abs(s0[3:]) ** 2))
    dims = sig_hat.shape[1:][::-1]
    den = np.sqrt(np.sum(np.abs(b_hat[:, act]) ** 2)) + 2.0 * np.pi / max(dims) * s0n
    return float(num / den) if den > 0 else float(num)


def _real(fh, what):
    f = ifft3(fh)
    scale = max(np.max(np.abs(f.real)), 1e-300)
    if np.max(np.abs(f.imag)) > 1e-9 * scale:
        raise AssertionError(f"{what}: spectrum is not Hermitian-consistent")
    return f.real.copy()


def displacement(eps, xi, lam0, mu0):
    """Periodic displacement u with sym grad u = eps - <eps> and zero mean:
    u_hat = -i G0(xi) (C0 eps_hat) xi on modes with xi != 0 (from Eq. 2.3)."""
    lam_tr = lam0 * (eps[0] + eps[1] + eps[2])
    c0e = 2.0 * mu0 * eps
    c0e[:3] += lam_tr
    s = to_full(fft3(c0e))
    v = np.stack([xi[0] * s[i][0] + xi[1] * s[i][1] + xi[2] * s[i][2] for i in range(3)])
    return _real(-1j * g0_apply(v, xi, lam0, mu0), "displacement")


# ---------------------------------------------------------------- Algorithm 1
def solve(phase, table, c0, b, mean_strain=(0.0,) * 6, tol=1e-10, maxit=1000,
          eps_init=None, history=False):
    """Modified basic scheme (Algorithm 1, Eqs. 5.7-5.10) for the ML-S equation
    (Eq. 2.14 / 5.3-5.4).  phase: int [z][y][x]; table: [(lam, mu)] per phase;
    c0 = (lam0, mu0); b: (3, nz, ny, nx) mean-free body force; mean_strain E
    (6 components).  Returns dict(eps, sig, u, sweeps, resid, hist)."""
    lam0, mu0 = c0
    nz, ny, nx = phase.shape
    dims = (nx, ny, nz)
    n = nx * ny * nz
    xi = wavevectors(dims)
    b_hat = fft3(b)
    eb0_hat = eps_b0_hat(b_hat, xi, lam0, mu0)
    eb0_hat[:, 0, 0, 0] = n * np.asarray(mean_strain, dtype=float)   # reading R3
    table1 = [(l - lam0, m - mu0) for (l, m) in table]               # L1 = L - L0

    if eps_init is None:
        eps = _real(eb0_hat, "eps0")                 # eps^[0] = eps^{b(0)} (+ E)
    else:
        eps = np.array(eps_init, dtype=float, copy=True)

    hist = []
    sweeps = 0
    for s in range(maxit):
        tau = apply_local(phase, table1, eps)                    # Eq. 5.7
        tau_hat = fft3(tau)                                      # Eq. 5.8
        r = residual(phase, table, eps, b_hat, xi)               # Eq. 5.11, of eps^s
        hist.append(r)
        eps_hat = u0_apply(tau_hat, xi, lam0, mu0) + eb0_hat     # Eq. 5.9 (+ eps^{b(0)})
        eps = _real(eps_hat, "eps")                              # Eq. 5.10
        sweeps = s + 1
        if r <= tol:
            break
    r_final = residual(phase, table, eps, b_hat, xi)
    sig = apply_local(phase, table, eps)
    u = displacement(eps, xi, lam0, mu0)
    out = dict(eps=eps, sig=sig, u=u, sweeps=sweeps, resid=r_final)
    if history:
        out["hist"] = hist
    return out


# ---------------------------------------------------------------- Algorithm 3
def disp_operator(phase, table, u_hat, xi):
    """A(u) = -i xi . F[L F^{-1}(sym(i xi (x) u_hat))]: the Fourier form of
    -div L grad^s u (Eqs. 5.15-5.17, reading R18 for the sign); 3 components."""
    eps = _real(sym_grad_hat(u_hat, xi), "A(u) strain")
    return -div_hat(fft3(apply_local(phase, table, eps)), xi)


def solve_cd(phase, table, c0, b, mean_strain=(0.0,) * 6, tol=1e-10, maxit=1000,
             precondition=False, history=False):
    """Displacement-based CG, Algorithm 3 (Eqs. 5.14-5.22), readings R18, R3, R4.

    Unknown: the displacement fluctuation u1 of Eq. 2.10 (u = u^{b(0)} + u1) in
    Fourier space; eps = eps^{b(0)} + grad^s u1, with the k = 0 mode of eps^{b(0)}
    set to the mean strain E (R3).  Plain CG as printed; precondition=True applies
    the reference medium's G0 (the inverse of -div L0 grad^s) to the residual.
    Iteration j: alpha = (r.z)/(p.A p), u1 += alpha p, r -= alpha A p, z = M^-1 r,
    beta = (r.z)_new/(r.z)_old, p = z + beta p; stop once r(eps^{j+1}) <= tol or
    after maxit iterations.  Inner products over the full complex spectrum.
    Returns dict(eps, sig, u, iters, resid, hist) like solve()."""
    lam0, mu0 = c0
    nz, ny, nx = phase.shape
    dims = (nx, ny, nz)
    n = nx * ny * nz
    xi = wavevectors(dims)
    b_hat = fft3(b)
    eb0_hat = eps_b0_hat(b_hat, xi, lam0, mu0)
    eb0_hat[:, 0, 0, 0] = n * np.asarray(mean_strain, dtype=float)   # reading R3
    eb0 = _real(eb0_hat, "eps_b0")
    table1 = [(l - lam0, m - mu0) for (l, m) in table]
    bA = div_hat(fft3(apply_local(phase, table1, eb0)), xi)         # b^A = div L1 eps^{b(0)}

    def precond(r):
        return g0_apply(r, xi, lam0, mu0) if precondition else r

    def dot(x, y):
        return float(np.real(np.sum(np.conj(x) * y)))

    def resid_of(r, u1_hat):
        # Eq. 5.11 (reading R4): r = i xi . sigma_hat + b_hat on modes with xi != 0
        q = xi[0] ** 2 + xi[1] ** 2 + xi[2] ** 2
        act = np.broadcast_to(q > 0, r.shape[1:])
        num = np.sqrt(np.sum(np.abs(r[:, act]) ** 2))
        eps = eb0 + _real(sym_grad_hat(u1_hat, xi), "eps")
        s0 = fft3(apply_local(phase, table, eps))[:, 0, 0, 0]
        s0n = np.sqrt(np.sum(np.abs(s0[:3]) ** 2) + 2.0 * np.sum(np.abs(s0[3:]) ** 2))
        den = np.sqrt(np.sum(np.abs(b_hat[:, act]) ** 2)) + 2.0 * np.pi / max(dims) * s0n
        return float(num / den) if den > 0 else float(num)

    u1 = np.zeros_like(bA)                     # u1^[0] = 0 (reading R18)
    r = bA.copy()                              # r^[0] = b^A - A(0)
    z = precond(r)
    p = z.copy()
    rz = dot(r, z)
    hist = [resid_of(r, u1)]
    iters = 0
    if hist[0] > tol:
        for j in range(maxit):
            q = disp_operator(phase, table, p, xi)
            alpha = rz / dot(p, q)                                  # Eq. 5.18
            u1 = u1 + alpha * p                                     # Eq. 5.19
            r = r - alpha * q                                       # Eq. 5.20
            z = precond(r)
            rz_new = dot(r, z)
            beta = rz_new / rz                                      # Eq. 5.21
            p = z + beta * p                                        # Eq. 5.22
            rz = rz_new
            iters = j + 1
            hist.append(resid_of(r, u1))
            if hist[-1] <= tol:
                break
    eps = eb0 + _real(sym_grad_hat(u1, xi), "eps")
    sig = apply_local(phase, table, eps)
    u = displacement(eps, xi, lam0, mu0)
    out = dict(eps=eps, sig=sig, u=u, iters=iters, resid=residual(phase, table, eps, b_hat, xi))
    if history:
        out["hist"] = hist
    return out


# ---------------------------------------------------------------- translated averaging
AVG_FIELDS = ("u", "u1", "eps", "eps1", "sig", "sig1")
AVG_WIDTH = {"u": 3, "u1": 3, "eps": 6, "eps1": 6, "sig": 6, "sig1": 6}


def translate_average(phase0, table, c0, b, shifts, mean_strain=(0.0,) * 6,
                      tol=1e-10, maxit=1000):
    """Translated averaging, Eqs. 3.3-3.6: for each integer shift chi the
    microstructure is translated (phase(x) = phase0(x - chi), b fixed), solved,
    and u, V u, eps, V eps, sigma, V sigma are summed and divided by the number
    of shifts (V = indicator of the inclusion phases, phase != 0).  Returns
    (avg (30, nz, ny, nx) in the order <u>, <u>^(1), <eps>, <eps>^(1), <sigma>,
    <sigma>^(1); hits (nz, ny, nx) int = number of shifts with V = 1; infos)."""
    nz, ny, nx = phase0.shape
    acc = np.zeros((30, nz, ny, nx))
    hits = np.zeros((nz, ny, nx), dtype=np.int64)
    infos = []
    for chi in np.asarray(shifts).reshape(-1, 3):
        ph = translate(phase0, chi)
        res = solve(ph, table, c0, b, mean_strain, tol, maxit)
        v = (ph != 0).astype(float)
        acc[0:3] += res["u"]
        acc[3:6] += v * res["u"]
        acc[6:12] += res["eps"]
        acc[12:18] += v * res["eps"]
        acc[18:24] += res["sig"]
        acc[24:30] += v * res["sig"]
        hits += (ph != 0)
        infos.append((res["sweeps"], res["resid"]))
    m = max(len(infos), 1)
    return acc / m, hits, infos


# ---------------------------------------------------------------- ensemble dataset D^d
def ensemble_average(configs, table, c0, b, mean_strain=(0.0,) * 6, tol=1e-10, maxit=1000):
    """Ensemble dataset of Eq. 3.8: the same load b is applied to each of the
    deterministic configurations X^j (phase maps, none derived from another),
    each is solved, and the fields are averaged over the configurations in the
    way Eq. 3.7 averages over translations: u, V u, eps, V eps, sigma, V sigma
    (V the inclusion indicator of the configuration, phase != 0) summed and
    divided by the number of configurations.  Returns (avg (30, nz, ny, nx) in
    the order of translate_average, hits (number of configurations with
    V = 1), infos)."""
    configs = list(configs)
    nz, ny, nx = configs[0].shape
    acc = np.zeros((30, nz, ny, nx))
    hits = np.zeros((nz, ny, nx), dtype=np.int64)
    infos = []
    for ph in configs:
        res = solve(ph, table, c0, b, mean_strain, tol, maxit)
        v = (ph != 0).astype(float)
        acc[0:3] += res["u"]
        acc[3:6] += v * res["u"]
        acc[6:12] += res["eps"]
        acc[12:18] += v * res["eps"]
        acc[18:24] += res["sig"]
        acc[24:30] += v * res["sig"]
        hits += (ph != 0)
        infos.append((res["sweeps"], res["resid"]))
    return acc / len(configs), hits, infos


# ---------------------------------------------------------------- RVE size (Def. 2.2)
def radial_profile(field, centre, nbins):
    """Largest pointwise norm of `field` in each spherical shell about `centre`:
    prof[k] = max |f(x)| over voxels x whose periodic minimum-image distance d
    from the centre satisfies k <= d < k + 1 (voxel centres at i + 0.5; the
    centre on the half-voxel lattice, so that every d^2 is a quarter integer
    and the shell of a voxel is decided exactly).  |f| is the Euclidean norm
    of a vector (3 components) or sqrt(f : f) of a symmetric tensor (6
    components, shears counted twice).  Empty shells give 0.  Returns (prof,
    counts)."""
    f = np.asarray(field, dtype=np.float64)
    ncomp, nz, ny, nx = f.shape
    w = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0] if ncomp == 6 else [1.0] * ncomp)
    norm = np.sqrt(np.tensordot(w, f * f, axes=(0, 0)))
    c2 = [int(round(2 * c)) for c in centre]
    if any(abs(2 * c - k) > 1e-12 for c, k in zip(centre, c2)):
        raise ValueError("the centre must lie on the half-voxel lattice")

    def dd(n, c):
        d = (2 * np.arange(n, dtype=np.int64) + 1 - c) % (2 * n)
        return np.where(d > n, d - 2 * n, d)

    dx, dy, dz = dd(nx, c2[0]), dd(ny, c2[1]), dd(nz, c2[2])
    D2 = dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2   # (2 d)^2
    shell = np.floor(np.sqrt(D2.astype(np.float64)) / 2.0).astype(np.int64)        # exact: see pins
    prof = np.zeros(nbins)
    counts = np.zeros(nbins, dtype=np.int64)
    inside = shell < nbins
    np.maximum.at(prof, shell[inside], norm[inside])
    np.add.at(counts, shell[inside], 1)
    return prof, counts


def rve_radius(profiles, tol_f, rmax):
    """RVE radius of Def. 2.2 from shell profiles: the smallest r such that in
    every shell k with r <= k < rmax each profile is at most tol_f times its
    largest value (fields vanish outside the RVE, relative to their maximum).
    None when even the outermost shell rmax - 1 exceeds that."""
    r = 0
    for prof in profiles:
        lim = tol_f * prof[:rmax].max()
        above = np.nonzero(prof[:rmax] > lim)[0]
        rp = 0 if above.size == 0 else int(above[-1]) + 1
        if rp >= rmax:
            return None
        r = max(r, rp)
    return r


def rve_size(cell, spheres, table, c0, a, sizes, tol=1e-8, tol_f=1e-3, maxit=4000):
    """RVE-size loop (Def. 2.2; Sec. 5: enlarge the body-force unit cell until
    the RVE lies inside it): for each cubic grid n in `sizes` (multiples of the
    microstructure cell), the BFCS problem of radius a centred at the cell
    corner nearest the grid centre is solved, the RVE radius is taken from the
    shell profiles of eps and sigma up to rmax = n / 2, and the grid is accepted
    when the RVE and an annulus of half the support radius fit inside it,
    r + a / 2 <= n / 2.  Stops at the first accepted grid.  Returns one record
    per grid solved."""
    out = []
    for n in sizes:
        dims = (n, n, n)
        ph = phase_map(dims, cell, spheres)
        centre = tuple(float(k * int(np.floor(n / (2.0 * k) + 0.5))) for k in cell)
        b = body_force(dims, centre, a)
        res = solve(ph, table, c0, b, tol=tol, maxit=maxit)
        rmax = n // 2
        pe, _ = radial_profile(res["eps"], centre, rmax)
        ps, _ = radial_profile(res["sig"], centre, rmax)
        r = rve_radius([pe, ps], tol_f, rmax)
        ok = r is not None and r + a / 2.0 <= n / 2.0
        out.append(dict(n=n, centre=centre, r_rve=r, contained=ok, sweeps=res["sweeps"], resid=res["resid"],
                        prof_eps=pe, prof_sig=ps))
        if ok:
            break
    return out


# ---------------------------------------------------------------- nonlocal kernel regression (Eqs. 6.5-6.6)
def bernstein(M, t):
    """Bernstein basis of degree M on [0, 1]: B_m(t) = C(M, m) t^m (1 - t)^(M - m), m = 0..M."""
    t = np.asarray(t, dtype=np.float64)
    return np.stack([math.comb(M, m) * t ** m * (1.0 - t) ** (M - m) for m in range(M + 1)])


def horizon_offsets(delta):
    """Integer voxel offsets xi with 0 < |xi| < delta (h = 1)."""
    r = int(math.ceil(delta))
    g = np.arange(-r, r + 1)
    off = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    d = np.sqrt((off.astype(np.float64) ** 2).sum(axis=1))
    keep = (d > 0) & (d < delta)
    return off[keep], d[keep]


def kernel_operator(u, coef, delta):
    """The nonlocal operator of Eq. 6.5 on the periodic voxel grid for the
    radial kernel K(r) = sum_m coef_m B_m(r / delta) (r < delta, 0 beyond):
    L[u](x) = sum over offsets 0 < |xi| < delta of K(|xi|) (u(x + xi) - u(x)),
    a direct sum (voxel volume 1).  u: (3, nz, ny, nx)."""
    coef = np.asarray(coef, dtype=np.float64)
    off, d = horizon_offsets(delta)
    K = coef @ bernstein(coef.size - 1, d / delta)
    out = np.zeros_like(u, dtype=np.float64)
    for (ox, oy, oz), k in zip(off, K):
        out += k * (np.roll(u, (-oz, -oy, -ox), axis=(-3, -2, -1)) - u)
    return out


def kernel_fit(us, gammas, delta, M, lam, iters=2000, lr=0.05, betas=(0.9, 0.999), eps=1e-8):
    """Kernel regression of Eq. 6.6 for gamma = b (Gamma_k = -b_k, u_k the
    averaged displacement of load k): minimise
      J(c) = sum_k sum_x |L_c[u_k](x) - Gamma_k(x)|^2 + lam |c|^2
    (Tikhonov regularisation) over the Bernstein coefficients c of K.  J is
    quadratic: with A_m = L_{e_m}, G_mn = sum_k <A_m u_k, A_n u_k>, g_m =
    sum_k <A_m u_k, Gamma_k> and s = sum_k |Gamma_k|^2, J = c.G.c - 2 g.c + s +
    lam |c|^2.  Returns the Adam iterate from c = 0 after `iters` steps (Adam,
    Kingma and Ba 2015: first/second moment averages with bias correction) with
    its J, the exact minimiser (G + lam I)^-1 g, G, g and s."""
    n = M + 1
    G = np.zeros((n, n))
    g = np.zeros(n)
    s = 0.0
    for u, gam in zip(us, gammas):
        A = [kernel_operator(u, np.eye(n)[m], delta) for m in range(n)]
        for a in range(n):
            g[a] += float((A[a] * gam).sum())
            for b in range(n):
                G[a, b] += float((A[a] * A[b]).sum())
        s += float((gam * gam).sum())
    exact = np.linalg.solve(G + lam * np.eye(n), g)
    c = np.zeros(n)
    m1 = np.zeros(n)
    v = np.zeros(n)
    for t in range(1, iters + 1):
        grad = 2.0 * (G @ c - g + lam * c)
        m1 = betas[0] * m1 + (1 - betas[0]) * grad
        v = betas[1] * v + (1 - betas[1]) * grad * grad
        mh = m1 / (1 - betas[0] ** t)
        vh = v / (1 - betas[1] ** t)
        c = c - lr * mh / (np.sqrt(vh) + eps)
    J = float(c @ G @ c - 2 * g @ c + s + lam * c @ c)
    return dict(coef=c, loss=J, exact=exact, G=G, g=g, s=s)


# ---------------------------------------------------------------- effective moduli and concentration
def unit_strain(J):
    """Unit mean strain of tensorial component J (xx yy zz yz xz xy): for a shear
    J both symmetric entries are 1."""
    E = [0.0] * 6
    E[J] = 1.0
    return tuple(E)


def effective_moduli(phase, table, c0, tol=1e-12, maxit=4000):
    """Effective stiffness L* of Eq. 6.3 (<sigma> = L* <eps>, averages of Eqs.
    6.1-6.2 over the unit cell) and strain concentration A* of Eq. 3.2 (<eps>_i =
    A* <eps>, <.>_i the average over the inclusion voxels, phase != 0): six
    solves with b = 0 and the unit mean strains of unit_strain(J) (the classical
    problem, Eq. 2.24).  Column J of each 6 x 6 matrix is the response to
    unit_strain(J) in tensorial components.  A* is NaN when there is no
    inclusion voxel."""
    nz, ny, nx = phase.shape
    b = np.zeros((3, nz, ny, nx))
    incl = phase != 0
    Ls = np.zeros((6, 6))
    As = np.full((6, 6), np.nan)
    for J in range(6):
        res = solve(phase, table, c0, b, unit_strain(J), tol=tol, maxit=maxit)
        Ls[:, J] = res["sig"].reshape(6, -1).mean(axis=1)
        if incl.any():
            As[:, J] = res["eps"][:, incl].mean(axis=1)
    return Ls, As
