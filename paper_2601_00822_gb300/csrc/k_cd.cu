// Displacement-based conjugate gradients, Algorithm 3 (Eqs. 5.14-5.22): the
// unknown is the displacement fluctuation u1 of Eq. 2.10 (u = u^{b(0)} + u1),
// held as a fully transformed half spectrum of three components, and the system
// is A(u1) = b^A with the positive operator A(u) = -i xi . F[L F^-1(sym(i xi (x)
// u_hat))] and b^A = i xi . F[L1 eps^{b(0)}] (Eq. 5.14 with L1 = L - L0 on the
// right, the form that follows from Eqs. 2.10-2.13).  The CG residual b^A - A(u1)
// is then the equilibrium defect i xi . sigma_hat + b_hat of the strain
// eps = eps^{b(0)} + grad^s u1, so the stop test is the residual of Eq. 5.11.
// Optional preconditioner: the reference medium's G0 (the inverse of -div L0
// grad^s), applied per mode.  Inner products run over the full spectrum: stored
// modes weighted 1 at kx = 0 and kx = nx/2 and 2 elsewhere (Hermitian pairs);
// per-mode products in the vectors' precision, sums in FP64.  Every kernel is
// batched over members (blockIdx.y) and a finished member returns at entry; the
// scalars alpha, beta, the residual and the stop test are formed on the device.
#include "kernels.h"

#ifndef BFCS_R
#define BFCS_R float
#endif

namespace bfcs {

constexpr int kCdThreads = 256;

namespace {

__device__ __forceinline__ double cd_reduce(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
  __syncthreads();
  return t;
}

// v = G0(xi) w: the inverse of the isotropic acoustic tensor mu0 |xi|^2 I + (lam0 +
// mu0) xi xi (Eqs. 2.6, 2.8), per mode; g0c = {(lam0 + mu0) / (lam0 + 2 mu0), 1 / mu0}
template <typename R> struct G0c { R c, inv_mu0; };
template <typename R> __device__ __forceinline__ G0c<R> g0_consts(double lam0, double mu0) {
  const R l = R(lam0), m = R(mu0);      // in R: no FP64 division on the device
  return G0c<R>{(l + m) / (l + R(2) * m), R(1) / m};
}
template <typename R>
__device__ __forceinline__ void cd_g0(const C2<R> (&w)[3], const R (&xi)[3], R qq, G0c<R> g0c, C2<R> (&v)[3]) {
  const R iq = R(1) / qq;
  const R f = iq * g0c.inv_mu0;
  const C2<R> xw = scale(w[0], xi[0]) + scale(w[1], xi[1]) + scale(w[2], xi[2]);
#pragma unroll
  for (int k = 0; k < 3; ++k) v[k] = scale(w[k] - scale(xw, g0c.c * xi[k] * iq), f);
}


// sym(i xi (x) v) in 6-component storage (xx yy zz yz xz xy), times f
template <typename R>
__device__ __forceinline__ void cd_symgrad(const C2<R> (&v)[3], const R (&xi)[3], R f, C2<R> (&e)[6]) {
  auto ih = [&](C2<R> a, R s) { return mk<R>(-a.y * s, a.x * s); };   // i a s
  const R h = R(0.5) * f;
  e[0] = ih(scale(v[0], xi[0]), f);
  e[1] = ih(scale(v[1], xi[1]), f);
  e[2] = ih(scale(v[2], xi[2]), f);
  e[3] = ih(scale(v[2], xi[1]) + scale(v[1], xi[2]), h);
  e[4] = ih(scale(v[2], xi[0]) + scale(v[0], xi[2]), h);
  e[5] = ih(scale(v[1], xi[0]) + scale(v[0], xi[1]), h);
}

// i xi . s for a symmetric tensor s in 6-component storage
template <typename R>
__device__ __forceinline__ void cd_div(const C2<R> (&s)[6], const R (&xi)[3], C2<R> (&d)[3]) {
  const C2<R> v0 = scale(s[0], xi[0]) + scale(s[5], xi[1]) + scale(s[4], xi[2]);
  const C2<R> v1 = scale(s[5], xi[0]) + scale(s[1], xi[1]) + scale(s[3], xi[2]);
  const C2<R> v2 = scale(s[4], xi[0]) + scale(s[3], xi[1]) + scale(s[2], xi[2]);
  d[0] = mk<R>(-v0.y, v0.x);
  d[1] = mk<R>(-v1.y, v1.x);
  d[2] = mk<R>(-v2.y, v2.x);
}

template <typename R>
__device__ __forceinline__ R cd_dot3(const C2<R> (&a)[3], const C2<R> (&b)[3]) {
  R s = R(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) s += a[k].x * b[k].x + a[k].y * b[k].y;
  return s;
}

}  // namespace

// Modes (CdMode):
//  INIT:    r = b^A = i xi . s (s: F[L1 eps^{b(0)}], 6 components), u = 0, p = z = M r;
//           partials <r, z>, <r, r>; the k = 0 thread stores s(0) in cd.s0b
//  (z = M r is never stored: every step that needs it forms it from r)
//  UPDATE:  r -= alpha q; partials <r, M r>, <r, r> (u += alpha p is taken by the
//           direction step of the fused inverse z kernel, which reads p anyway)
//  FINAL:   s = sym(i xi (x) (G0 b_hat + u)) / N, s(0) = E (the returned strain)
//  FINAL_U: s = (G0 b_hat + u) / N in components 0..2 (the returned displacement)
//  RESID:   partial |i xi . s + b_hat|^2 over xi != 0 (s: F[L eps]); s(0) into cd.s0u
//  (FINAL and FINAL_U add the last alpha p first when an update step ended the member)
// The products q = A p and <p, q> (PQ) and the direction step (DIR) run fused with
// the z transforms, in k_zcd.
template <typename R>
__global__ void __launch_bounds__(kCdThreads) k_cd_vec(CdArgs<R> a, int mode) {
  const int m = blockIdx.y;
  const bool all = mode == CdMode::FINAL || mode == CdMode::FINAL_U || mode == CdMode::RESID;
  if (!all && a.cd[m].done) return;
  __shared__ double red[32];
  const Geo g = a.g;
  C2<R>* const u = a.u + m * a.ms;
  C2<R>* const r = a.r + m * a.ms;
  C2<R>* const p = a.p + m * a.ms;
  C2<R>* const q = a.q + m * a.ms;
  C2<R>* const s = a.s + m * a.sms;
  const C2<R>* const bh = a.bhat + m * a.b_ms;
  __shared__ R cst[3];          // alpha and G0's constants, converted once per block
  if (threadIdx.x == 0) {
    const G0c<R> c = g0_consts<R>(a.lam0, a.mu0);
    cst[0] = (R)a.cd[m].alpha;
    cst[1] = c.c;
    cst[2] = c.inv_mu0;
  }
  __syncthreads();
  const R alpha = cst[0];
  const G0c<R> g0c{cst[1], cst[2]};
  const R inv_n = R(1) / R(g.n);
  const R two_pi = R(6.283185307179586);
  const R dk0 = two_pi / R(g.nx), dk1 = two_pi / R(g.ny), dk2 = two_pi / R(g.nz);
  const long long modes = (long long)g.nz * g.ny * g.mx;
  // partial sums: 16 grid-stride modes in R (their products are R), then one FP64 add,
  // so few FP64 instructions run (GB300 issues FP64 at a small fraction of the FP32 rate)
  double acc1 = 0.0, acc2 = 0.0;
  const int stride = gridDim.x * blockDim.x;
  // 32-bit index arithmetic: a member's spectrum has at most 256 * 256 * 129 modes
  for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < (int)modes; i0 += 16 * stride) {
    R p1 = R(0), p2 = R(0);
    for (int j = 0; j < 16; ++j) {
      const int i = i0 + j * stride;
      if (i >= (int)modes) break;
      const int kx = i % g.mx;
      const int rr = i / g.mx;
      const int ky = rr % g.ny, kz = rr / g.ny;
      const long long gi = (long long)rr * g.p + kx;
      const R w = (kx == 0 || 2 * kx == g.nx) ? R(1) : R(2);
      R xi[3];
      xi[0] = dk0 * R(signed_k(kx, g.nx));
      xi[1] = dk1 * R(signed_k(ky, g.ny));
      xi[2] = dk2 * R(signed_k(kz, g.nz));
      const R qq = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
      const bool nz = qq != R(0);
      auto ld3 = [&](const C2<R>* v, C2<R> (&o)[3]) {
#pragma unroll
        for (int k = 0; k < 3; ++k) o[k] = v[k * g.cs + gi];
      };
      auto st3 = [&](C2<R>* v, const C2<R> (&o)[3]) {
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k * g.cs + gi] = o[k];
      };
      auto ld6 = [&](C2<R> (&o)[6]) {
#pragma unroll
        for (int k = 0; k < 6; ++k) o[k] = s[k * g.cs + gi];
      };
      auto precond = [&](const C2<R> (&x)[3], C2<R> (&y)[3]) {
        if (a.precond && nz) {
          cd_g0<R>(x, xi, qq, g0c, y);
        } else {
#pragma unroll
          for (int k = 0; k < 3; ++k) y[k] = a.precond ? mk<R>(0, 0) : x[k];
        }
      };
      if (mode == CdMode::INIT) {
        C2<R> t[6], rv[3], zv[3];
        ld6(t);
        if (i == 0) {
#pragma unroll
          for (int k = 0; k < 6; ++k) a.cd[m].s0b[k] = (double)t[k].x;
        }
        cd_div<R>(t, xi, rv);
        if (!nz) rv[0] = rv[1] = rv[2] = mk<R>(0, 0);
        precond(rv, zv);
        const C2<R> zero[3] = {mk<R>(0, 0), mk<R>(0, 0), mk<R>(0, 0)};
        st3(r, rv);
        st3(p, zv);      // p = z (the direction step then forms the operator input with beta = 0)
        st3(u, zero);
        p1 += w * cd_dot3<R>(rv, zv);
        p2 += w * cd_dot3<R>(rv, rv);
      } else if (mode == CdMode::UPDATE) {
        // r -= alpha q; u1 += alpha p follows in the direction step, which reads p anyway
        C2<R> rv[3], qv[3], zv[3];
        ld3(r, rv);
        ld3(q, qv);
#pragma unroll
        for (int k = 0; k < 3; ++k) rv[k] = rv[k] - scale(qv[k], alpha);
        precond(rv, zv);                 // z = M r is formed where it is used, not stored
        st3(r, rv);
        p1 += w * cd_dot3<R>(rv, zv);
        p2 += w * cd_dot3<R>(rv, rv);
      } else if (mode == CdMode::FINAL || mode == CdMode::FINAL_U) {
        C2<R> uv[3], bv[3], gb[3] = {mk<R>(0, 0), mk<R>(0, 0), mk<R>(0, 0)};
        ld3(u, uv);
        if (a.cd[m].pend) {              // the last update's alpha p, not yet added by a direction step
          C2<R> pv[3];
          ld3(p, pv);
#pragma unroll
          for (int k = 0; k < 3; ++k) uv[k] = uv[k] + scale(pv[k], alpha);
        }
        ld3(bh, bv);
        if (nz) cd_g0<R>(bv, xi, qq, g0c, gb);
#pragma unroll
        for (int k = 0; k < 3; ++k) uv[k] = uv[k] + gb[k];      // u_hat = G0 b_hat + u1_hat (Eqs. 2.8, 2.10)
        if (mode == CdMode::FINAL_U) {
#pragma unroll
          for (int k = 0; k < 3; ++k) s[k * g.cs + gi] = nz ? scale(uv[k], inv_n) : mk<R>(0, 0);
        } else {
          C2<R> e[6];
          cd_symgrad<R>(uv, xi, inv_n, e);
          const double* E = a.mem[m].E;
#pragma unroll
          for (int k = 0; k < 6; ++k) s[k * g.cs + gi] = nz ? e[k] : mk<R>(0, 0);
          if (i == 0)                  // xi = 0: the prescribed mean strain
#pragma unroll
            for (int k = 0; k < 6; ++k) s[k * g.cs + gi] = mk<R>((R)E[k], R(0));
        }
      } else {   // RESID
        C2<R> t[6], d[3], bv[3];
        ld6(t);
        if (i == 0) {
#pragma unroll
          for (int k = 0; k < 6; ++k) a.cd[m].s0u[k] = (double)t[k].x;
        }
        if (nz) {
          cd_div<R>(t, xi, d);
          ld3(bh, bv);
#pragma unroll
          for (int k = 0; k < 3; ++k) d[k] = d[k] + bv[k];
          p1 += w * cd_dot3<R>(d, d);
        }
      }
    }
    acc1 += (double)p1;
    acc2 += (double)p2;
  }
  if (mode == CdMode::FINAL || mode == CdMode::FINAL_U) return;
  const double t1 = cd_reduce(acc1, red);
  const double t2 = cd_reduce(acc2, red);
  if (threadIdx.x == 0) {
    a.part[((long long)m * gridDim.x + blockIdx.x) * 2] = t1;
    a.part[((long long)m * gridDim.x + blockIdx.x) * 2 + 1] = t2;
  }
}

// |sigma_hat(0)|_F with shear components counted twice (Eq. 5.11 normaliser)
__device__ __forceinline__ double cd_s0norm(const double (&s)[6]) {
  return sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + 2.0 * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]));
}

// Per member: sums its partials in a fixed order and advances its scalars.
//  INIT:   rz = <r, z>; residual of eps^{b(0)} (sigma_hat(0) = s0b + N L0 E); done at
//          r <= tol or maxit = 0
//  PQ:     alpha = rz / <p, A p> (a non-positive <p, A p> ends the member: breakdown)
//  UPDATE: beta = <r, z>_new / rz; s0u += alpha s0p; iterations + 1; residual from
//          <r, r>; done at r <= tol, NaN or the iteration limit
//  RESID:  the residual of the returned strain into resid_final
// The skip flags of the FFT passes follow done; the member's IterState receives the
// iteration count, residuals and status fields read by the host.
static __global__ void k_cd_scalar(const double* part, int nparts, CdState* cd, IterState* skip, IterState* ist,
                                   const Member* mem, double lam0, double mu0, double n, int maxdim, int mode) {
  __shared__ double red[32];
  const int m = blockIdx.x;
  CdState& S = cd[m];
  if (mode != CdMode::RESID && S.done) return;
  double a1 = 0.0, a2 = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    a1 += part[((long long)m * nparts + i) * 2];
    a2 += part[((long long)m * nparts + i) * 2 + 1];
  }
  const double t1 = cd_reduce(a1, red);
  const double t2 = cd_reduce(a2, red);
  if (threadIdx.x != 0) return;
  IterState& st = ist[m];
  const double xmin = 6.283185307179586 / (double)maxdim;
  auto resid = [&](const double (&s0)[6], double rr) {
    const double den = st.bden + xmin * cd_s0norm(s0);
    return den > 0.0 ? sqrt(rr) / den : sqrt(rr);
  };
  bool fin = false;
  if (mode == CdMode::INIT) {
    const double* E = mem[m].E;
    const double trE = E[0] + E[1] + E[2];
    for (int k = 0; k < 6; ++k) {
      // sigma_hat(0) of L eps^{b(0)} = F[L1 eps^{b(0)}](0) + N L0 E
      S.s0b[k] += n * ((k < 3 ? lam0 * trE : 0.0) + 2.0 * mu0 * E[k]);
      S.s0u[k] = 0.0;
    }
    S.rz = t1;
    S.iters = 0;
    S.alpha = 0.0;     // the first direction step adds nothing to u = 0
    S.beta = 0.0;
    S.resid = resid(S.s0b, t2);
    st.resid_last = S.resid;
    if (!(S.resid == S.resid)) { S.status = 3; fin = true; }
    else if (S.resid <= S.tol) { S.status = 1; fin = true; }
    else if (S.maxit <= 0) { S.status = 2; fin = true; }
  } else if (mode == CdMode::PQ) {
    if (t1 > 0.0 && t1 == t1) {
      S.alpha = S.rz / t1;
    } else {
      S.status = 3;
      fin = true;
    }
  } else if (mode == CdMode::UPDATE) {
    S.beta = S.rz > 0.0 ? t1 / S.rz : 0.0;
    S.rz = t1;
    for (int k = 0; k < 6; ++k) S.s0u[k] += S.alpha * S.s0p[k];
    S.iters += 1;
    double s0[6];
    for (int k = 0; k < 6; ++k) s0[k] = S.s0b[k] + S.s0u[k];
    S.resid = resid(s0, t2);
    st.resid_last = S.resid;
    if (!(S.resid == S.resid)) { S.status = 3; fin = true; }
    else if (S.resid <= S.tol) { S.status = 1; fin = true; }
    else if (S.iters >= S.maxit) { S.status = 2; fin = true; }
    S.pend = fin ? 1 : 0;
  } else {   // RESID: the true residual of the returned strain (s0u holds its sigma_hat(0))
    st.resid_final = resid(S.s0u, t1);
    st.iters = S.iters;
    st.done = S.status == 1 ? 1 : 0;
    st.diverged = S.status == 3 ? 1 : 0;
    return;
  }
  if (fin) {
    S.done = 1;
    skip[m].done = 1;
  }
}

// ---------------------------------------------------------------- fused z passes
// The operator's z transforms fused with the pointwise CG steps next to them, in
// the tile of the z/Green pass: a block holds T = 4 kx columns of one ky row for
// all L z modes of the 6 components (24 line columns), its shared-memory slots
// swizzled by row (components swap in every other pair of rows), and runs the
// four-step line FFT in registers and shared memory.
//  forward (ZFWD): stage 1 from global memory, stage 2, then per mode
//     q = -i xi . sigma_hat (stored), the partial <p, q> and sigma_hat(0)  (PQ)
//  inverse (ZINV): per mode u += alpha p and p = M r + beta p (both stored) and
//     sym(i xi (x) p) / N into the tile (DIR), then the inverse transform written to
//     the work spectrum
constexpr int kCdT = 4;
constexpr int kCdNcol = 6 * kCdT;
template <int L> struct ZCfg {
  static constexpr int TASKS = kCdNcol * LineInfo<L>::RMAX;
  static constexpr int BLOCK = (TASKS + 31) / 32 * 32;
};
__device__ __forceinline__ int cd_slot(int row, int c) { return c ^ (((row >> 1) & 1) << 2); }

template <typename R, int L, bool FWD>
__global__ void __launch_bounds__(ZCfg<L>::BLOCK) k_zcd(CdArgs<R> a) {
  const int m = blockIdx.z;
  if (a.cd[m].done) return;
  constexpr int T = kCdT, NCOL = kCdNcol;
  constexpr int R1 = LineInfo<L>::R1, R2 = LineInfo<L>::R2;
  constexpr int TASKS = ZCfg<L>::TASKS;
  extern __shared__ unsigned char smem_cd[];
  C2<R>* const sm = reinterpret_cast<C2<R>*>(smem_cd);          // [n][slot], L x NCOL
  C2<R>* const pre = sm + L * NCOL;                             // p (forward) or u (inverse) tile [arr][n][col]
  __shared__ double red[32];
  const Geo g = a.g;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int ky = blockIdx.y, col0 = blockIdx.x * T;
  const long long zs = (long long)g.ny * g.p, rowbase = (long long)ky * g.p;
  C2<R>* const s = a.s + m * a.sms;
  const long long vo = m * a.ms;
  auto column = [&](int c) { const int q = c / T; return s + q * g.cs + rowbase + col0 + (c - q * T); };
  const R two_pi = R(6.283185307179586);
  const R dk0 = two_pi / R(g.nx), dk1 = two_pi / R(g.ny), dk2 = two_pi / R(L);
  // 16-byte copies of [arr][n][col] tiles of 3-component vectors (T columns of every row)
  constexpr int PER = 16 / sizeof(C2<R>);
  constexpr int CPR = T / PER;
  auto stage = [&](C2<R>* dst, const C2<R>* v, int arr0) {
    for (int idx = tid; idx < 3 * L * CPR; idx += nthr) {
      const int part = idx % CPR, n = (idx / CPR) % L, arr = idx / (CPR * L);
      cp_async16(dst + ((arr0 + arr) * L + n) * T + part * PER, v + vo + arr * g.cs + n * zs + rowbase + col0 + part * PER);
    }
  };
  R acc = R(0);                 // this thread's <p, q> share (at most a few modes)
  if (FWD) {
    stage(pre, a.p, 0);                                         // p lands during the transform
    cp_async_commit();
    for (int task = tid; task < TASKS; task += nthr) {
      const int c = task % NCOL, j = task / NCOL;
      if (j >= R2) continue;
      const bool cvalid = col0 + (c % T) < g.mx;
      const C2<R>* gcol = column(c);
      C2<R> x[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) x[n1] = cvalid ? gcol[(R2 * n1 + j) * zs] : mk<R>(0, 0);
      stage1<R, L, -1>(x, j, a.tw);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) sm[(j * R1 + k1) * NCOL + cd_slot(j * R1 + k1, c)] = x[k1];
    }
    __syncthreads();
    for (int task = tid; task < TASKS; task += nthr) {
      const int c = task % NCOL, j = task / NCOL;
      if (j >= R1) continue;
      C2<R> y[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) y[n2] = sm[(n2 * R1 + j) * NCOL + cd_slot(n2 * R1 + j, c)];
      stage2<R, L, -1>(y);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) sm[(j + R1 * k2) * NCOL + cd_slot(j + R1 * k2, c)] = y[k2];
    }
    cp_async_wait_all();
    __syncthreads();
    for (int idx = tid; idx < T * L; idx += nthr) {
      const int col = idx % T, n = idx / T;
      const int kx = col0 + col;
      if (kx >= g.mx) continue;
      C2<R>* const mrow = sm + n * NCOL + col;
      const int qs = (n >> 1) & 1;
      C2<R> t[6], qv[3];
#pragma unroll
      for (int q = 0; q < 6; ++q) t[q] = mrow[(q ^ qs) * T];
      if (kx == 0 && ky == 0 && n == 0) {
#pragma unroll
        for (int q = 0; q < 6; ++q) a.cd[m].s0p[q] = (double)t[q].x;
      }
      R xi[3];
      xi[0] = dk0 * R(signed_k(kx, g.nx));
      xi[1] = dk1 * R(signed_k(ky, g.ny));
      xi[2] = dk2 * R(signed_k(n, L));
      const bool nz = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2] != R(0);
      cd_div<R>(t, xi, qv);
      const long long gi = n * zs + rowbase + kx;
      R dot = R(0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        qv[k] = nz ? mk<R>(-qv[k].x, -qv[k].y) : mk<R>(0, 0);
        a.q[vo + k * g.cs + gi] = qv[k];
        const C2<R> pk = pre[(k * L + n) * T + col];
        dot += pk.x * qv[k].x + pk.y * qv[k].y;
      }
      acc += ((kx == 0 || 2 * kx == g.nx) ? R(1) : R(2)) * dot;
    }
    // the warp's 32 shares in R (the products themselves are R), warps in FP64
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((tid & 31) == 0) red[tid >> 5] = (double)acc;
    __syncthreads();
    if (tid == 0) {
      double tsum = 0.0;
      for (int w = 0; w < nthr / 32; ++w) tsum += red[w];
      const long long slot = (long long)m * gridDim.x * gridDim.y + (long long)blockIdx.y * gridDim.x + blockIdx.x;
      a.part[slot * 2] = tsum;
      a.part[slot * 2 + 1] = 0.0;
    }
    return;
  }
  // ---- inverse: r (arrays 0-2) and p (3-5) of mode (n, col) land in the six tile slots
  // its strain spectrum will take (row n, slots (q ^ qs) T + col), so each mode is read
  // and rewritten by one thread; u lands in the extra tile
  {
    constexpr int PER = 16 / sizeof(C2<R>);
    constexpr int CPR = T / PER;
    for (int idx = tid; idx < 6 * L * CPR; idx += nthr) {
      const int part = idx % CPR, n = (idx / CPR) % L, arr = idx / (CPR * L);
      const C2<R>* v = arr < 3 ? a.r + arr * g.cs : a.p + (arr - 3) * g.cs;
      const int qs = (n >> 1) & 1;
      cp_async16(sm + n * NCOL + (arr ^ qs) * T + part * PER, v + vo + n * zs + rowbase + col0 + part * PER);
    }
  }
  stage(pre, a.u, 0);
  cp_async_commit();
  __shared__ R cst[4];          // alpha, beta and G0's constants, converted once per block
  if (tid == 0) {
    const G0c<R> g0c = g0_consts<R>(a.lam0, a.mu0);
    cst[0] = (R)a.cd[m].alpha;
    cst[1] = (R)a.cd[m].beta;
    cst[2] = g0c.c;
    cst[3] = g0c.inv_mu0;
  }
  cp_async_wait_all();
  __syncthreads();
  const R alpha = cst[0], beta = cst[1];
  const G0c<R> g0c{cst[2], cst[3]};
  const R inv_n = R(1) / R(g.n);
  for (int idx = tid; idx < T * L; idx += nthr) {
    const int col = idx % T, n = idx / T;
    const int kx = col0 + col;
    C2<R>* const mrow = sm + n * NCOL + col;
    const int qs = (n >> 1) & 1;
    auto M = [&](int q) -> C2<R>& { return mrow[(q ^ qs) * T]; };
    if (kx >= g.mx) {
#pragma unroll
      for (int q = 0; q < 6; ++q) M(q) = mk<R>(0, 0);
      continue;
    }
    C2<R> rv[3], pv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      rv[c] = M(c);
      pv[c] = M(3 + c);
    }
    R xi[3];
    xi[0] = dk0 * R(signed_k(kx, g.nx));
    xi[1] = dk1 * R(signed_k(ky, g.ny));
    xi[2] = dk2 * R(signed_k(n, L));
    const R qq = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
    const bool nz = qq != R(0);
    C2<R> zv[3], e[6];
    if (a.precond && nz) {                         // z = G0 r, formed here rather than stored
      cd_g0<R>(rv, xi, qq, g0c, zv);
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) zv[c] = a.precond ? mk<R>(0, 0) : rv[c];
    }
    const long long gi = n * zs + rowbase + kx;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      a.u[vo + c * g.cs + gi] = pre[(c * L + n) * T + col] + scale(pv[c], alpha);   // u1 += alpha p
      pv[c] = zv[c] + scale(pv[c], beta);
      a.p[vo + c * g.cs + gi] = pv[c];
    }
    cd_symgrad<R>(pv, xi, inv_n, e);
#pragma unroll
    for (int q = 0; q < 6; ++q) M(q) = nz ? e[q] : mk<R>(0, 0);
  }
  __syncthreads();
  // ---- inverse z transform (four-step rule, decimation-in-frequency order) to the work spectrum
  for (int task = tid; task < TASKS; task += nthr) {
    const int c = task % NCOL, j = task / NCOL;
    if (j >= R1) continue;
    C2<R> y[R2];
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) y[k2] = sm[(j + R1 * k2) * NCOL + cd_slot(j + R1 * k2, c)];
    Dft<R, R2, +1>::run(y);
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) sm[(j + R1 * n2) * NCOL + cd_slot(j + R1 * n2, c)] = y[n2];
  }
  __syncthreads();
  for (int task = tid; task < TASKS; task += nthr) {
    const int c = task % NCOL, j = task / NCOL;
    if (j >= R2) continue;
    C2<R> x[R1];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) x[k1] = sm[(j * R1 + k1) * NCOL + cd_slot(j * R1 + k1, c)];
    twiddle_then_dft<R, L, R1, +1>(x, j, a.tw);
    if (col0 + (c % T) < g.mx) {
      C2<R>* gcol = column(c);
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) gcol[(R2 * n1 + j) * zs] = x[n1];
    }
  }
}

template <typename R, int L>
static cudaError_t zcd_L(const CdArgs<R>& a, bool fwd, int batch, cudaStream_t st) {
  const dim3 grid((a.g.mx + kCdT - 1) / kCdT, a.g.ny, batch);
  const size_t smem = sizeof(C2<R>) * (size_t)L * (kCdNcol + 3 * kCdT);   // + the p (forward) or u tile
  auto k = fwd ? k_zcd<R, L, true> : k_zcd<R, L, false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, ZCfg<L>::BLOCK, smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_zcd(const CdArgs<R>& a, bool fwd, int batch, IterState* ist, const Member* mem, int maxdim,
                       cudaStream_t st) {
  cudaError_t e = cudaErrorInvalidValue;
  switch (a.g.nz) {
#define BFCS_ZCD(L) case L: e = zcd_L<R, L>(a, fwd, batch, st); break;
    BFCS_ZCD(4) BFCS_ZCD(6) BFCS_ZCD(8) BFCS_ZCD(12) BFCS_ZCD(16) BFCS_ZCD(24) BFCS_ZCD(32) BFCS_ZCD(48)
    BFCS_ZCD(64) BFCS_ZCD(96) BFCS_ZCD(128) BFCS_ZCD(192) BFCS_ZCD(256)
#undef BFCS_ZCD
    default: break;
  }
  if (e != cudaSuccess || !fwd) return e;
  // alpha from <p, q>: one partial pair per tile
  const int nparts = ((a.g.mx + kCdT - 1) / kCdT) * a.g.ny;
  k_cd_scalar<<<batch, kCdThreads, 0, st>>>(a.part, nparts, a.cd, a.skip, ist, mem, a.lam0, a.mu0, (double)a.g.n,
                                            maxdim, CdMode::PQ);
  count_launches(1);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_cd_vec(const CdArgs<R>& a, int mode, int batch, IterState* ist, const Member* mem, int maxdim,
                          cudaStream_t st) {
  k_cd_vec<R><<<dim3(kCdParts, batch), kCdThreads, 0, st>>>(a, mode);
  count_launches(1);
  if (mode == CdMode::FINAL || mode == CdMode::FINAL_U) return cudaGetLastError();
  k_cd_scalar<<<batch, kCdThreads, 0, st>>>(a.part, kCdParts, a.cd, a.skip, ist, mem, a.lam0, a.mu0,
                                            (double)a.g.n, maxdim, mode);
  count_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_cd_vec<BFCS_R>(const CdArgs<BFCS_R>&, int, int, IterState*, const Member*, int,
                                           cudaStream_t);
template cudaError_t launch_zcd<BFCS_R>(const CdArgs<BFCS_R>&, bool, int, IterState*, const Member*, int,
                                        cudaStream_t);

}  // namespace bfcs
