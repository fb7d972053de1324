// Fused z pass of a sweep: forward FFT along z of the six polarization
// components, the Green-operator apply of the modified Lippmann-Schwinger
// equation in Fourier space (Eqs. 5.4, 5.9 with U0 of Eqs. 2.16-2.18 and the
// reference strain of Eqs. 2.8-2.9), the equilibrium residual partial sums
// (Eq. 5.11) and the inverse FFT along z, on one tile held in shared memory.
//
// Per mode k with xi != 0, using d = tau_hat . xi:
//   w = d - i b_hat,  v = G0(xi) w,  G0 = [I - c xi xi/|xi|^2] / (mu0 |xi|^2),
//   c = (lam0 + mu0)/(lam0 + 2 mu0),
//   eps_hat^{s+1} = -sym(xi (x) v)   (= U0 tau_hat + sym(i xi (x) G0 b_hat))
// because U0 tau = -sym(xi (x) G0 (tau xi)) is the factored form of Eq. 2.16.
// The residual numerator of eps^s is |i xi . sigma_hat + b_hat| = |d^s - d^{s-1}|,
// since eps^s = -Gamma0 tau^{s-1} + eps^{b(0)} and xi.C0.Gamma0 tau = xi.tau.
// The displacement consistent with eps^{s+1} is u_hat = i v (Eq. 2.9-2.10).
// Modes with xi = 0: eps_hat = N E at k = 0 (prescribed mean strain), else 0.
#include "kernels.h"

#include <algorithm>
#include <cstdlib>

#ifndef BFCS_R
#define BFCS_R float
#endif

namespace bfcs {

constexpr int kGreenT = 4;   // kx columns per block; 6 components -> 24 line columns

template <int L> struct GCfg {
  static constexpr int NCOL = 6 * kGreenT;
  static constexpr int THREADS = NCOL * LineInfo<L>::RMAX;
  // block size of the z pass: whole warps (the full-mask shuffles of the residual
  // reduction need them); threads past THREADS take no FFT task
  static constexpr int BLOCK = (THREADS + 31) / 32 * 32;
};

// Shared-memory slot of line-column c in tile row `row`: rows with bit 1 set
// swap neighbouring components (c ^ 4 with T = 4 columns per component).  Each
// row keeps the same set of slots for every aligned group of 8 columns, so the
// FFT exchanges (32 consecutive columns over one or two rows) stay
// conflict-free, and the Green phase (8 rows x 4 columns of one component per
// warp) covers all 16 eight-byte bank pairs twice instead of 8 of them 4 times.
static_assert(kGreenT == 4 && (6 * kGreenT) % 8 == 0, "the swizzle flips one component bit");
__device__ __forceinline__ int gslot(int row, int c) { return c ^ (((row >> 1) & 1) << 2); }

template <typename R>
__device__ __forceinline__ void g0_apply(const C2<R> g[3], const R xi[3], R q, R inv_mu0, R c,
                                         C2<R> v[3]) {
  const C2<R> xg = scale(g[0], xi[0]) + scale(g[1], xi[1]) + scale(g[2], xi[2]);
  const R iq = recip(q);
  const R a = iq * inv_mu0;
  const R b = c * iq;
#pragma unroll
  for (int i = 0; i < 3; ++i) v[i] = scale(g[i] - scale(xg, b * xi[i]), a);
}

// Green operators on one tile held in shared memory (rows n = z frequency,
// columns c = component * T + kx offset, slots per gslot): every mode of the
// tile is replaced by eps_hat^{s+1} / N (GM_SWEEP / GM_INIT) or u_hat / N
// (GM_FINAL); d = tau_hat . xi is written to dprev (sweep / init); returns this
// thread's share of the residual numerator sum.
template <typename R, int L>
__device__ __forceinline__ R green_tile(const GArgs<R>& a, C2<R>* s, const C2<R>* pre, int col0, int ky, int mode,
                                        C2<R>* dprev, IterState* stm, const R* Em, bool rd = true,
                                        bool wr = true) {
  // GM_SWEEP: rd = this sweep forms the residual (d_prev staged), wr = it stores d
  const bool rd_d = mode == GM_FINAL || (mode == GM_SWEEP && rd);
  const bool wr_d = mode == GM_INIT || (mode == GM_SWEEP && wr);
  constexpr int T = kGreenT;
  constexpr int NCOL = GCfg<L>::NCOL;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int nx = a.g.nx, ny = a.g.ny, mx = a.g.mx, p = a.g.p;
  const long long cs = a.g.cs;
  const long long zs = (long long)ny * p;
  const long long rowbase = (long long)ky * p;
  const R two_pi = R(6.283185307179586);
  const R fx = two_pi / R(nx), fy = two_pi / R(ny), fz = two_pi / R(L);
  const R mu0 = a.mu0, c0 = (a.lam0 + a.mu0) / (a.lam0 + R(2) * a.mu0);
  const R inv_n = a.inv_n;
  R acc = R(0);
  for (int idx = tid; idx < T * L; idx += nthr) {
    const int col = idx % T, n = idx / T;
    const int kx = col0 + col;
    C2<R>* const m = s + n * NCOL + col;
    const int qs = (n >> 1) & 1;                    // component q sits at m[(q ^ qs) * T] (gslot)
    auto M = [&](int q) -> C2<R>& { return m[(q ^ qs) * T]; };
    const C2<R>* pm = pre + n * T + col;            // array r at pm[r * L * T]
    if (kx >= mx) {
#pragma unroll
      for (int q = 0; q < 6; ++q) M(q) = mk<R>(0, 0);
      continue;
    }
    const long long gi = n * zs + rowbase + kx;     // index in a 3-component spectrum
    R xi[3];
    xi[0] = fx * R(signed_k(kx, nx));
    xi[1] = fy * R(signed_k(ky, ny));
    xi[2] = fz * R(signed_k(n, L));
    const R qq = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
    const R wgt = (kx == 0 || 2 * kx == nx) ? R(1) : R(2);

    if (qq == R(0)) {
      const bool k0 = (kx == 0 && ky == 0 && n == 0);
      if (k0 && mode != GM_INIT && mode != GM_APPLY) {
#pragma unroll
        for (int q = 0; q < 6; ++q) stm->tau0[q] = (double)M(q).x;
      }
      if (wr_d) {
        dprev[gi] = mk<R>(0, 0); dprev[cs + gi] = mk<R>(0, 0); dprev[2 * cs + gi] = mk<R>(0, 0);
      }
#pragma unroll
      for (int q = 0; q < 6; ++q)
        M(q) = (mode != GM_FINAL && mode != GM_APPLY && k0) ? mk<R>(Em[q], R(0)) : mk<R>(0, 0);
      continue;
    }
    const bool load = mode != GM_APPLY;
    C2<R> bh0 = mk<R>(0, 0), bh1 = mk<R>(0, 0), bh2 = mk<R>(0, 0);
    C2<R> dp[3] = {mk<R>(0, 0), mk<R>(0, 0), mk<R>(0, 0)};
    if (load) { bh0 = pm[0]; bh1 = pm[L * T]; bh2 = pm[2 * L * T]; }
    if (rd_d) { dp[0] = pm[3 * L * T]; dp[1] = pm[4 * L * T]; dp[2] = pm[5 * L * T]; }

    C2<R> d[3] = {mk<R>(0, 0), mk<R>(0, 0), mk<R>(0, 0)};
    if (mode != GM_INIT) {
      // d_i = tau_hat_ij xi_j (xx yy zz yz xz xy)
      const C2<R> t0 = M(0), t1 = M(1), t2 = M(2), t3 = M(3), t4 = M(4), t5 = M(5);
      d[0] = scale(t0, xi[0]) + scale(t5, xi[1]) + scale(t4, xi[2]);
      d[1] = scale(t5, xi[0]) + scale(t1, xi[1]) + scale(t3, xi[2]);
      d[2] = scale(t4, xi[0]) + scale(t3, xi[1]) + scale(t2, xi[2]);
      R r2 = R(0);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const R ex = d[i].x - dp[i].x, ey = d[i].y - dp[i].y;
        r2 += ex * ex + ey * ey;
      }
      if (rd_d) acc += wgt * r2;
      if (mode == GM_FINAL) { d[0] = dp[0]; d[1] = dp[1]; d[2] = dp[2]; }
    }
    if (wr_d) {
      dprev[gi] = d[0]; dprev[cs + gi] = d[1]; dprev[2 * cs + gi] = d[2];
    }
    // w = d - i b_hat
    C2<R> w[3];
    w[0] = mk<R>(d[0].x + bh0.y, d[0].y - bh0.x);
    w[1] = mk<R>(d[1].x + bh1.y, d[1].y - bh1.x);
    w[2] = mk<R>(d[2].x + bh2.y, d[2].y - bh2.x);
    C2<R> v[3];
    g0_apply<R>(w, xi, qq, recip(mu0), c0, v);
    if (mode == GM_FINAL) {
      // u_hat = i v, scaled for the unnormalised inverse transforms
#pragma unroll
      for (int i = 0; i < 3; ++i) M(i) = mk<R>(-v[i].y * inv_n, v[i].x * inv_n);
#pragma unroll
      for (int q = 3; q < 6; ++q) M(q) = mk<R>(0, 0);
    } else {
      const R h = R(-0.5) * inv_n;
      M(0) = scale(v[0], -xi[0] * inv_n);
      M(1) = scale(v[1], -xi[1] * inv_n);
      M(2) = scale(v[2], -xi[2] * inv_n);
      M(3) = scale(scale(v[2], xi[1]) + scale(v[1], xi[2]), h);
      M(4) = scale(scale(v[2], xi[0]) + scale(v[0], xi[2]), h);
      M(5) = scale(scale(v[1], xi[0]) + scale(v[0], xi[1]), h);
    }
  }

  return acc;
}

// Each FFT stage is a loop over its (line column c, row group j) tasks; with the
// block of GCfg<L>::BLOCK threads every thread takes at most one.  The b_hat and
// d_prev tiles are staged in shared memory while the forward transform runs.
template <typename R, int L>
__global__ void __launch_bounds__(GCfg<L>::BLOCK, sizeof(R) == 4 ? 2 : 1) k_zgreen(GArgs<R> a) {
  const int mbr = blockIdx.z;
  if (a.skip_done && a.st[mbr].done) return;     // a member that has converged skips
  // this member's buffers and mean strain
  C2<R>* const spec = a.spec + mbr * a.spec_ms;
  const C2<R>* const bhat = a.bhat + mbr * a.b_ms;
  C2<R>* const dprev = a.dprev + mbr * a.d_ms;
  ResidSlot* const part = a.part + mbr * a.part_ms;
  IterState* const stm = a.st + mbr;
  const R* const Em = a.use_me ? a.mE[mbr] : a.E;
  constexpr int T = kGreenT;
  constexpr int NCOL = GCfg<L>::NCOL;
  constexpr int R1 = LineInfo<L>::R1, R2 = LineInfo<L>::R2;
  constexpr int TASKS = NCOL * LineInfo<L>::RMAX;   // (column, row group) tasks of a stage
  extern __shared__ unsigned char smem_raw[];
  C2<R>* s = reinterpret_cast<C2<R>*>(smem_raw);      // [n][c], c = component * T + column
  C2<R>* pre = s + L * NCOL;                          // [6][n][col]: b_hat 0..2, d_prev 3..5
  __shared__ double red[32];

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int ny = a.g.ny, mx = a.g.mx, p = a.g.p;
  const long long cs = a.g.cs;
  const int ky = blockIdx.y;
  const int col0 = blockIdx.x * T;
  const long long zs = (long long)ny * p;          // z stride
  const long long rowbase = (long long)ky * p;
  const int mode = a.mode;
  // sparse residual evaluation (GM_SWEEP): read d_prev and form the residual only
  // on the member's next check sweep; store d on that sweep, the one before it
  // and the last sweep of the call (the final step reads it)
  bool rd = true, wr = true;
  if (mode == GM_SWEEP && a.sparse) {
    const int sw = stm->iters, nc = stm->next_check;
    rd = sw == nc;
    wr = rd || sw + 1 == nc || sw + 1 >= a.maxit;
  }
  // element z of line column c at column(c)[z * zs]
  auto column = [&](int c) { const int q = c / T; return spec + q * cs + rowbase + col0 + (c - q * T); };

  // ---- start the copies of the b_hat and d_prev tiles; they land during the FFT
  {
    constexpr int PER = 16 / sizeof(C2<R>);          // complex values per 16-byte copy
    constexpr int CPR = T / PER;                     // copies per row of the tile
    const int narr = mode == GM_INIT ? 3 : mode == GM_APPLY ? 0 : (rd ? 6 : 3);
    for (int idx = tid; idx < narr * L * CPR; idx += nthr) {
      const int part = idx % CPR, n = (idx / CPR) % L, arr = idx / (CPR * L);
      const C2<R>* src = (arr < 3 ? bhat + arr * cs : dprev + (arr - 3) * cs) + n * zs + rowbase +
                         col0 + part * PER;
      cp_async16(pre + (arr * L + n) * T + part * PER, src);
    }
    cp_async_commit();
  }

  // ---- forward transform along z: stage 1 straight from global
  if (mode != GM_INIT) {
    for (int task = tid; task < TASKS; task += nthr) {
      const int c = task % NCOL, j = task / NCOL;
      if (j >= R2) continue;
      const bool cvalid = col0 + (c % T) < mx;
      const C2<R>* gcol = column(c);
      C2<R> x[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) x[n1] = cvalid ? gcol[(R2 * n1 + j) * zs] : mk<R>(0, 0);
      stage1<R, L, -1>(x, j, a.tw);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) s[(j * R1 + k1) * NCOL + gslot(j * R1 + k1, c)] = x[k1];
    }
    __syncthreads();
    // stage 2 reads and writes the same slots (rows j + R1 m, m < R2, of column c):
    // no other task touches them, so no barrier separates the read and the write
    for (int task = tid; task < TASKS; task += nthr) {
      const int c = task % NCOL, j = task / NCOL;
      if (j >= R1) continue;
      C2<R> y[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) y[n2] = s[(n2 * R1 + j) * NCOL + gslot(n2 * R1 + j, c)];
      stage2<R, L, -1>(y);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) s[(j + R1 * k2) * NCOL + gslot(j + R1 * k2, c)] = y[k2];
    }
    __syncthreads();
  }

  cp_async_wait_all();
  __syncthreads();

  // ---- Green operators per mode
  R acc = green_tile<R, L>(a, s, pre, col0, ky, mode, dprev, stm, Em, rd, wr);

  // ---- residual partial of this block in FP64 (fixed order: deterministic)
  const bool resid = (mode == GM_SWEEP && rd) || mode == GM_FINAL;
  if (resid) {
    double accd = (double)acc;
    for (int off = 16; off > 0; off >>= 1) accd += __shfl_down_sync(0xffffffffu, accd, off);
    if ((tid & 31) == 0) red[tid >> 5] = accd;
  }
  __syncthreads();
  if (resid && tid == 0) {
    double t = 0.0;
    for (int w = 0; w < (nthr + 31) / 32; ++w) t += red[w];
    part[blockIdx.y * gridDim.x + blockIdx.x].num = t;
  }

  // ---- inverse transform along z in the other order of the four-step rule
  // (k = k1 + R1 k2, z = R2 n1 + n2): an R2-point step over the rows k1 + R1 m of
  // each column, written back to the same rows (no other task touches them), then
  // the twiddled R1-point step over the rows n2 R1 + k1, straight to global memory
  for (int task = tid; task < TASKS; task += nthr) {
    const int c = task % NCOL, j = task / NCOL;
    if (j >= R1) continue;
    C2<R> y[R2];
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) y[k2] = s[(j + R1 * k2) * NCOL + gslot(j + R1 * k2, c)];
    Dft<R, R2, +1>::run(y);
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) s[(j + R1 * n2) * NCOL + gslot(j + R1 * n2, c)] = y[n2];
  }
  __syncthreads();
  for (int task = tid; task < TASKS; task += nthr) {
    const int c = task % NCOL, j = task / NCOL;
    if (j >= R2) continue;
    const bool keep = (mode != GM_FINAL || c / T < 3) && col0 + (c % T) < mx;
    C2<R> x[R1];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) x[k1] = s[(j * R1 + k1) * NCOL + gslot(j * R1 + k1, c)];
    twiddle_then_dft<R, L, R1, +1>(x, j, a.tw);
    if (keep) {
      C2<R>* gcol = column(c);
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) gcol[(R2 * n1 + j) * zs] = x[n1];
    }
  }
}

// Persistent, double-buffered form of the sweep's z pass (GM_SWEEP, FP32).
// One block per SM walks the tiles t = blockIdx.x, + gridDim.x, ... of all
// members (tile = member, ky, group of 4 kx columns; converged members are
// skipped).  While the block transforms tile t in one shared-memory buffer,
// cp.async streams tile t + gridDim.x (six spectral components, b_hat, d_prev)
// into the other, so HBM keeps working during the FFT and Green arithmetic.
// The tile sits in shared memory in the same swizzled layout as k_zgreen's,
// and the stages run in place.  Residual partials: one slot per (member,
// block), at part[m * gridDim.x + blockIdx.x] (gridDim.x <= tiles per member,
// so every block visits every member it has to report).
template <int L> struct GPCfg {
  static constexpr int TILE = L * GCfg<L>::NCOL;   // complex values of the 6-component tile
  static constexpr int PRE = 6 * L * kGreenT;      // b_hat (3) and d_prev (3) tiles
  static constexpr size_t SMEM = 2 * (size_t)(TILE + PRE) * sizeof(C2<float>);
};

template <int L>
__global__ void __launch_bounds__(GCfg<L>::THREADS, 1)
    k_zgreen_p(GArgs<float> a, int tiles_x, int tiles_pm, int total) {
  using R = float;
  constexpr int T = kGreenT;
  constexpr int NCOL = GCfg<L>::NCOL;
  constexpr int R1 = LineInfo<L>::R1, R2 = LineInfo<L>::R2;
  constexpr int TILE = GPCfg<L>::TILE, PRE = GPCfg<L>::PRE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<R>* const base = reinterpret_cast<C2<R>*>(smem_raw);
  __shared__ double red[32];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int G = gridDim.x;
  const int ny = a.g.ny, p = a.g.p;
  const long long cs = a.g.cs;
  const long long zs = (long long)ny * p;
  const int c = tid % NCOL, j = tid / NCOL;
  const int ccomp = c / T, ccol = c - ccomp * T;

  auto skip = [&](int t) { return a.st[t / tiles_pm].done != 0; };
  auto next = [&](int t) {
    t += G;
    while (t < total && skip(t)) t += G;
    return t;
  };
  // copies of tile t into buffer b: 6 spectral components, b_hat, d_prev (16 bytes = 2 kx each)
  auto issue = [&](int t, int b) {
    C2<R>* S = base + b * (TILE + PRE);
    C2<R>* P = S + TILE;
    const int m = t / tiles_pm, r = t - m * tiles_pm;
    const int ky = r / tiles_x, col0 = (r - ky * tiles_x) * T;
    const long long rb = (long long)ky * p + col0;
    const C2<R>* spec = a.spec + m * a.spec_ms + rb;
    const C2<R>* bh = a.bhat + m * a.b_ms + rb;
    const C2<R>* dp = a.dprev + m * a.d_ms + rb;
    for (int idx = tid; idx < 12 * L * 2; idx += nthr) {
      const int half = idx & 1, n = (idx >> 1) % L, arr = idx / (2 * L);
      if (arr < 6) {
        cp_async16(S + n * NCOL + gslot(n, arr * T + 2 * half), spec + arr * cs + n * zs + 2 * half);
      } else {
        const int q = arr - 6;
        const C2<R>* src = (q < 3 ? bh + q * cs : dp + (q - 3) * cs) + n * zs + 2 * half;
        cp_async16(P + (q * L + n) * T + 2 * half, src);
      }
    }
  };
  auto flush = [&](int m, double accd) {
    for (int off = 16; off > 0; off >>= 1) accd += __shfl_down_sync(0xffffffffu, accd, off);
    if ((tid & 31) == 0) red[tid >> 5] = accd;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < (nthr + 31) / 32; ++w) t += red[w];
      a.part[(long long)m * G + blockIdx.x].num = t;
    }
    __syncthreads();
  };

  int t = blockIdx.x;
  while (t < total && skip(t)) t += G;
  if (t < total) issue(t, 0);
  cp_async_commit();
  int cur = 0, m_acc = -1;
  double acc = 0.0;          // this thread's share of the member's residual numerator
  while (t < total) {
    const int tn = next(t);
    if (tn < total) issue(tn, cur ^ 1);
    cp_async_commit();
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // tile t has landed
    __syncthreads();
    const int m = t / tiles_pm, r = t - m * tiles_pm;
    const int ky = r / tiles_x, col0 = (r - ky * tiles_x) * T;
    if (m != m_acc) {
      if (m_acc >= 0) flush(m_acc, acc);
      m_acc = m;
      acc = 0.0;
    }
    C2<R>* s = base + cur * (TILE + PRE);
    const C2<R>* pre = s + TILE;
    C2<R>* const dprev = a.dprev + m * a.d_ms;
    IterState* const stm = a.st + m;
    const R* const Em = a.use_me ? a.mE[m] : a.E;
    // forward z transform, in place in the tile
    {
      C2<R> x[R1];
      if (j < R2) {
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) x[n1] = s[(R2 * n1 + j) * NCOL + gslot(R2 * n1 + j, c)];
        stage1<R, L, -1>(x, j, a.tw);
      }
      __syncthreads();
      if (j < R2) {
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) s[(j * R1 + k1) * NCOL + gslot(j * R1 + k1, c)] = x[k1];
      }
    }
    __syncthreads();
    {
      C2<R> y[R2];
      if (j < R1) {
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) y[n2] = s[(n2 * R1 + j) * NCOL + gslot(n2 * R1 + j, c)];
        stage2<R, L, -1>(y);
      }
      __syncthreads();
      if (j < R1) {
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) s[(j + R1 * k2) * NCOL + gslot(j + R1 * k2, c)] = y[k2];
      }
    }
    __syncthreads();
    acc += (double)green_tile<R, L>(a, s, pre, col0, ky, GM_SWEEP, dprev, stm, Em);
    __syncthreads();
    // inverse z transform in the order of the one-tile-per-block form (the same
    // arithmetic, so the two forms give identical fields): in-place R2-point step,
    // then the twiddled R1-point step straight to global memory
    if (j < R1) {
      C2<R> y[R2];
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) y[k2] = s[(j + R1 * k2) * NCOL + gslot(j + R1 * k2, c)];
      Dft<R, R2, +1>::run(y);
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) s[(j + R1 * n2) * NCOL + gslot(j + R1 * n2, c)] = y[n2];
    }
    __syncthreads();
    if (j < R2) {
      C2<R> x[R1];
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) x[k1] = s[(j * R1 + k1) * NCOL + gslot(j * R1 + k1, c)];
      twiddle_then_dft<R, L, R1, +1>(x, j, a.tw);
      const int kx = col0 + ccol;
      if (kx < a.g.mx) {
        C2<R>* gcol = a.spec + m * a.spec_ms + ccomp * cs + (long long)ky * p + kx;
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) gcol[(R2 * n1 + j) * zs] = x[n1];
      }
    }
    __syncthreads();   // buffer `cur` is free for the prefetch after next
    cur ^= 1;
    t = tn;
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  if (m_acc >= 0) flush(m_acc, acc);
}

// SM count of the current device (cached)
static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || n < 1)
      n = 1;
  }
  return n;
}

// The persistent form runs only with BFCS_ZGREEN_PERSISTENT=1: at 256^3 it measured
// 0.52 ms per launch against 0.49 ms for the one-tile-per-block form (two
// co-resident blocks of 12 warps overlap one tile's loads with the other's
// arithmetic better than one block of 12 warps with a prefetched second tile).
static bool persistent_green_enabled() {
  const char* e = std::getenv("BFCS_ZGREEN_PERSISTENT");
  return e != nullptr && std::atoi(e) == 1;
}

// Blocks of the persistent z pass for grid g (0: the persistent form does not apply)
template <typename R>
int green_persistent_blocks(const Geo& g) {
  if (sizeof(R) != 4 || !persistent_green_enabled()) return 0;
  const int tiles_pm = ((g.mx + kGreenT - 1) / kGreenT) * g.ny;
  if (tiles_pm < 2 * sm_count()) return 0;
  return std::min(sm_count(), tiles_pm);
}

// Defect of an approximate strain (precision ladder): R_hat = i xi . sigma_hat +
// b_hat on modes with xi != 0 (Eq. 2.1 in Fourier form with Eq. 4.8), the load
// of the correction problem.  Grid-stride over the stored modes.
template <typename R>
__global__ void k_defect(DArgs<R> a) {
  __shared__ double red[32];
  const Geo g = a.g;
  {
    const int j = blockIdx.y, m = a.idx[j];
    a.spec += j * a.spec_ms;
    a.part += j * gridDim.x;
    a.bhat += m * a.b_ms;
    a.out32 += m * a.o_ms;
    a.st += m;
  }
  const long long modes = (long long)g.nz * g.ny * g.mx;
  const R two_pi = R(6.283185307179586);
  const R dk0 = two_pi / R(g.nx), dk1 = two_pi / R(g.ny), dk2 = two_pi / R(g.nz);
  double acc = 0.0;
  // 32-bit index arithmetic: a member's spectrum has at most 256 * 256 * 129 modes
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (int)modes; i += gridDim.x * blockDim.x) {
    const int kx = i % g.mx;
    const int r = i / g.mx;
    const int ky = r % g.ny, kz = r / g.ny;
    const long long gi = (long long)r * g.p + kx;
    const C2<R>* sp = a.spec + gi;
    const R xi0 = dk0 * R(signed_k(kx, g.nx));
    const R xi1 = dk1 * R(signed_k(ky, g.ny));
    const R xi2 = dk2 * R(signed_k(kz, g.nz));
    const C2<R> s0 = sp[0], s1 = sp[g.cs], s2 = sp[2 * g.cs], s3 = sp[3 * g.cs], s4 = sp[4 * g.cs],
                s5 = sp[5 * g.cs];
    if (kx == 0 && ky == 0 && kz == 0) {
      a.st->tau0[0] = (double)s0.x; a.st->tau0[1] = (double)s1.x; a.st->tau0[2] = (double)s2.x;
      a.st->tau0[3] = (double)s3.x; a.st->tau0[4] = (double)s4.x; a.st->tau0[5] = (double)s5.x;
    }
    C2<R> d[3];
    if (xi0 == R(0) && xi1 == R(0) && xi2 == R(0)) {
      d[0] = d[1] = d[2] = mk<R>(0, 0);
    } else {
      // sigma_hat . xi (xx yy zz yz xz xy), then i (.) + b_hat
      const C2<R> v0 = scale(s0, xi0) + scale(s5, xi1) + scale(s4, xi2);
      const C2<R> v1 = scale(s5, xi0) + scale(s1, xi1) + scale(s3, xi2);
      const C2<R> v2 = scale(s4, xi0) + scale(s3, xi1) + scale(s2, xi2);
      const C2<R> b0 = a.bhat[gi], b1 = a.bhat[g.cs + gi], b2 = a.bhat[2 * g.cs + gi];
      d[0] = mk<R>(-v0.y + b0.x, v0.x + b0.y);
      d[1] = mk<R>(-v1.y + b1.x, v1.x + b1.y);
      d[2] = mk<R>(-v2.y + b2.x, v2.x + b2.y);
      const double w = (kx == 0 || 2 * kx == g.nx) ? 1.0 : 2.0;
      double t = 0.0;
      for (int c = 0; c < 3; ++c) t += norm2<R>(d[c]);
      acc += w * t;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) a.out32[c * g.cs + gi] = mk<float>((float)d[c].x, (float)d[c].y);
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
    a.part[blockIdx.x].num = t;
  }
}

template <typename R>
cudaError_t launch_defect(const DArgs<R>& a, int blocks, int batch, cudaStream_t st) {
  k_defect<R><<<dim3(blocks, batch), 256, 0, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

template <typename R>
__global__ void k_symgrad(C2<R>* spec, long long ms, Geo g, R inv_n, const Member* mem) {
  spec += blockIdx.y * ms;
  const double* E = mem[blockIdx.y].E;
  const R E0 = (R)E[0], E1 = (R)E[1], E2 = (R)E[2], E3 = (R)E[3], E4 = (R)E[4], E5 = (R)E[5];
  const long long modes = (long long)g.nz * g.ny * g.mx;
  const R two_pi = R(6.283185307179586);
  const R dk0 = two_pi / R(g.nx), dk1 = two_pi / R(g.ny), dk2 = two_pi / R(g.nz);
  // 32-bit index arithmetic: a member's spectrum has at most 256 * 256 * 129 modes
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (int)modes; i += gridDim.x * blockDim.x) {
    const int kx = i % g.mx;
    const int r = i / g.mx;
    const int ky = r % g.ny, kz = r / g.ny;
    C2<R>* sp = spec + (long long)r * g.p + kx;
    const R x0 = dk0 * R(signed_k(kx, g.nx));
    const R x1 = dk1 * R(signed_k(ky, g.ny));
    const R x2 = dk2 * R(signed_k(kz, g.nz));
    const C2<R> u0 = sp[0], u1 = sp[g.cs], u2 = sp[2 * g.cs];
    C2<R> e[6];
    if (x0 == R(0) && x1 == R(0) && x2 == R(0)) {
      const bool k0 = kx == 0 && ky == 0 && kz == 0;
      e[0] = mk<R>(k0 ? E0 : R(0), 0); e[1] = mk<R>(k0 ? E1 : R(0), 0); e[2] = mk<R>(k0 ? E2 : R(0), 0);
      e[3] = mk<R>(k0 ? E3 : R(0), 0); e[4] = mk<R>(k0 ? E4 : R(0), 0); e[5] = mk<R>(k0 ? E5 : R(0), 0);
    } else {
      // eps_ij = (i/2)(xi_i u_j + xi_j u_i); i (a + ib) = (-b, a)
      const R h = R(0.5) * inv_n;
      auto ih = [&](C2<R> v, R f) { return mk<R>(-v.y * f, v.x * f); };
      e[0] = ih(scale(u0, x0), inv_n);
      e[1] = ih(scale(u1, x1), inv_n);
      e[2] = ih(scale(u2, x2), inv_n);
      e[3] = ih(scale(u2, x1) + scale(u1, x2), h);
      e[4] = ih(scale(u2, x0) + scale(u0, x2), h);
      e[5] = ih(scale(u1, x0) + scale(u0, x1), h);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) sp[c * g.cs] = e[c];
  }
}

template <typename R>
cudaError_t launch_symgrad(C2<R>* spec, long long ms, const Geo& g, const Member* mem, int batch, cudaStream_t st) {
  k_symgrad<R><<<dim3(4 * 152, batch), 256, 0, st>>>(spec, ms, g, R(1.0 / (double)g.n), mem);
  count_launches(1);
  return cudaGetLastError();
}


// ---- Green step on a dense half spectrum, for transforms made outside the fused
// passes (a library real-to-complex 3D FFT: rows of nx/2 + 1 modes, g.p = g.mx).
// Per mode with xi != 0: d = tau_hat . xi, w = d - i b_hat, v = G0(xi) w and
// eps_hat^{s+1} = -sym(xi (x) v), which is U0 tau_hat + eps_hat^{b(0)} (Eqs.
// 5.9, 2.16-2.18, 2.8-2.9) in the factored form of the fused pass; the k = 0
// mode takes N E (the DFT of the prescribed mean strain), the other modes with
// xi = 0 take 0.  The result is unnormalised (an inverse transform that
// divides by N follows).  With dprev, the residual numerator of Eq. 5.11
// (reading R4) accumulates w_kx |d - d_prev|^2 per block into part[blockIdx.x]
// and d is stored for the next sweep.
template <typename R> struct E6 { R e[6]; };

template <typename R>
__global__ void k_green_dense(C2<R>* spec, const C2<R>* bhat, C2<R>* dprev, Geo g, R lam0, R mu0, E6<R> E,
                              ResidSlot* part) {
  __shared__ double red[32];
  const long long modes = (long long)g.nz * g.ny * g.mx;
  const R two_pi = R(6.283185307179586);
  const R dk0 = two_pi / R(g.nx), dk1 = two_pi / R(g.ny), dk2 = two_pi / R(g.nz);
  const R inv_mu0 = R(1) / mu0, c0 = (lam0 + mu0) / (lam0 + R(2) * mu0);
  const R nn = R((double)g.n);
  R acc = R(0);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < modes;
       i += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(i % g.mx);
    const long long r = i / g.mx;
    const int ky = (int)(r % g.ny), kz = (int)(r / g.ny);
    C2<R>* sp = spec + r * g.p + kx;
    const long long gi = r * g.p + kx;
    R xi[3];
    xi[0] = dk0 * R(signed_k(kx, g.nx));
    xi[1] = dk1 * R(signed_k(ky, g.ny));
    xi[2] = dk2 * R(signed_k(kz, g.nz));
    const R qq = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
    if (qq == R(0)) {
      const bool k0 = kx == 0 && ky == 0 && kz == 0;
#pragma unroll
      for (int c = 0; c < 6; ++c) sp[c * g.cs] = mk<R>(k0 ? nn * E.e[c] : R(0), R(0));
      if (dprev != nullptr) {
#pragma unroll
        for (int c = 0; c < 3; ++c) dprev[c * g.cs + gi] = mk<R>(0, 0);
      }
      continue;
    }
    const C2<R> t0 = sp[0], t1 = sp[g.cs], t2 = sp[2 * g.cs], t3 = sp[3 * g.cs], t4 = sp[4 * g.cs],
                t5 = sp[5 * g.cs];
    C2<R> d[3];
    d[0] = scale(t0, xi[0]) + scale(t5, xi[1]) + scale(t4, xi[2]);
    d[1] = scale(t5, xi[0]) + scale(t1, xi[1]) + scale(t3, xi[2]);
    d[2] = scale(t4, xi[0]) + scale(t3, xi[1]) + scale(t2, xi[2]);
    if (dprev != nullptr) {
      R r2 = R(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const C2<R> dp = dprev[c * g.cs + gi];
        const R ex = d[c].x - dp.x, ey = d[c].y - dp.y;
        r2 += ex * ex + ey * ey;
        dprev[c * g.cs + gi] = d[c];
      }
      acc += ((kx == 0 || 2 * kx == g.nx) ? R(1) : R(2)) * r2;
    }
    C2<R> w[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const C2<R> b = bhat[c * g.cs + gi];
      w[c] = mk<R>(d[c].x + b.y, d[c].y - b.x);
    }
    C2<R> v[3];
    g0_apply<R>(w, xi, qq, inv_mu0, c0, v);
    const R h = R(-0.5);
    sp[0] = scale(v[0], -xi[0]);
    sp[g.cs] = scale(v[1], -xi[1]);
    sp[2 * g.cs] = scale(v[2], -xi[2]);
    sp[3 * g.cs] = scale(scale(v[2], xi[1]) + scale(v[1], xi[2]), h);
    sp[4 * g.cs] = scale(scale(v[2], xi[0]) + scale(v[0], xi[2]), h);
    sp[5 * g.cs] = scale(scale(v[1], xi[0]) + scale(v[0], xi[1]), h);
  }
  if (part == nullptr) return;
  double accd = (double)acc;
  for (int off = 16; off > 0; off >>= 1) accd += __shfl_down_sync(0xffffffffu, accd, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = accd;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x + 31) / 32; ++k) t += red[k];
    part[blockIdx.x].num = t;
  }
}

// Displacement of the last iterate without the final pass: eps^S = -Gamma0
// tau^{S-1} + eps^{b(0)} has u_hat^S = i G0(xi) (d - i b_hat) / N with d = tau_hat^{S-1}
// . xi, the d_prev the last sweep stored (Eqs. 2.9-2.10; 0 on the modes with xi = 0),
// written into components 0..2 of the fully transformed spectrum.  Member
// blockIdx.y at spec_ms, b_ms and d_ms; grid-stride over the stored modes.
template <typename R>
__global__ void k_uhat(GArgs<R> a) {
  const int m = blockIdx.y;
  const Geo g = a.g;
  C2<R>* const spec = a.spec + m * a.spec_ms;
  const C2<R>* const bhat = a.bhat + m * a.b_ms;
  const C2<R>* const dprev = a.dprev + m * a.d_ms;
  const R two_pi = R(6.283185307179586);
  const R dk0 = two_pi / R(g.nx), dk1 = two_pi / R(g.ny), dk2 = two_pi / R(g.nz);
  const R inv_mu0 = recip(a.mu0), c0 = (a.lam0 + a.mu0) / (a.lam0 + R(2) * a.mu0);
  const long long modes = (long long)g.nz * g.ny * g.mx;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < modes;
       i += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(i % g.mx);
    const long long r = i / g.mx;
    const int ky = (int)(r % g.ny), kz = (int)(r / g.ny);
    const long long gi = r * g.p + kx;
    R xi[3];
    xi[0] = dk0 * R(signed_k(kx, g.nx));
    xi[1] = dk1 * R(signed_k(ky, g.ny));
    xi[2] = dk2 * R(signed_k(kz, g.nz));
    const R qq = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
    C2<R> u[3] = {mk<R>(0, 0), mk<R>(0, 0), mk<R>(0, 0)};
    if (qq != R(0)) {
      C2<R> w[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const C2<R> d = dprev[c * g.cs + gi], b = bhat[c * g.cs + gi];
        w[c] = mk<R>(d.x + b.y, d.y - b.x);     // d - i b_hat
      }
      C2<R> v[3];
      g0_apply<R>(w, xi, qq, inv_mu0, c0, v);
#pragma unroll
      for (int c = 0; c < 3; ++c) u[c] = mk<R>(-v[c].y * a.inv_n, v[c].x * a.inv_n);   // i v / N
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) spec[c * g.cs + gi] = u[c];
  }
}

template <typename R>
cudaError_t launch_uhat(const GArgs<R>& a, int batch, cudaStream_t st) {
  const long long modes = (long long)a.g.nz * a.g.ny * a.g.mx;
  const int blocks = (int)std::min<long long>((modes + 255) / 256, 4 * 152);
  k_uhat<R><<<dim3(blocks, batch), 256, 0, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

// sum of the block partials in block order (deterministic) into *out
static __global__ void k_sum_slots(const ResidSlot* part, int n, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i].num;
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x + 31) / 32; ++k) t += red[k];
    *out = t;
  }
}

template <typename R>
cudaError_t launch_green_dense(C2<R>* spec, const C2<R>* bhat, C2<R>* dprev, const Geo& g, double lam0,
                               double mu0, const double* E, ResidSlot* part, int nblocks, double* num_out,
                               cudaStream_t st) {
  E6<R> e{};
  for (int c = 0; c < 6; ++c) e.e[c] = (R)E[c];
  const bool resid = dprev != nullptr && num_out != nullptr;
  k_green_dense<R><<<nblocks, 256, 0, st>>>(spec, bhat, dprev, g, (R)lam0, (R)mu0, e, resid ? part : nullptr);
  count_launches(1);
  if (resid) {
    k_sum_slots<<<1, 1024, 0, st>>>(part, nblocks, num_out);
    count_launches(1);
  }
  return cudaGetLastError();
}

template <typename R>
int green_nparts(const Geo& g) {
  return ((g.mx + kGreenT - 1) / kGreenT) * g.ny;
}

template <typename R, int L>
static cudaError_t zgreen_L(const GArgs<R>& a, int batch, cudaStream_t st) {
  dim3 grid((a.g.mx + kGreenT - 1) / kGreenT, a.g.ny, batch);
  const size_t smem = sizeof(C2<R>) * (size_t)L * (GCfg<L>::NCOL + 6 * kGreenT);
  cudaError_t e = cudaFuncSetAttribute(k_zgreen<R, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_zgreen<R, L><<<grid, GCfg<L>::BLOCK, smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

template <int L>
static cudaError_t zgreen_p_L(const GArgs<float>& a, int batch, int blocks, cudaStream_t st) {
  const int tiles_x = (a.g.mx + kGreenT - 1) / kGreenT;
  const int tiles_pm = tiles_x * a.g.ny;
  const size_t smem = GPCfg<L>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(k_zgreen_p<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_zgreen_p<L><<<blocks, GCfg<L>::THREADS, smem, st>>>(a, tiles_x, tiles_pm, tiles_pm * batch);
  count_launches(1);
  return cudaGetLastError();
}

template <typename R>
int green_sweep_parts(const Geo& g) {
  const int pb = green_persistent_blocks<R>(g);
  return pb > 0 ? pb : green_nparts<R>(g);
}

template <typename R>
cudaError_t launch_zgreen_b(const GArgs<R>& a, int batch, cudaStream_t st) {
  if constexpr (sizeof(R) == 4) {
    const int pb = green_persistent_blocks<R>(a.g);
    if (pb > 0 && a.mode == GM_SWEEP && a.skip_done && !a.sparse && GPCfg<256>::SMEM <= 227 * 1024) {
      switch (a.g.nz) {
#define BFCS_GP(L) case L: return zgreen_p_L<L>(a, batch, pb, st);
        BFCS_GP(32) BFCS_GP(48) BFCS_GP(64) BFCS_GP(96) BFCS_GP(128) BFCS_GP(192) BFCS_GP(256)
#undef BFCS_GP
        default: break;
      }
    }
  }
  switch (a.g.nz) {
#define BFCS_G(L) case L: return zgreen_L<R, L>(a, batch, st);
    BFCS_G(4) BFCS_G(6) BFCS_G(8) BFCS_G(12) BFCS_G(16) BFCS_G(24) BFCS_G(32) BFCS_G(48)
    BFCS_G(64) BFCS_G(96) BFCS_G(128) BFCS_G(192) BFCS_G(256)
#undef BFCS_G
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
cudaError_t launch_zgreen(const GArgs<R>& a, cudaStream_t st) { return launch_zgreen_b<R>(a, 1, st); }

#ifndef BFCS_FF   // the float-float build carries only the ladder's defect kernels
template cudaError_t launch_zgreen<BFCS_R>(const GArgs<BFCS_R>&, cudaStream_t);
template cudaError_t launch_zgreen_b<BFCS_R>(const GArgs<BFCS_R>&, int, cudaStream_t);
template int green_nparts<BFCS_R>(const Geo&);
template int green_sweep_parts<BFCS_R>(const Geo&);
template cudaError_t launch_green_dense<BFCS_R>(C2<BFCS_R>*, const C2<BFCS_R>*, C2<BFCS_R>*, const Geo&, double,
                                                double, const double*, ResidSlot*, int, double*, cudaStream_t);
#endif
template cudaError_t launch_defect<BFCS_R>(const DArgs<BFCS_R>&, int, int, cudaStream_t);
template cudaError_t launch_symgrad<BFCS_R>(C2<BFCS_R>*, long long, const Geo&, const Member*, int, cudaStream_t);
template cudaError_t launch_uhat<BFCS_R>(const GArgs<BFCS_R>&, int, cudaStream_t);

}  // namespace bfcs
