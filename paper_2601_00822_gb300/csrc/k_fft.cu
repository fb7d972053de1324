// FFT passes of one sweep of the modified basic scheme (Algorithm 1):
//  * the x pass, where the inverse transform along x (Eq. 5.10), the
//    polarization tau = L1 eps (Eq. 5.7) and the forward transform along x
//    (Eq. 5.8) run back to back on lines held in shared memory, so the
//    real-space strain never goes to HBM between sweeps;
//  * the column passes along y and z on the half spectrum.
// Compiled once per precision with BFCS_R = float or double.
#include "kernels.h"

#ifndef BFCS_R
#define BFCS_R float
#endif

namespace bfcs {

// lines per block of the x pass: about 64 register-DFT tasks per pair column
template <int L> struct XCfg {
  static constexpr int RMAX = LineInfo<L>::RMAX;
  static constexpr int LPB = 64 / RMAX > 0 ? 64 / RMAX : 1;
  static constexpr int NCOL = 3 * LPB;        // up to 3 complex pair-columns per line
  static constexpr int THREADS = NCOL * RMAX;
};

template <typename R, int L>
__global__ void __launch_bounds__(XCfg<L>::THREADS) k_xpass(XArgs<R> a) {
  if (a.done != nullptr && *a.done) return;
  constexpr int LPB = XCfg<L>::LPB;
  constexpr int H = L / 2;
  extern __shared__ unsigned char smem_raw[];
  C2<R>* s = reinterpret_cast<C2<R>*>(smem_raw);

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int ncomp = a.ncomp;
  const int npair = (ncomp + 1) >> 1;
  const int ncol = LPB * npair;
  const long long lines = (long long)a.g.ny * a.g.nz;
  const long long line0 = (long long)blockIdx.x * LPB;
  const long long cs = a.g.cs, rn = a.g.n;
  const int p = a.g.p;
  const int mode = a.mode;

  // ---- 1. stage the lines in shared memory, column f = i * npair + q
  if (mode == XM_SWEEP || mode == XM_C2R || mode == XM_SWEEPSIG) {
    // Hermitian extension of the half spectrum into a full line for the pair
    // Z = A + i B; DC and Nyquist keep only their real parts (C2R rule).
    for (int idx = tid; idx < ncol * L; idx += nthr) {
      const int k = idx % L, f = idx / L;
      const int i = f / npair, q = f - i * npair;
      const long long line = line0 + i;
      C2<R> z = mk<R>(0, 0);
      if (line < lines) {
        const int kk = k <= H ? k : L - k;
        const C2<R>* row = a.spec_in + line * p + kk;
        C2<R> A = row[(2 * q) * cs];
        C2<R> B = (2 * q + 1 < ncomp) ? row[(2 * q + 1) * cs] : mk<R>(0, 0);
        if (kk == 0 || kk == H) { A.y = 0; B.y = 0; }
        if (k > H) { A.y = -A.y; B.y = -B.y; }
        z = mk<R>(A.x - B.y, A.y + B.x);
      }
      s[k * ncol + f] = z;
    }
    fft_cols<R, L, +1>(s, ncol, a.tw);
  } else {
    for (int idx = tid; idx < ncol * L; idx += nthr) {
      const int n = idx % L, f = idx / L;
      const int i = f / npair, q = f - i * npair;
      const long long line = line0 + i;
      C2<R> z = mk<R>(0, 0);
      if (line < lines) {
        const R* row = a.real_in + line * L + n;
        z.x = row[(2 * q) * rn];
        z.y = (2 * q + 1 < ncomp) ? row[(2 * q + 1) * rn] : R(0);
      }
      s[n * ncol + f] = z;
    }
    __syncthreads();
  }

  if (mode == XM_C2R) {
    for (int idx = tid; idx < ncol * L; idx += nthr) {
      const int n = idx % L, f = idx / L;
      const int i = f / npair, q = f - i * npair;
      const long long line = line0 + i;
      if (line >= lines) continue;
      const C2<R> z = s[n * ncol + f];
      R* row = a.real_out + line * L + n;
      row[(2 * q) * rn] = z.x;
      if (2 * q + 1 < ncomp) row[(2 * q + 1) * rn] = z.y;
    }
    return;
  }

  // ---- 2. polarization tau = (L(x) - L0) eps, isotropic phases (Eq. 5.7);
  //         in XM_REALSIG the full stress sigma = L(x) eps instead
  if (mode == XM_SWEEP || mode == XM_REALTAU || mode == XM_REALSIG || mode == XM_SWEEPSIG) {
    const bool full = mode == XM_REALSIG || mode == XM_SWEEPSIG;
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    for (int idx = tid; idx < LPB * L; idx += nthr) {
      const int n = idx % L, i = idx / L;
      const long long line = line0 + i;
      if (line >= lines) continue;
      const int y = (int)(line % ny), z = (int)(line / ny);
      C2<R>* c = s + n * ncol + i * 3;
      const C2<R> p0 = c[0], p1 = c[1], p2 = c[2];
      // eps: xx yy zz yz xz xy
      const R e0 = p0.x, e1 = p0.y, e2 = p1.x, e3 = p1.y, e4 = p2.x, e5 = p2.y;
      int xs = n - a.sx, ys = y - a.sy, zs = z - a.sz;
      xs %= nx; if (xs < 0) xs += nx;
      ys %= ny; if (ys < 0) ys += ny;
      zs %= nz; if (zs < 0) zs += nz;
      const int ph = a.phase[((long long)zs * ny + ys) * nx + xs];
      const R tr = e0 + e1 + e2;
      const long long vox = line * L + n;
      if (a.eps_out != nullptr) {
        R* o = a.eps_out + vox;
        o[0] = e0; o[rn] = e1; o[2 * rn] = e2; o[3 * rn] = e3; o[4 * rn] = e4; o[5 * rn] = e5;
      }
      if (a.sig_out != nullptr) {
        const R lt = a.tab.lam[ph] * tr, m2 = R(2) * a.tab.mu[ph];
        R* o = a.sig_out + vox;
        o[0] = lt + m2 * e0; o[rn] = lt + m2 * e1; o[2 * rn] = lt + m2 * e2;
        o[3 * rn] = m2 * e3; o[4 * rn] = m2 * e4; o[5 * rn] = m2 * e5;
      }
      const R lt = (full ? a.tab.lam[ph] : a.tab.lam1[ph]) * tr;
      const R m2 = R(2) * (full ? a.tab.mu[ph] : a.tab.mu1[ph]);
      c[0] = mk<R>(lt + m2 * e0, lt + m2 * e1);
      c[1] = mk<R>(lt + m2 * e2, m2 * e3);
      c[2] = mk<R>(m2 * e4, m2 * e5);
    }
  }

  // ---- 3. forward transform of the pair lines and split into two half spectra
  fft_cols<R, L, -1>(s, ncol, a.tw);
  for (int idx = tid; idx < ncol * (H + 1); idx += nthr) {
    const int k = idx % (H + 1), f = idx / (H + 1);
    const int i = f / npair, q = f - i * npair;
    const long long line = line0 + i;
    if (line >= lines) continue;
    const C2<R> Z = s[k * ncol + f];
    const C2<R> Zm = s[((L - k) % L) * ncol + f];
    C2<R>* row = a.spec_out + line * p + k;
    row[(2 * q) * cs] = mk<R>(R(0.5) * (Z.x + Zm.x), R(0.5) * (Z.y - Zm.y));
    if (2 * q + 1 < ncomp) row[(2 * q + 1) * cs] = mk<R>(R(0.5) * (Z.y + Zm.y), R(-0.5) * (Z.x - Zm.x));
  }
}

// Column FFT along y or z: each block owns T consecutive kx columns of one
// (other-axis, component) slab; loads are T-wide contiguous row segments.
constexpr int kColT = 16;

template <int L> struct CCfg {
  static constexpr int THREADS = kColT * LineInfo<L>::RMAX;
};

template <typename R, int L, int DIR>
__global__ void __launch_bounds__(CCfg<L>::THREADS) k_colpass(CArgs<R> a) {
  if (a.done != nullptr && *a.done) return;
  extern __shared__ unsigned char smem_raw[];
  C2<R>* s = reinterpret_cast<C2<R>*>(smem_raw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int mx = a.g.mx, p = a.g.p, ny = a.g.ny;
  const int other = a.axis == 1 ? a.g.nz : ny;
  const int c = blockIdx.y / other, o = blockIdx.y - c * other;
  const long long ls = a.axis == 1 ? (long long)p : (long long)ny * p;
  C2<R>* base = a.data + c * a.g.cs + (a.axis == 1 ? (long long)o * ny * p : (long long)o * p);
  const int col0 = blockIdx.x * kColT;
  for (int idx = tid; idx < kColT * L; idx += nthr) {
    const int col = idx % kColT, n = idx / kColT;
    const int kx = col0 + col;
    s[n * kColT + col] = kx < mx ? base[n * ls + kx] : mk<R>(0, 0);
  }
  fft_cols<R, L, DIR>(s, kColT, a.tw);
  for (int idx = tid; idx < kColT * L; idx += nthr) {
    const int col = idx % kColT, n = idx / kColT;
    const int kx = col0 + col;
    if (kx < mx) base[n * ls + kx] = s[n * kColT + col];
  }
}

// ---------------------------------------------------------------- dispatch
template <typename R, int L>
static cudaError_t xpass_L(const XArgs<R>& a, cudaStream_t st) {
  using C = XCfg<L>;
  const long long lines = (long long)a.g.ny * a.g.nz;
  const unsigned grid = (unsigned)((lines + C::LPB - 1) / C::LPB);
  const size_t smem = sizeof(C2<R>) * (size_t)L * C::NCOL;
  cudaError_t e = cudaFuncSetAttribute(k_xpass<R, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_xpass<R, L><<<grid, C::THREADS, smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_xpass(const XArgs<R>& a, cudaStream_t st) {
  switch (a.g.nx) {
#define BFCS_X(L) case L: return xpass_L<R, L>(a, st);
    BFCS_X(4) BFCS_X(6) BFCS_X(8) BFCS_X(12) BFCS_X(16) BFCS_X(24) BFCS_X(32) BFCS_X(48)
    BFCS_X(64) BFCS_X(96) BFCS_X(128) BFCS_X(192) BFCS_X(256)
#undef BFCS_X
    default: return cudaErrorInvalidValue;
  }
}

template <typename R, int L, int DIR>
static cudaError_t colpass_L(const CArgs<R>& a, cudaStream_t st) {
  const int other = a.axis == 1 ? a.g.nz : a.g.ny;
  dim3 grid((a.g.mx + kColT - 1) / kColT, other * a.ncomp);
  const size_t smem = sizeof(C2<R>) * (size_t)L * kColT;
  cudaError_t e = cudaFuncSetAttribute(k_colpass<R, L, DIR>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_colpass<R, L, DIR><<<grid, CCfg<L>::THREADS, smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_colpass(const CArgs<R>& a, int dir, cudaStream_t st) {
  const int n = a.axis == 1 ? a.g.ny : a.g.nz;
  switch (n) {
#define BFCS_C(L) case L: return dir < 0 ? colpass_L<R, L, -1>(a, st) : colpass_L<R, L, +1>(a, st);
    BFCS_C(4) BFCS_C(6) BFCS_C(8) BFCS_C(12) BFCS_C(16) BFCS_C(24) BFCS_C(32) BFCS_C(48)
    BFCS_C(64) BFCS_C(96) BFCS_C(128) BFCS_C(192) BFCS_C(256)
#undef BFCS_C
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_xpass<BFCS_R>(const XArgs<BFCS_R>&, cudaStream_t);
template cudaError_t launch_colpass<BFCS_R>(const CArgs<BFCS_R>&, int, cudaStream_t);

}  // namespace bfcs
