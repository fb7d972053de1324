// FFT passes of one sweep of the modified basic scheme (Algorithm 1):
//  * the x pass, where the inverse transform along x (Eq. 5.10), the
//    polarization tau = L1 eps (Eq. 5.7) and the forward transform along x
//    (Eq. 5.8) run back to back on lines held in shared memory, so the
//    real-space strain never goes to HBM between sweeps;
//  * the column passes along y and z on the half spectrum.
// Compiled once per arithmetic type with BFCS_R = float, double or ff
// (float-float arithmetic on FP64 fields, for the precision ladder).
#include "kernels.h"

#include <cuda.h>

#ifndef BFCS_R
#define BFCS_R float
#endif

namespace bfcs {

// x pass: LPB lines per block, each line as up to 3 complex pair-lines
// (components 2q and 2q+1 as real and imaginary parts), one group of TPF
// threads per pair-line.  Pair-line f keeps its L values in shared memory at
// s[f * LP + pad(n)], pad(n) = n + n/16, which keeps every access below free
// of bank conflicts.
template <int L> struct XCfg {
  static constexpr int RMAX = LineInfo<L>::RMAX;
  static constexpr int TPF = RMAX <= 2 ? 2 : RMAX <= 4 ? 4 : RMAX <= 8 ? 8 : 16;   // threads per pair-line
  static constexpr int LPB = 64 / TPF;
  static constexpr int NCOL = 3 * LPB;
  static constexpr int LP = L + L / 16 + 1;
  static constexpr int THREADS = NCOL * TPF;
};

__device__ __forceinline__ int xpad(int n) { return n + (n >> 4); }

// Blocks per SM the register budget is sized for: FP32 6 (56 registers, a few
// bytes of spill at L >= 96; measured at L = 256: 0.221 ms against 0.231 ms with
// 5 blocks and 0.251 ms with 4, while 7 and 8 spill hundreds of bytes and take
// 0.32-0.33 ms; 1-4% faster than 5 blocks at 96, 128 and 192), float-float 3
// (a 256^3 ladder solve: 100.9 ms, against 101.8 ms with 2 and 101.2 ms with 4).
template <typename R> constexpr int xpass_min_blocks() {
  return sizeof(R) == 4 ? 6 : std::is_same<R, ff>::value ? 3 : 0;
}

template <typename R, int L>
__global__ void __launch_bounds__(XCfg<L>::THREADS, xpass_min_blocks<R>()) k_xpass(XArgs<R> a) {
  const int m = blockIdx.z;
  if (a.st != nullptr && a.st[m].done) return;   // a member that has converged skips
  using C = XCfg<L>;
  using RT = typename RealOf<R>::T;   // storage type of the real fields
  constexpr int LPB = C::LPB, TPF = C::TPF, LP = C::LP;
  constexpr int R1 = LineInfo<L>::R1, R2 = LineInfo<L>::R2;
  constexpr int H = L / 2;
  extern __shared__ unsigned char smem_raw[];
  C2<R>* s = reinterpret_cast<C2<R>*>(smem_raw);
  __shared__ int prow_s[LPB];     // phase-map row of each line of the block, translated by chi
  __shared__ int sx_s;            // x translation in [0, nx)

  const int tid = threadIdx.x;
  const int ncomp = a.ncomp;
  const int npair = (ncomp + 1) >> 1;
  const int ncol = LPB * npair;
  const long long lines = (long long)a.g.ny * a.g.nz;
  const long long line0 = (long long)blockIdx.x * LPB;
  const long long cs = a.g.cs, rn = a.g.n;
  const int p = a.g.p;
  // member-specific fields are read from the launch arguments (a.xm[m]) at
  // their point of use, so none of them stays live in registers across the FFT
  const int mode = a.mode;
  // this thread's pair-line and lane within it
  const int f = tid / TPF, t = tid % TPF;
  const int li = f / npair, q = f - li * npair;
  const long long line = line0 + li;
  const bool fval = f < ncol && line < lines;
  const bool has_b = 2 * q + 1 < ncomp;
  C2<R>* sf = s + f * LP;

  // per-line translation bookkeeping of the polarization (made visible by the
  // barriers of step 1): the phase of voxel (n, y, z) is phase0(n - sx, y - sy, z - sz)
  if (tid < LPB && (mode == XM_SWEEP || mode == XM_REALTAU || mode == XM_REALSIG || mode == XM_SWEEPSIG)) {
    const XMember& M = a.xm[m];
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    const long long ln = line0 + tid;
    if (ln < lines) {
      int y = (int)(ln % ny) - ((M.sy % ny) + ny) % ny, z = (int)(ln / ny) - ((M.sz % nz) + nz) % nz;
      if (y < 0) y += ny;
      if (z < 0) z += nz;
      prow_s[tid] = (z * ny + y) * nx;
    }
    if (tid == 0) sx_s = ((M.sx % nx) + nx) % nx;
  }
  // the block's phase-map rows (untranslated in x) stream into shared memory during
  // the inverse transform, so the polarization does not wait on one load per voxel
  constexpr bool kPhaseStaged = L % 16 == 0;
  __shared__ __align__(16) int8_t ph_s[kPhaseStaged ? LPB : 1][kPhaseStaged ? L : 16];
  const bool polar = mode == XM_SWEEP || mode == XM_REALTAU || mode == XM_REALSIG || mode == XM_SWEEPSIG;
  // 16-byte copies need a 16-byte aligned map (a caller may pass an offset view: then direct loads)
  const bool staged = kPhaseStaged && polar && ((reinterpret_cast<uintptr_t>(a.xm[m].phase) & 15u) == 0);
  if (staged) {
    const XMember& M = a.xm[m];
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    constexpr int CH = kPhaseStaged ? L / 16 : 1;  // 16-byte pieces per row
    for (int q = tid; q < LPB * CH; q += blockDim.x) {
      const int i = q / CH, ch = q - i * CH;
      const long long ln = line0 + i;
      if (ln >= lines) continue;
      int y = (int)(ln % ny) - ((M.sy % ny) + ny) % ny, z = (int)(ln / ny) - ((M.sz % nz) + nz) % nz;
      if (y < 0) y += ny;
      if (z < 0) z += nz;
      cp_async16(&ph_s[i][ch * 16], M.phase + (long long)(z * ny + y) * nx + ch * 16);
    }
    cp_async_commit();
  }

  // ---- 1. inverse transform along x of the pair-line Z = A + i B (C2R), or load real data
  if (mode == XM_SWEEP || mode == XM_C2R || mode == XM_SWEEPSIG) {
    if (fval && t < R2) {
      const C2<R>* rowA = a.spec_in + m * a.spec_ms + (2 * q) * cs + line * p;
      const C2<R>* rowB = rowA + cs;
      C2<R> x[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) {
        const int k = R2 * n1 + t;
        const int kk = k <= H ? k : L - k;
        C2<R> A = rowA[kk];
        C2<R> B = has_b ? rowB[kk] : mk<R>(0, 0);
        if (kk == 0 || kk == H) { A.y = 0; B.y = 0; }     // DC and Nyquist keep their real parts
        if (k > H) { A.y = -A.y; B.y = -B.y; }            // Hermitian extension
        x[n1] = mk<R>(A.x - B.y, A.y + B.x);
      }
      stage1<R, L, +1>(x, t, a.tw);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) sf[xpad(t * R1 + k1)] = x[k1];
    }
    __syncthreads();
    // stage 2 reads and writes the same slots of its pair-line (t + R1 m, m < R2)
    if (fval && t < R1) {
      C2<R> y[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) y[n2] = sf[xpad(n2 * R1 + t)];
      stage2<R, L, +1>(y);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) sf[xpad(t + R1 * k2)] = y[k2];
    }
  } else {
    for (int idx = tid; idx < ncol * L; idx += blockDim.x) {
      const int n = idx % L, ff = idx / L;
      const int i = ff / npair, qq = ff - i * npair;
      const long long ln = line0 + i;
      C2<R> z = mk<R>(0, 0);
      if (ln < lines) {
        const RT* row = (const RT*)a.xm[m].real_in + ln * L + n;
        z.x = ld_real<R>(row[(2 * qq) * rn]);
        z.y = (2 * qq + 1 < ncomp) ? ld_real<R>(row[(2 * qq + 1) * rn]) : R(0);
      }
      s[ff * LP + xpad(n)] = z;
    }
  }
  if (staged) cp_async_wait_all();
  __syncthreads();

  if (mode == XM_C2R) {
    if (a.xm[m].real_out == nullptr) return;     // a member without this output
    for (int idx = tid; idx < ncol * L; idx += blockDim.x) {
      const int n = idx % L, ff = idx / L;
      const int i = ff / npair, qq = ff - i * npair;
      const long long ln = line0 + i;
      if (ln >= lines) continue;
      const C2<R> z = s[ff * LP + xpad(n)];
      RT* row = (RT*)a.xm[m].real_out + ln * L + n;
      row[(2 * qq) * rn] = st_real<R>(z.x);
      if (2 * qq + 1 < ncomp) row[(2 * qq + 1) * rn] = st_real<R>(z.y);
    }
    return;
  }

  // ---- 2. polarization tau = (L(x) - L0) eps, isotropic phases (Eq. 5.7);
  //         sigma = L(x) eps instead in the stress modes
  if (mode == XM_SWEEP || mode == XM_REALTAU || mode == XM_REALSIG || mode == XM_SWEEPSIG) {
    const bool full = mode == XM_REALSIG || mode == XM_SWEEPSIG;
    const int nx = a.g.nx;
    const int sx = sx_s;
    for (int idx = tid; idx < LPB * L; idx += blockDim.x) {
      const int n = idx % L, i = idx / L;
      const long long ln = line0 + i;
      if (ln >= lines) continue;
      C2<R>* c0 = s + (i * 3) * LP + xpad(n);
      const C2<R> p0 = c0[0], p1 = c0[LP], p2 = c0[2 * LP];
      // eps: xx yy zz yz xz xy
      const R e0 = p0.x, e1 = p0.y, e2 = p1.x, e3 = p1.y, e4 = p2.x, e5 = p2.y;
      const XMember& M = a.xm[m];
      int xs = n - sx;
      if (xs < 0) xs += nx;
      const int ph = staged ? (int)ph_s[kPhaseStaged ? i : 0][kPhaseStaged ? xs : 0] : (int)M.phase[prow_s[i] + xs];
      const R tr = e0 + e1 + e2;
      const long long vox = ln * L + n;
      if (M.eps_out != nullptr) {
        RT* o = (RT*)M.eps_out + vox;
        o[0] = st_real<R>(e0); o[rn] = st_real<R>(e1); o[2 * rn] = st_real<R>(e2);
        o[3 * rn] = st_real<R>(e3); o[4 * rn] = st_real<R>(e4); o[5 * rn] = st_real<R>(e5);
      }
      if (M.sig_out != nullptr) {
        const R lt = a.tab.lam[ph] * tr, m2 = R(2) * a.tab.mu[ph];
        RT* o = (RT*)M.sig_out + vox;
        o[0] = st_real<R>(lt + m2 * e0); o[rn] = st_real<R>(lt + m2 * e1); o[2 * rn] = st_real<R>(lt + m2 * e2);
        o[3 * rn] = st_real<R>(m2 * e3); o[4 * rn] = st_real<R>(m2 * e4); o[5 * rn] = st_real<R>(m2 * e5);
      }
      const R lt = (full ? a.tab.lam[ph] : a.tab.lam1[ph]) * tr;
      const R m2 = R(2) * (full ? a.tab.mu[ph] : a.tab.mu1[ph]);
      c0[0] = mk<R>(lt + m2 * e0, lt + m2 * e1);
      c0[LP] = mk<R>(lt + m2 * e2, m2 * e3);
      c0[2 * LP] = mk<R>(m2 * e4, m2 * e5);
    }
    __syncthreads();
  }

  // ---- 3. forward transform along x and split the pair-line into two half spectra
  {
    C2<R> x[R1];
    if (fval && t < R2) {
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) x[n1] = sf[xpad(R2 * n1 + t)];
      stage1<R, L, -1>(x, t, a.tw);
    }
    __syncthreads();
    if (fval && t < R2) {
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) sf[xpad(t * R1 + k1)] = x[k1];
    }
  }
  __syncthreads();
  C2<R> y[R2];
  if (fval && t < R1) {
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) y[n2] = sf[xpad(n2 * R1 + t)];
    stage2<R, L, -1>(y);
  }
  // Thread k1 owns Z[k1 + R1 k2]; Z[L - k] sits in thread (R1 - k1) % R1 at
  // k2' = R2 - 1 - k2 (k1 > 0) or (R2 - k2) % R2 (k1 = 0): one shuffle per k2.
  const int lane = threadIdx.x & 31;
  const int src = (lane & ~(TPF - 1)) | ((R1 - t) % R1);
  const R half = R(0.5) * ((mode == XM_R2C && a.out_scale != R(0)) ? a.out_scale : R(1));
  C2<R>* rowA = a.spec_out + m * a.spec_ms + (2 * q) * cs + line * p;
  C2<R>* rowB = rowA + cs;
  // only the outputs k <= H are stored: k = t + R1 k2 with t < R1 needs k2 <= H / R1
  constexpr int K2MAX = H / R1 + 1 < R2 ? H / R1 + 1 : R2;
#pragma unroll
  for (int k2 = 0; k2 < K2MAX; ++k2) {
    const C2<R> send = (t == 0) ? y[(R2 - k2) % R2] : y[(R2 - 1 - k2 + R2) % R2];
    C2<R> zm;
    zm.x = shfl_real<R>(send.x, src);
    zm.y = shfl_real<R>(send.y, src);
    const int k = t + R1 * k2;
    if (fval && t < R1 && k <= H) {
      const C2<R> Z = y[k2];
      rowA[k] = mk<R>(half * (Z.x + zm.x), half * (Z.y - zm.y));
      if (has_b) rowB[k] = mk<R>(half * (Z.y + zm.y), -half * (Z.x - zm.x));
    }
  }
}

// Column FFT along y or z: each block owns T consecutive kx columns of one
// (other-axis, component) slab; loads are T-wide contiguous row segments.
// L = F1 * F2 in the order given by SW (the default order of Fac<L>, or
// swapped); T and SW are the autotuned choices of an FP32 plan.
constexpr int kColT = 16;

template <int L, int T, bool SW> struct CCfg {
  static constexpr int F1 = SW ? Fac<L>::R2 : Fac<L>::R1;
  static constexpr int F2 = SW ? Fac<L>::R1 : Fac<L>::R2;
  static constexpr int RMAX = F1 > F2 ? F1 : F2;
  static constexpr int THREADS = T * RMAX;
};
template <typename R, int T> constexpr int col_min_blocks() {
  return sizeof(R) == 4 ? (T == 8 ? 6 : T == 16 ? 3 : 1) : 2;
}

template <typename R, int L, int DIR, int T, bool SW>
__global__ void __launch_bounds__(CCfg<L, T, SW>::THREADS, col_min_blocks<R, T>()) k_colpass(CArgs<R> a) {
  const int m = blockIdx.z;
  if (a.st != nullptr && a.st[m].done) return;   // a member that has converged skips
  constexpr int R1 = CCfg<L, T, SW>::F1, R2 = CCfg<L, T, SW>::F2;
  extern __shared__ unsigned char smem_raw[];
  C2<R>* s = reinterpret_cast<C2<R>*>(smem_raw);
  const int tid = threadIdx.x;
  const int mx = a.g.mx, p = a.g.p, ny = a.g.ny;
  const int other = a.axis == 1 ? a.g.nz : ny;
  const int comp = blockIdx.y / other, o = blockIdx.y - comp * other;
  const long long ls = a.axis == 1 ? (long long)p : (long long)ny * p;
  C2<R>* base = a.data + m * a.ms + comp * a.g.cs + (a.axis == 1 ? (long long)o * ny * p : (long long)o * p);
  const int c = tid % T, j = tid / T;
  const int kx = blockIdx.x * T + c;
  const bool valid = kx < mx;
  C2<R>* col = base + kx;
  // stage 1 straight from global: thread (c, j) owns rows R2 n1 + j of column c
  if (j < R2) {
    C2<R> x[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) x[n1] = valid ? col[(R2 * n1 + j) * ls] : mk<R>(0, 0);
    stage1f<R, L, R1, DIR>(x, j, a.tw);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) s[(j * R1 + k1) * T + c] = x[k1];
  }
  __syncthreads();
  // stage 2, outputs straight to global: thread (c, j) owns rows j + R1 k2
  if (j < R1) {
    C2<R> y[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) y[n2] = s[(n2 * R1 + j) * T + c];
    stage2f<R, R2, DIR>(y);
    if (valid) {
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) col[(j + R1 * k2) * ls] = y[k2];
    }
  }
}

// Column FFT along y with the tile loaded by the tensor memory accelerator: one
// bulk tensor copy per block brings the T x L tile (T kx columns, all ny rows of
// one (component, z) plane) into shared memory, completing on an mbarrier;
// stage 1 then reads its rows there (in place, one barrier between the reads
// and the writes) and stage 2 writes straight to global memory as k_colpass.
// The tensor map (a 3D view of the 6-component spectra: floats along kx with
// extent 2 mx, rows of pitch p, planes (member, component, z)) is built by the
// plan; columns past mx read as zeros (out-of-bounds fill) and are not stored.
// The wait is bounded: a copy that does not complete sets the member's fault
// flag (IterState.diverged = 2, reported as a timeout) and the block returns.
[[maybe_unused]] constexpr unsigned kTmaSpinLimit = 1u << 26;   // (FP32 builds only use it)

template <int L, int DIR, int T>
__global__ void __launch_bounds__(CCfg<L, T, false>::THREADS, T == 8 ? 6 : 3)
    k_colpass_tma(CArgs<float> a, const __grid_constant__ CUtensorMap tm) {
  using R = float;
  const int m = blockIdx.z;
  if (a.st != nullptr && a.st[m].done) return;   // a member that has converged skips
  constexpr int R1 = CCfg<L, T, false>::F1, R2 = CCfg<L, T, false>::F2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C2<R>* s = reinterpret_cast<C2<R>*>(smem_raw);   // [row][T], as the copy lands
  __shared__ __align__(8) unsigned long long bar;
  const int tid = threadIdx.x;
  const unsigned bar_a = (unsigned)__cvta_generic_to_shared(&bar);
  const int plane = m * 6 * a.g.nz + blockIdx.y;   // (member, component, z) with blockIdx.y = comp * nz + z
  const int kx0 = blockIdx.x * T;
  if (tid == 0) {
    // fetch the tensor map while the barrier is set up: between y passes other
    // kernels run, so the block's one copy would otherwise wait for it
    asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<unsigned long long>(&tm)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_a));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar_a),
                 "r"((unsigned)(L * T * sizeof(C2<R>)))
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(&tm)), "r"(2 * kx0), "r"(0), "r"(plane), "r"(bar_a)
        : "memory");
  }
  unsigned done = 0, spins = 0;
  while (!done) {
    asm volatile(
        "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], 0;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(bar_a)
        : "memory");
    if (!done && ++spins > kTmaSpinLimit) break;
  }
  if (__syncthreads_or(!done)) {
    // give the copy in flight a second bounded wait before the block leaves its buffer
    for (unsigned k = 0; !done && k < kTmaSpinLimit; ++k)
      asm volatile(
          "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], 0;\nselp.u32 %0, 1, 0, q;\n}\n"
          : "=r"(done)
          : "r"(bar_a)
          : "memory");
    if (tid == 0 && a.st != nullptr) {
      IterState* st = const_cast<IterState*>(a.st) + m;
      atomicExch(&st->diverged, 2);
      atomicExch(&st->done, 1);
    }
    return;
  }
  const int c = tid % T, j = tid / T;
  const int kx = kx0 + c;
  const bool valid = kx < a.g.mx;
  const int ny = a.g.ny, p = a.g.p;
  C2<R>* col = a.data + m * a.ms + (long long)blockIdx.y * ny * p + kx;
  // stage 1 from the landed tile, in place: thread (c, j) owns rows R2 n1 + j
  C2<R> x[R1];
  if (j < R2) {
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) x[n1] = s[(R2 * n1 + j) * T + c];
    stage1f<R, L, R1, DIR>(x, j, a.tw);
  }
  __syncthreads();
  if (j < R2) {
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) s[(j * R1 + k1) * T + c] = x[k1];
  }
  __syncthreads();
  // stage 2, outputs straight to global: thread (c, j) owns rows j + R1 k2
  if (j < R1) {
    C2<R> y[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) y[n2] = s[(n2 * R1 + j) * T + c];
    stage2f<R, R2, DIR>(y);
    if (valid) {
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) col[(long long)(j + R1 * k2) * p] = y[k2];
    }
  }
}

// ---------------------------------------------------------------- dispatch
template <typename R, int L>
static cudaError_t xpass_L(const XArgs<R>& a, int batch, cudaStream_t st) {
  using C = XCfg<L>;
  const long long lines = (long long)a.g.ny * a.g.nz;
  const dim3 grid((unsigned)((lines + C::LPB - 1) / C::LPB), 1, batch);
  const size_t smem = sizeof(C2<R>) * (size_t)C::LP * C::NCOL;
  cudaError_t e = cudaFuncSetAttribute(k_xpass<R, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_xpass<R, L><<<grid, C::THREADS, smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_xpass_b(const XArgs<R>& a0, int batch, cudaStream_t st) {
  const XArgs<R>* ap = &a0;
  XArgs<R> one;
  if (!a0.use_xm) {          // single launch: its scalar fields become member 0
    one = a0;
    XMember& x = one.xm[0];
    x.phase = a0.phase;
    x.sx = a0.sx; x.sy = a0.sy; x.sz = a0.sz;
    x.warm = 0;
    x.real_in = a0.real_in;
    x.eps_out = a0.eps_out;
    x.sig_out = a0.sig_out;
    x.real_out = a0.real_out;
    one.use_xm = 1;
    ap = &one;
  }
  const XArgs<R>& a = *ap;
  switch (a.g.nx) {
#define BFCS_X(L) case L: return xpass_L<R, L>(a, batch, st);
    BFCS_X(4) BFCS_X(6) BFCS_X(8) BFCS_X(12) BFCS_X(16) BFCS_X(24) BFCS_X(32) BFCS_X(48)
    BFCS_X(64) BFCS_X(96) BFCS_X(128) BFCS_X(192) BFCS_X(256)
#undef BFCS_X
    default: return cudaErrorInvalidValue;
  }
}

template <typename R, int L, int DIR, int T, bool SW>
static cudaError_t colpass_LT(const CArgs<R>& a, int batch, cudaStream_t st) {
  const int other = a.axis == 1 ? a.g.nz : a.g.ny;
  dim3 grid((a.g.mx + T - 1) / T, other * a.ncomp, batch);
  const size_t smem = sizeof(C2<R>) * (size_t)L * T;
  cudaError_t e = cudaFuncSetAttribute(k_colpass<R, L, DIR, T, SW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_colpass<R, L, DIR, T, SW><<<grid, CCfg<L, T, SW>::THREADS, smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

template <int L, int DIR, int T>
static cudaError_t colpass_tma_LT(const CArgs<float>& a, int batch, cudaStream_t st) {
  dim3 grid((a.g.mx + T - 1) / T, a.g.nz * 6, batch);
  const size_t smem = sizeof(C2<float>) * (size_t)L * T;
  cudaError_t e = cudaFuncSetAttribute(k_colpass_tma<L, DIR, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_colpass_tma<L, DIR, T><<<grid, CCfg<L, T, false>::THREADS, smem, st>>>(
      a, reinterpret_cast<const CUtensorMap*>(a.tmap)[T == 8 ? 0 : 1]);
  count_launches(1);
  return cudaGetLastError();
}

template <typename R, int L, int DIR>
static cudaError_t colpass_L(const CArgs<R>& a, int batch, cudaStream_t st) {
  if constexpr (sizeof(R) == 4 && L >= 32) {
    // tensor-map tiles: only the sweep's y passes over the 6-component spectra the map
    // was encoded for; any other buffer (the CG vectors) takes the same tile with direct loads
    if (col_variant_tma(a.variant)) {
      const bool map = a.tmap != nullptr && a.data == a.tmap_data && a.axis == 1 && a.ncomp == 6 &&
                       a.ms == 6 * a.g.cs;
      if (a.variant == 6) return map ? colpass_tma_LT<L, DIR, 8>(a, batch, st) : colpass_LT<R, L, DIR, 8, false>(a, batch, st);
      return map ? colpass_tma_LT<L, DIR, 16>(a, batch, st) : colpass_LT<R, L, DIR, 16, false>(a, batch, st);
    }
  }
  if constexpr (sizeof(R) == 4 && L >= 32 && Fac<L>::R1 != Fac<L>::R2) {
    switch (a.variant) {
      case 1: return colpass_LT<R, L, DIR, 8, false>(a, batch, st);
      case 2: return colpass_LT<R, L, DIR, 32, false>(a, batch, st);
      case 3: return colpass_LT<R, L, DIR, 16, true>(a, batch, st);
      case 4: return colpass_LT<R, L, DIR, 8, true>(a, batch, st);
      case 5: return colpass_LT<R, L, DIR, 32, true>(a, batch, st);
      default: break;
    }
  } else if constexpr (sizeof(R) == 4 && L >= 32) {
    switch (a.variant) {
      case 1: return colpass_LT<R, L, DIR, 8, false>(a, batch, st);
      case 2: return colpass_LT<R, L, DIR, 32, false>(a, batch, st);
      default: break;
    }
  }
  return colpass_LT<R, L, DIR, kColT, false>(a, batch, st);
}

template <typename R>
cudaError_t launch_colpass_b(const CArgs<R>& a, int dir, int batch, cudaStream_t st) {
  const int n = a.axis == 1 ? a.g.ny : a.g.nz;
  switch (n) {
#define BFCS_C(L) case L: return dir < 0 ? colpass_L<R, L, -1>(a, batch, st) : colpass_L<R, L, +1>(a, batch, st);
    BFCS_C(4) BFCS_C(6) BFCS_C(8) BFCS_C(12) BFCS_C(16) BFCS_C(24) BFCS_C(32) BFCS_C(48)
    BFCS_C(64) BFCS_C(96) BFCS_C(128) BFCS_C(192) BFCS_C(256)
#undef BFCS_C
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
cudaError_t launch_xpass(const XArgs<R>& a, cudaStream_t st) { return launch_xpass_b<R>(a, 1, st); }
template <typename R>
cudaError_t launch_colpass(const CArgs<R>& a, int dir, cudaStream_t st) { return launch_colpass_b<R>(a, dir, 1, st); }

template cudaError_t launch_xpass<BFCS_R>(const XArgs<BFCS_R>&, cudaStream_t);
template cudaError_t launch_colpass<BFCS_R>(const CArgs<BFCS_R>&, int, cudaStream_t);
template cudaError_t launch_xpass_b<BFCS_R>(const XArgs<BFCS_R>&, int, cudaStream_t);
template cudaError_t launch_colpass_b<BFCS_R>(const CArgs<BFCS_R>&, int, int, cudaStream_t);

}  // namespace bfcs
