// Conjugate gradients on the operator of Eq. 5.13 (Algorithm 2):
//   A(eps) = eps - F^-1{ U0(xi) : F[ L1(x) : eps ] },
// solved for the strain correction in the compatible, zero-mean fields, where
// A is self-adjoint and positive definite in the inner product
// <a, b>_C0 = sum over voxels of a : C0 : b  (it equals sum a : L(x) : b there).
// The vectors live in the sweep's state layout (x transformed, y and z in real
// space, component-major half spectrum); by Parseval along x an inner product
// is sum over stored modes of w(kx) Re(a : C0 : conj b) with w = 1 at kx = 0
// and kx = nx/2 and 2 elsewhere (a common factor nx is dropped).  Every kernel
// is batched over members (blockIdx.y) and returns at entry for a member whose
// CG has finished; the scalars alpha, beta and the convergence test are
// computed on the device, so an iteration needs no host synchronisation.
#include "kernels.h"

#ifndef BFCS_R
#define BFCS_R float
#endif

namespace bfcs {

constexpr int kCgThreads = 256;

// Re(a : C0 : conj b) for the 6 tensorial components (xx yy zz yz xz xy), in the
// vectors' precision (FP32 vectors: FP32 per mode; the caller sums 16 modes in R
// and then adds in FP64: GB300's FP64 pipe would otherwise bound the vector kernels)
template <typename R>
__device__ __forceinline__ R c0dot(const C2<R> (&a)[6], const C2<R> (&b)[6], R lam0, R mu0) {
  const R ta_r = a[0].x + a[1].x + a[2].x, ta_i = a[0].y + a[1].y + a[2].y;
  const R tb_r = b[0].x + b[1].x + b[2].x, tb_i = b[0].y + b[1].y + b[2].y;
  R s = R(0);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const R w = c < 3 ? R(1) : R(2);
    s += w * (a[c].x * b[c].x + a[c].y * b[c].y);
  }
  return lam0 * (ta_r * tb_r + ta_i * tb_i) + R(2) * mu0 * s;
}

__device__ __forceinline__ double block_reduce(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
  return t;
}

struct CgMode { enum : int { INIT = 0, PQ = 1, UPDATE = 2, DIR = 3 }; };

// INIT:   r = s - c (s = one sweep applied to c), p = r, partial <r, r>
// PQ:     q = p - q (q held U0 * L1 p), partial <p, q>
// UPDATE: c += alpha p, r -= alpha q, partial <r, r>
// DIR:    p = r + beta p
template <typename R>
__global__ void __launch_bounds__(kCgThreads) k_cg_vec(CgArgs<R> a, int mode) {
  const int m = blockIdx.y;
  if (a.cg[m].done) return;
  __shared__ double red[32];
  const Geo g = a.g;
  const long long off = m * a.ms;
  C2<R>* c = a.c + off;
  C2<R>* r = a.r + off;
  C2<R>* p = a.p + off;
  C2<R>* q = a.q + off;
  const C2<R>* s = a.s != nullptr ? a.s + off : nullptr;
  __shared__ R cst[4];          // alpha, beta, lam0, mu0, converted once per block
  if (threadIdx.x == 0) {
    cst[0] = (R)a.cg[m].alpha;
    cst[1] = (R)a.cg[m].beta;
    cst[2] = (R)a.lam0;
    cst[3] = (R)a.mu0;
  }
  __syncthreads();
  const R alpha = cst[0], beta = cst[1], lam0 = cst[2], mu0 = cst[3];
  const long long modes = (long long)g.nz * g.ny * g.mx;
  // partial sums: 16 grid-stride modes in R (their products are R), then one FP64 add
  double acc = 0.0;
  const int stride = gridDim.x * blockDim.x;
  // 32-bit index arithmetic: a member's spectrum has at most 256 * 256 * 129 modes
  for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < (int)modes; i0 += 16 * stride) {
    R part = R(0);
    for (int j = 0; j < 16; ++j) {
      const int i = i0 + j * stride;
      if (i >= (int)modes) break;
      const int kx = i % g.mx;
      const long long gi = (long long)(i / g.mx) * g.p + kx;
      const R w = (kx == 0 || 2 * kx == g.nx) ? R(1) : R(2);
      C2<R> u[6], v[6];
      if (mode == CgMode::INIT) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const C2<R> x = s[k * g.cs + gi] - c[k * g.cs + gi];
          r[k * g.cs + gi] = x;
          p[k * g.cs + gi] = x;
          u[k] = x;
        }
        part += w * c0dot<R>(u, u, lam0, mu0);
      } else if (mode == CgMode::PQ) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          u[k] = p[k * g.cs + gi];
          v[k] = u[k] - q[k * g.cs + gi];
          q[k * g.cs + gi] = v[k];
        }
        part += w * c0dot<R>(u, v, lam0, mu0);
      } else if (mode == CgMode::UPDATE) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          c[k * g.cs + gi] = c[k * g.cs + gi] + scale(p[k * g.cs + gi], alpha);
          u[k] = r[k * g.cs + gi] - scale(q[k * g.cs + gi], alpha);
          r[k * g.cs + gi] = u[k];
        }
        part += w * c0dot<R>(u, u, lam0, mu0);
      } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) p[k * g.cs + gi] = r[k * g.cs + gi] + scale(p[k * g.cs + gi], beta);
      }
    }
    acc += (double)part;
  }
  if (mode == CgMode::DIR) return;
  const double t = block_reduce(acc, red);
  if (threadIdx.x == 0) a.part[(long long)m * gridDim.x + blockIdx.x] = t;
}

// Sum the partials of each member in a fixed order and advance its scalars:
//  INIT:   rr = rr0 = <r0, r0>
//  PQ:     alpha = rr / <p, A p> (a non-positive <p, A p> ends the member: breakdown)
//  UPDATE: beta = <r, r> / rr, rr = <r, r>, iterations + 1; done once
//          <r, r> <= tol^2 rr0, at the iteration limit, or when <r, r> has not
//          reached a new minimum for kCgStagnation iterations
static __global__ void k_cg_scalar(const double* part, int nparts, CgState* cg, IterState* skip, int mode) {
  __shared__ double red[32];
  const int m = blockIdx.x;
  CgState& S = cg[m];
  if (S.done) return;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[(long long)m * nparts + i];
  const double t = block_reduce(acc, red);
  if (threadIdx.x != 0) return;
  bool fin = false;
  if (mode == CgMode::INIT) {
    S.rr = S.rr0 = S.best = t;
    S.iters = S.best_it = 0;
    fin = !(t > 0.0);
  } else if (mode == CgMode::PQ) {
    if (t > 0.0 && t == t) S.alpha = S.rr / t;
    else fin = true;
  } else {
    S.beta = S.rr > 0.0 ? t / S.rr : 0.0;
    S.rr = t;
    S.iters += 1;
    if (t < S.best) { S.best = t; S.best_it = S.iters; }
    // converged, at the iteration limit, or stagnating at the rounding floor
    fin = !(t == t) || t <= S.tol2 * S.rr0 || S.iters >= S.maxit || S.iters - S.best_it >= kCgStagnation;
  }
  if (fin) {
    S.done = 1;
    skip[m].done = 1;
  }
}

template <typename R>
cudaError_t launch_cg_vec(const CgArgs<R>& a, int mode, int batch, cudaStream_t st) {
  k_cg_vec<R><<<dim3(kCgParts, batch), kCgThreads, 0, st>>>(a, mode);
  count_launches(1);
  if (mode == CgMode::DIR) return cudaGetLastError();
  k_cg_scalar<<<batch, kCgThreads, 0, st>>>(a.part, kCgParts, a.cg, a.skip, mode);
  count_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_cg_vec<BFCS_R>(const CgArgs<BFCS_R>&, int, int, cudaStream_t);

}  // namespace bfcs
