// Setup and bookkeeping kernels: phase-map voxelisation (integer), the BFCS
// body-force field, input validation, FP64 reductions of the residual and the
// translated-averaging accumulation (Eqs. 3.5-3.6).
#include "kernels.h"

#include <atomic>

namespace bfcs {

static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

bool supported_len(int n) {
  switch (n) {
    case 4: case 6: case 8: case 12: case 16: case 24: case 32: case 48: case 64:
    case 96: case 128: case 192: case 256: return true;
    default: return false;
  }
}

constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)((blockDim.x + 31) / 32); ++w) t += red[w];
  return t;   // valid in thread 0
}

// ---------------------------------------------------------------- a1: phase map
// A voxel with doubled centre 2i+1 (cell coordinates) is inside sphere
// (X, Y, Z, T, phase) when the squared periodic minimum-image distance on the
// doubled grid is <= T; the last containing sphere wins; else phase 0.
__device__ __forceinline__ int min_image2(int v, int n2) {   // v in doubled units, period n2 = 2n
  int d = v % n2;
  if (d < 0) d += n2;
  if (d >= n2 / 2) d -= n2;
  return d;
}

__global__ void k_voxelize(int8_t* out, int nx, int ny, int nz, int cx, int cy, int cz,
                           const int* __restrict__ sph, int nsph) {
  // one thread per voxel of the unit cell; its phase is written to every
  // periodic replica of that voxel in the grid
  extern __shared__ int ssph[];
  const long long ncell = (long long)cx * cy * cz;
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int x = (int)(v % cx), y = (int)((v / cx) % cy), z = (int)(v / ((long long)cx * cy));
  const int ix = 2 * x + 1, iy = 2 * y + 1, iz = 2 * z + 1;
  int ph = 0;
  for (int base = 0; base < nsph; base += 1024) {
    const int cnt = min(1024, nsph - base);
    __syncthreads();
    for (int k = threadIdx.x; k < cnt * 5; k += blockDim.x) ssph[k] = sph[base * 5 + k];
    __syncthreads();
    if (v < ncell) {
      for (int k = 0; k < cnt; ++k) {
        const int* S = ssph + 5 * k;
        const int dx = min_image2(ix - S[0], 2 * cx);
        const int dy = min_image2(iy - S[1], 2 * cy);
        const int dz = min_image2(iz - S[2], 2 * cz);
        if (dx * dx + dy * dy + dz * dz <= S[3]) ph = S[4];
      }
    }
  }
  if (v >= ncell) return;
  const int rx = nx / cx, ry = ny / cy, rz = nz / cz;
  for (int kz = 0; kz < rz; ++kz)
    for (int ky = 0; ky < ry; ++ky)
      for (int kx = 0; kx < rx; ++kx)
        out[((long long)(kz * cz + z) * ny + (ky * cy + y)) * nx + (kx * cx + x)] = (int8_t)ph;
}

cudaError_t launch_voxelize(int8_t* out, int nx, int ny, int nz, int cx, int cy, int cz,
                            const int* sph_dev, int nsph, cudaStream_t s) {
  const long long ncell = (long long)cx * cy * cz;
  const unsigned grid = (unsigned)((ncell + 255) / 256);
  k_voxelize<<<grid, 256, 1024 * 5 * sizeof(int), s>>>(out, nx, ny, nz, cx, cy, cz, sph_dev, nsph);
  count_launches(1);
  return cudaGetLastError();
}

// voxel (x, y, z) of linear index v = x + nx (y + ny z): 32-bit unsigned
// arithmetic when the grid has fewer than 2^32 voxels (`small`), else 64-bit
__device__ __forceinline__ void lin_xyz(long long v, int nx, int ny, bool small, int& x, int& y, int& z) {
  if (small) {
    const unsigned u = (unsigned)v, t = u / (unsigned)nx;
    x = (int)(u - t * (unsigned)nx);
    y = (int)(t % (unsigned)ny);
    z = (int)(t / (unsigned)ny);
  } else {
    x = (int)(v % nx);
    y = (int)((v / nx) % ny);
    z = (int)(v / ((long long)nx * ny));
  }
}

// ---------------------------------------------------------------- a2: body force
// b1 = d phi/d x1, phi = (1 - r^2/a^2)^3 for r < a (Eq. 2.5 form), at voxel
// centres i + 0.5, periodic minimum image about the centre; FP64, mean removed.
// rn = (1/nx, 1/ny, 1/nz) in FP32 for the screen: a product and a quotient can
// round differently only at offsets of exactly half a period, where both images
// are equally far, so the screen's decision is the same.
__device__ __forceinline__ double bf_value(int x, int y, int z, int nx, int ny, int nz, float3 rn, double cx,
                                           double cy, double cz, double a) {
  {
    // cheap FP32 screen: voxels clearly outside the support (beyond a + 1 voxel) are 0
    float fx = (float)x + 0.5f - (float)cx, fy = (float)y + 0.5f - (float)cy, fz = (float)z + 0.5f - (float)cz;
    fx -= (float)nx * rintf(fx * rn.x);
    fy -= (float)ny * rintf(fy * rn.y);
    fz -= (float)nz * rintf(fz * rn.z);
    const float lim = (float)a + 1.0f;
    if (fabsf(fx) > lim || fabsf(fy) > lim || fabsf(fz) > lim) return 0.0;
  }
  double dx = x + 0.5 - cx, dy = y + 0.5 - cy, dz = z + 0.5 - cz;
  dx -= nx * rint(dx / nx);
  dy -= ny * rint(dy / ny);
  dz -= nz * rint(dz / nz);
  const double r2 = dx * dx + dy * dy + dz * dz, a2 = a * a;
  if (!(r2 < a2)) return 0.0;
  const double s = 1.0 - r2 / a2;
  return -6.0 * dx * s * s / a2;
}

constexpr int kBfBlocks = 1024;

__global__ void k_bf_partial(double* part, long long n, int nx, int ny, int nz, double cx, double cy,
                             double cz, double a) {
  __shared__ double red[32];
  double acc = 0.0;
  const bool small = n <= 0xFFFFFFFFLL;
  const float3 rn = make_float3(1.0f / (float)nx, 1.0f / (float)ny, 1.0f / (float)nz);
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    lin_xyz(v, nx, ny, small, x, y, z);
    acc += bf_value(x, y, z, nx, ny, nz, rn, cx, cy, cz, a);
  }
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_sum_parts(double* part, int nparts, double* out, double scale) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[i];
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) *out = t * scale;
}

template <typename R>
__global__ void k_bf_write(R* b, long long n, int nx, int ny, int nz, double cx, double cy, double cz,
                           double a, const double* mean) {
  const double m = *mean;
  const bool small = n <= 0xFFFFFFFFLL;
  const float3 rn = make_float3(1.0f / (float)nx, 1.0f / (float)ny, 1.0f / (float)nz);
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    lin_xyz(v, nx, ny, small, x, y, z);
    b[v] = (R)(bf_value(x, y, z, nx, ny, nz, rn, cx, cy, cz, a) - m);
    b[n + v] = R(0);
    b[2 * n + v] = R(0);
  }
}

int body_force_scratch(long long) { return kBfBlocks + 1; }

template <typename R>
cudaError_t launch_body_force(R* b, int nx, int ny, int nz, double cx, double cy, double cz, double a,
                              double* scratch, cudaStream_t s) {
  const long long n = (long long)nx * ny * nz;
  k_bf_partial<<<kBfBlocks, kRedThreads, 0, s>>>(scratch, n, nx, ny, nz, cx, cy, cz, a);
  k_sum_parts<<<1, kRedThreads, 0, s>>>(scratch, kBfBlocks, scratch + kBfBlocks, 1.0 / (double)n);
  k_bf_write<R><<<kBfBlocks, kRedThreads, 0, s>>>(b, n, nx, ny, nz, cx, cy, cz, a, scratch + kBfBlocks);
  count_launches(3);
  return cudaGetLastError();
}

// Same three kernels with a caller-chosen block count; the scratch holds
// `blocks` FP64 partial sums and the mean at scratch[blocks].
template <typename R>
cudaError_t launch_body_force_blocks(R* b, int nx, int ny, int nz, double cx, double cy, double cz,
                                     double a, int blocks, double* scratch, cudaStream_t s) {
  const long long n = (long long)nx * ny * nz;
  k_bf_partial<<<blocks, kRedThreads, 0, s>>>(scratch, n, nx, ny, nz, cx, cy, cz, a);
  k_sum_parts<<<1, kRedThreads, 0, s>>>(scratch, blocks, scratch + blocks, 1.0 / (double)n);
  k_bf_write<R><<<blocks, kRedThreads, 0, s>>>(b, n, nx, ny, nz, cx, cy, cz, a, scratch + blocks);
  count_launches(3);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- polarization (Eq. 5.7)
template <typename R>
__global__ void k_polarize(R* tau, const R* eps, const int8_t* phase, PhaseTab<R> tab, long long n) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    int ph = phase[v];
    ph = (ph >= 0 && ph < kMaxPhases) ? ph : 0;
    const R l1 = tab.lam1[ph], m2 = R(2) * tab.mu1[ph];
    R e[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = eps[c * n + v];
    const R lt = l1 * (e[0] + e[1] + e[2]);
#pragma unroll
    for (int c = 0; c < 6; ++c) tau[c * n + v] = m2 * e[c] + (c < 3 ? lt : R(0));
  }
}

template <typename R>
cudaError_t launch_polarize(R* tau, const R* eps, const int8_t* phase, const PhaseTab<R>& tab, long long n,
                            cudaStream_t s) {
  const long long want = (n + kRedThreads - 1) / kRedThreads;
  const int blocks = (int)std::min<long long>(want, 8LL * 152);
  k_polarize<R><<<std::max(blocks, 1), kRedThreads, 0, s>>>(tau, eps, phase, tab, n);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- validation
constexpr int kValBlocks = 512;

template <typename R>
__global__ void k_validate(const int8_t* phase, const R* b, long long n, int* iout, double* part) {
  __shared__ double red[32];
  __shared__ int smin, smax;
  if (threadIdx.x == 0) { smin = 127; smax = -128; }
  __syncthreads();
  int lmin = 127, lmax = -128;
  double s[3] = {0, 0, 0}, sa[3] = {0, 0, 0};
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const int ph = phase[v];
    lmin = min(lmin, ph); lmax = max(lmax, ph);
    if (b != nullptr) {
#pragma unroll
      for (int c = 0; c < 3; ++c) { const double x = (double)b[c * n + v]; s[c] += x; sa[c] += fabs(x); }
    }
  }
  atomicMin(&smin, lmin);
  atomicMax(&smax, lmax);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double t = block_sum(s[c], red);
    if (threadIdx.x == 0) part[(2 * c) * gridDim.x + blockIdx.x] = t;
    const double ta = block_sum(sa[c], red);
    if (threadIdx.x == 0) part[(2 * c + 1) * gridDim.x + blockIdx.x] = ta;
  }
  __syncthreads();
  if (threadIdx.x == 0) { atomicMin(&iout[0], smin); atomicMax(&iout[1], smax); }
}

__global__ void k_validate_final(const double* part, int nparts, double* dout) {
  __shared__ double red[32];
  for (int j = 0; j < 6; ++j) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[j * nparts + i];
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) dout[(j & 1) * 3 + j / 2] = t;
    __syncthreads();
  }
}

__global__ void k_init_minmax(int* iout) { iout[0] = 127; iout[1] = -128; }

int validate_scratch(long long) { return 6 * kValBlocks; }

template <typename R>
cudaError_t launch_validate(const int8_t* phase, const R* b, long long n, int* iout, double* dout,
                            double* scratch, cudaStream_t s) {
  k_init_minmax<<<1, 1, 0, s>>>(iout);
  k_validate<R><<<kValBlocks, kRedThreads, 0, s>>>(phase, b, n, iout, scratch);
  k_validate_final<<<1, kRedThreads, 0, s>>>(scratch, kValBlocks, dout);
  count_launches(3);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- residual denominators
// sum over modes with xi != 0 of w |b_hat|^2 (w = 2 for 0 < kx < nx/2: the
// mirrored half of the spectrum), giving the full-spectrum norm of b_hat.
template <typename R>
__global__ void k_bden(const C2<R>* bhat, Geo g, ResidSlot* part, long long b_ms) {
  __shared__ double red[32];
  const int m = blockIdx.y;
  bhat += m * b_ms;
  part += m * gridDim.x;
  const long long modes = (long long)g.nz * g.ny * g.mx;
  double acc = 0.0;
  // 32-bit index arithmetic: a member's spectrum has at most 256 * 256 * 129 modes
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (int)modes; i += gridDim.x * blockDim.x) {
    const int kx = i % g.mx;
    const int r = i / g.mx;
    const int ky = r % g.ny, kz = r / g.ny;
    const int sx = signed_k(kx, g.nx), sy = signed_k(ky, g.ny), sz = signed_k(kz, g.nz);
    if (sx == 0 && sy == 0 && sz == 0) continue;
    const double w = (kx == 0 || 2 * kx == g.nx) ? 1.0 : 2.0;
    const long long gi = (long long)r * g.p + kx;
    if constexpr (sizeof(R) == 4) {
      // |b_hat|^2 of the mode in FP32 (relative 1e-7 is ample for a normaliser), summed in
      // FP64: one FP64 operation per mode instead of twelve on GB300's slow FP64 pipe
      float t = 0.0f;
      for (int c = 0; c < 3; ++c) {
        const C2<R> v = bhat[c * g.cs + gi];
        t += v.x * v.x + v.y * v.y;
      }
      acc += w * (double)t;
    } else {
      for (int c = 0; c < 3; ++c) {
        const C2<R> v = bhat[c * g.cs + gi];
        acc += w * ((double)v.x * v.x + (double)v.y * v.y);
      }
    }
  }
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x].num = t;
}

__global__ void k_bden_final(const ResidSlot* part, int nparts, IterState* st) {
  __shared__ double red[32];
  const int m = blockIdx.x;
  part += m * nparts;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[i].num;
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) st[m].bden = sqrt(t);
}

template <typename R>
cudaError_t launch_bden(const C2<R>* bhat, const Geo& g, ResidSlot* part, IterState* st, cudaStream_t s,
                        int batch, long long b_ms) {
  const int blocks = 512;
  k_bden<R><<<dim3(blocks, batch), kRedThreads, 0, s>>>(bhat, g, part, b_ms);
  k_bden_final<<<batch, kRedThreads, 0, s>>>(part, blocks, st);
  count_launches(2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- residual reduction (Eq. 5.11)
// r = sqrt(sum partials) / D, D = ||b_hat|| + xi_min |sigma_hat(0)|_F with
// sigma_hat(0) = N C0 E + tau_hat(0) and xi_min = 2 pi / max N_a.
__global__ void k_resid_reduce(const ResidSlot* part, int nparts, IterState* sts, const Member* mem,
                               double* hist, int hist_cap, double tol, double lam0, double mu0, double E0,
                               double E1, double E2, double E3, double E4, double E5, double n, int maxdim,
                               int mode, int warm_all, int stall_window, int check_max, int maxit,
                               unsigned long long* io) {
  __shared__ double red[32];
  const int m = blockIdx.x;
  IterState* st = sts + m;
  if (mode == GM_SWEEP && st->done) return;
  __shared__ int no_check;   // decided by one thread: thread 0 advances st->iters below
  if (threadIdx.x == 0) {
    const int sw = st->iters, nc = st->next_check;
    no_check = mode == GM_SWEEP && check_max > 1 && sw != nc;
    if (io != nullptr && mode == GM_SWEEP) {
      // what the Green pass of this sweep moved besides its fixed traffic: d_prev read, d written
      const bool rd = check_max <= 1 || sw == nc;
      const bool wr = check_max <= 1 || rd || sw + 1 == nc || sw + 1 >= maxit;
      atomicAdd(io, (unsigned long long)rd);
      atomicAdd(io + 1, (unsigned long long)wr);
    }
  }
  __syncthreads();
  if (no_check) {
    // no residual on this sweep (the Green pass wrote no partials)
    if (threadIdx.x == 0) {
      const int sweep = st->iters;
      if (sweep < hist_cap && hist != nullptr) hist[(long long)m * hist_cap + sweep] = NAN;
      st->iters = sweep + 1;
    }
    return;
  }
  part += m * nparts;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[i].num;
  const double t = block_sum(acc, red);
  if (threadIdx.x != 0) return;
  double E[6] = {E0, E1, E2, E3, E4, E5};
  int warm = warm_all;
  if (mem != nullptr) {
    for (int c = 0; c < 6; ++c) E[c] = mem[m].E[c];
    warm = mem[m].warm;
    if (mem[m].tol >= 0.0) tol = mem[m].tol;
  }
  const double trE = E[0] + E[1] + E[2];
  double s0[6];
  for (int c = 0; c < 6; ++c)
    s0[c] = mode == kReduceDefect ? st->tau0[c]
                                  : n * (2.0 * mu0 * E[c] + (c < 3 ? lam0 * trE : 0.0)) + st->tau0[c];
  const double s0n = sqrt(s0[0] * s0[0] + s0[1] * s0[1] + s0[2] * s0[2] +
                          2.0 * (s0[3] * s0[3] + s0[4] * s0[4] + s0[5] * s0[5]));
  const double den = st->bden + 6.283185307179586 / (double)maxdim * s0n;
  double r = den > 0.0 ? sqrt(t) / den : sqrt(t);
  if (mode == GM_FINAL || mode == kReduceDefect) { st->resid_final = r; return; }
  const int sweep = st->iters;
  const bool skip_check = warm && sweep == 0;
  if (skip_check) r = INFINITY;
  if (sweep < hist_cap && hist != nullptr) hist[(long long)m * hist_cap + sweep] = r;
  // sweep of the next evaluation: with sparse evaluation, where the contraction
  // rate between the last two evaluations predicts r <= tol (at most check_max
  // sweeps ahead; every check_max sweeps when tol = 0), else the next sweep
  int gap = 1;
  if (check_max > 1 && !skip_check) {
    if (!(tol > 0.0)) {
      gap = check_max;
    } else if (st->checks > 0 && sweep > st->last_check && r > tol && r < st->resid_last && r > 0.0) {
      const double rate = pow(r / st->resid_last, 1.0 / (double)(sweep - st->last_check));
      const double need = ceil(log(tol / r) / log(rate));
      gap = (int)fmin(fmax(need, 1.0), (double)check_max);
    }
  }
  st->next_check = sweep + gap;
  if (!skip_check) {
    st->last_check = sweep;
    st->checks += 1;
  }
  st->resid_last = r;
  st->iters = sweep + 1;
  if (skip_check) return;
  if (!(r == r && r < INFINITY)) { st->diverged = 1; st->done = 1; return; }
  if (r <= tol) { st->done = 1; return; }
  // stall: the residual did not drop by 10% over stall_window sweeps
  if (stall_window > 0) {
    if (st->stall_ref == 0.0) { st->stall_ref = r; st->stall_at = sweep; }
    else if (sweep - st->stall_at >= stall_window) {
      if (r > 0.9 * st->stall_ref) { st->stalled = 1; st->done = 1; }
      else { st->stall_ref = r; st->stall_at = sweep; }
    }
  }
}

cudaError_t launch_resid_reduce(const ResidSlot* part, int nparts, IterState* st, const Member* mem,
                                double* hist, int hist_cap, double tol, double lam0, double mu0,
                                const double* E, long long n, int maxdim, int mode, int warm_all,
                                int stall_window, int check_max, int maxit, unsigned long long* io, int batch,
                                cudaStream_t s) {
  k_resid_reduce<<<batch, 1024, 0, s>>>(part, nparts, st, mem, hist, hist_cap, tol, lam0, mu0, E[0], E[1],
                                        E[2], E[3], E[4], E[5], (double)n, maxdim, mode, warm_all,
                                        stall_window, check_max, maxit, io);
  count_launches(1);
  return cudaGetLastError();
}

struct SlotIdx { int idx[kMaxBatch]; };

__global__ void k_defect_final(const ResidSlot* part, int nparts, IterState* sts, SlotIdx si, int maxdim) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  part += j * nparts;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[i].num;
  const double t = block_sum(acc, red);
  if (threadIdx.x != 0) return;
  IterState* st = sts + si.idx[j];
  const double* s0 = st->tau0;
  const double s0n = sqrt(s0[0] * s0[0] + s0[1] * s0[1] + s0[2] * s0[2] +
                          2.0 * (s0[3] * s0[3] + s0[4] * s0[4] + s0[5] * s0[5]));
  const double den = st->bden + 6.283185307179586 / (double)maxdim * s0n;
  st->resid_final = den > 0.0 ? sqrt(t) / den : sqrt(t);
}

cudaError_t launch_defect_final(const ResidSlot* part, int nparts, IterState* st, const int* idx_host, int batch,
                                int maxdim, cudaStream_t s) {
  SlotIdx si{};
  for (int j = 0; j < batch; ++j) si.idx[j] = idx_host[j];
  k_defect_final<<<batch, kRedThreads, 0, s>>>(part, nparts, st, si, maxdim);
  count_launches(1);
  return cudaGetLastError();
}

bool col_variant_valid(int v, int n) {
  if (v == 0) return true;
  if (v < 0 || v >= kColVariants || n < 32 || !supported_len(n)) return false;
  if (col_variant_tma(v)) return n <= 256;   // one box of n rows (a box edge is at most 256)
  if (!col_variant_swap(v)) return true;
  return n != 64 && n != 256;   // 64 = 8 x 8 and 256 = 16 x 16 have one order only
}

// ---------------------------------------------------------------- a10: translated averaging
// acc layout (30 x N, FP64): <u> 3, <u>^(1) 3, <eps> 6, <eps>^(1) 6, <sigma> 6, <sigma>^(1) 6.
template <typename R>
__global__ void k_accumulate(double* acc, int* hits, const R* eps, const R* sig, const R* u,
                             const int8_t* phase, int sx, int sy, int sz, int nx, int ny, int nz) {
  const long long n = (long long)nx * ny * nz;
  const bool small = n <= 0xFFFFFFFFLL;
  // shifts reduced to [0, n) once: the per-voxel translation is then one compare
  const int sxr = ((sx % nx) + nx) % nx, syr = ((sy % ny) + ny) % ny, szr = ((sz % nz) + nz) % nz;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    lin_xyz(v, nx, ny, small, x, y, z);
    int xs = x - sxr; if (xs < 0) xs += nx;
    int ys = y - syr; if (ys < 0) ys += ny;
    int zs = z - szr; if (zs < 0) zs += nz;
    const bool in = phase[((long long)zs * ny + ys) * nx + xs] != 0;
    for (int c = 0; c < 3; ++c) {
      const double val = (double)u[c * n + v];
      acc[c * n + v] += val;
      if (in) acc[(3 + c) * n + v] += val;
    }
    for (int c = 0; c < 6; ++c) {
      const double e = (double)eps[c * n + v], sg = (double)sig[c * n + v];
      acc[(6 + c) * n + v] += e;
      acc[(18 + c) * n + v] += sg;
      if (in) { acc[(12 + c) * n + v] += e; acc[(24 + c) * n + v] += sg; }
    }
    if (in) hits[v] += 1;
  }
}

template <typename R>
cudaError_t launch_accumulate(double* acc, int* hits, const R* eps, const R* sig, const R* u,
                              const int8_t* phase, int sx, int sy, int sz, int nx, int ny, int nz,
                              cudaStream_t s) {
  k_accumulate<R><<<4 * 152, 256, 0, s>>>(acc, hits, eps, sig, u, phase, sx, sy, sz, nx, ny, nz);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_scale(double* acc, long long count, double f) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    acc[i] *= f;
}

cudaError_t launch_scale(double* acc, long long count, double f, cudaStream_t s) {
  k_scale<<<4 * 152, 256, 0, s>>>(acc, count, f);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- small device -> pinned-host reads
// A kernel writes the words straight into the pinned host buffer (its address is
// valid on the device under unified addressing): the read takes no copy engine, so
// it never waits behind large transfers that other streams keep on the engines.
__global__ void k_copy_words(unsigned* dst, const unsigned* src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
  __threadfence_system();
}
cudaError_t launch_copy_words(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  k_copy_words<<<1, 256, 0, s>>>((unsigned*)dst, (const unsigned*)src, (int)(bytes / sizeof(unsigned)));
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- RVE diagnostic (Def. 2.2)
// Shell maxima of the pointwise norm about a centre on the half-voxel lattice
// (doubled coordinates c2): voxel v lies in shell k = floor(d) where (2d)^2 =
// D2 is an integer, so the shell is decided exactly (k = isqrt(D2) >> 1).  Per
// block the maxima are kept in shared memory as the bit patterns of
// non-negative doubles (their unsigned order is the numeric order), then merged
// into bits[] with one atomicMax per shell: the result does not depend on order.
template <typename R>
__global__ void __launch_bounds__(256) k_radial_max(const R* f, int ncomp, int nx, int ny, int nz, int c2x, int c2y,
                                                  int c2z, int nbins, unsigned long long* bits,
                                                  unsigned long long* counts) {
  extern __shared__ unsigned long long rsh[];      // [nbins] maxima, [nbins] counts
  for (int i = threadIdx.x; i < 2 * nbins; i += blockDim.x) rsh[i] = 0ull;
  __syncthreads();
  const int n = nx * ny * nz;                      // at most 256^3
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int x = v % nx, y = (v / nx) % ny, z = v / (nx * ny);
    int dx = (2 * x + 1 - c2x) % (2 * nx), dy = (2 * y + 1 - c2y) % (2 * ny), dz = (2 * z + 1 - c2z) % (2 * nz);
    if (dx < 0) dx += 2 * nx;
    if (dy < 0) dy += 2 * ny;
    if (dz < 0) dz += 2 * nz;
    if (dx > nx) dx -= 2 * nx;
    if (dy > ny) dy -= 2 * ny;
    if (dz > nz) dz -= 2 * nz;
    const int D2 = dx * dx + dy * dy + dz * dz;
    int r = (int)sqrtf((float)D2);
    while (r * r > D2) --r;
    while ((r + 1) * (r + 1) <= D2) ++r;
    const int k = r >> 1;
    if (k >= nbins) continue;
    double q = 0.0;
    for (int c = 0; c < ncomp; ++c) {
      const double fc = (double)f[(long long)c * n + v];
      q += (c < 3 ? 1.0 : 2.0) * fc * fc;
    }
    atomicMax(&rsh[k], (unsigned long long)__double_as_longlong(sqrt(q)));
    atomicAdd(&rsh[nbins + k], 1ull);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nbins; i += blockDim.x)
    if (rsh[nbins + i] != 0ull) {
      atomicMax(&bits[i], rsh[i]);
      atomicAdd(&counts[i], rsh[nbins + i]);
    }
}

template <typename R>
cudaError_t launch_radial_max(const R* f, int ncomp, int nx, int ny, int nz, const int c2[3], int nbins,
                              unsigned long long* bits, unsigned long long* counts, cudaStream_t s) {
  k_radial_max<R><<<2 * 152, 256, 2 * (size_t)nbins * sizeof(unsigned long long), s>>>(
      f, ncomp, nx, ny, nz, c2[0], c2[1], c2[2], nbins, bits, counts);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- effective moduli (Eqs. 6.1-6.3, 3.2)
// Per member m (blockIdx.y): the 13 FP64 sums  sum sigma_c (6), sum over the
// inclusion voxels (phase != 0) of eps_c (6) and their count, as one partial per
// block in part[(m * gridDim.x + block) * 13 + j]; k_moduli_final adds them in
// block order, so the result does not depend on the launch.
template <typename R>
__global__ void __launch_bounds__(256) k_moduli_partial(ModArgs<R> a, double* part) {
  const int m = blockIdx.y;
  const R* eps = a.eps[m];
  const R* sig = a.sig[m];
  const long long n = a.n;
  double acc[kModSums];
#pragma unroll
  for (int j = 0; j < kModSums; ++j) acc[j] = 0.0;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const bool in = a.phase[v] != 0;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      acc[c] += (double)sig[c * n + v];
      if (in) acc[6 + c] += (double)eps[c * n + v];
    }
    if (in) acc[12] += 1.0;
  }
  __shared__ double red[kModSums][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kModSums; ++j) {
    double t = acc[j];
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    if (lane == 0) red[j][w] = t;
  }
  __syncthreads();
  if (threadIdx.x < kModSums) {
    double t = 0.0;
    for (int k = 0; k < (int)blockDim.x / 32; ++k) t += red[threadIdx.x][k];
    part[((long long)m * gridDim.x + blockIdx.x) * kModSums + threadIdx.x] = t;
  }
}

__global__ void k_moduli_final(const double* part, int nparts, double* out) {
  const int m = blockIdx.x, j = threadIdx.x;
  if (j >= kModSums) return;
  double t = 0.0;
  for (int k = 0; k < nparts; ++k) t += part[((long long)m * nparts + k) * kModSums + j];
  out[m * kModSums + j] = t;
}

template <typename R>
cudaError_t launch_moduli(const ModArgs<R>& a, int batch, double* part, double* out, cudaStream_t s) {
  k_moduli_partial<R><<<dim3(kModParts, batch), 256, 0, s>>>(a, part);
  k_moduli_final<<<batch, 32, 0, s>>>(part, kModParts, out);
  count_launches(2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- precision-ladder helpers
__global__ void k_cast_d2f(float* dst, const double* src, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}
__global__ void k_cast_f2d(double* dst, const float* src, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}
__global__ void k_add_f2d(double* dst, const float* src, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] += (double)src[i];
}
cudaError_t launch_cast_d2f(float* dst, const double* src, long long count, cudaStream_t s) {
  k_cast_d2f<<<8 * 152, 256, 0, s>>>(dst, src, count);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_cast_f2d(double* dst, const float* src, long long count, cudaStream_t s) {
  k_cast_f2d<<<8 * 152, 256, 0, s>>>(dst, src, count);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_add_f2d(double* dst, const float* src, long long count, cudaStream_t s) {
  k_add_f2d<<<8 * 152, 256, 0, s>>>(dst, src, count);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_cast_spec(C2<float>* dst, const C2<double>* src, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const C2<double> v = src[i];
    dst[i] = mk<float>((float)v.x, (float)v.y);
  }
}
cudaError_t launch_cast_spec(C2<float>* dst, const C2<double>* src, const Geo& g, int ncomp, cudaStream_t s) {
  k_cast_spec<<<8 * 152, 256, 0, s>>>(dst, src, (long long)ncomp * g.cs);
  count_launches(1);
  return cudaGetLastError();
}

// float-float spectrum -> complex64 (the FP32 phases' copy of the load)
__global__ void k_cast_spec_ff(C2<float>* dst, const C2<ff>* src, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const C2<ff> v = src[i];
    dst[i] = mk<float>((float)v.x, (float)v.y);
  }
}
cudaError_t launch_cast_spec_ff(C2<float>* dst, const C2<ff>* src, const Geo& g, int ncomp, cudaStream_t s) {
  k_cast_spec_ff<<<8 * 152, 256, 0, s>>>(dst, src, (long long)ncomp * g.cs);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void k_stress(double* sig, const double* eps, const int8_t* phase, PhaseTab<double> tab, int sx,
                         int sy, int sz, int nx, int ny, int nz) {
  const long long n = (long long)nx * ny * nz;
  const bool small = n <= 0xFFFFFFFFLL;
  // shifts reduced to [0, n) once: the per-voxel translation is then one compare
  const int sxr = ((sx % nx) + nx) % nx, syr = ((sy % ny) + ny) % ny, szr = ((sz % nz) + nz) % nz;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    lin_xyz(v, nx, ny, small, x, y, z);
    int xs = x - sxr; if (xs < 0) xs += nx;
    int ys = y - syr; if (ys < 0) ys += ny;
    int zs = z - szr; if (zs < 0) zs += nz;
    const int ph = phase[((long long)zs * ny + ys) * nx + xs];
    const double e0 = eps[v], e1 = eps[n + v], e2 = eps[2 * n + v];
    const double lt = tab.lam[ph] * (e0 + e1 + e2), m2 = 2.0 * tab.mu[ph];
    sig[v] = lt + m2 * e0;
    sig[n + v] = lt + m2 * e1;
    sig[2 * n + v] = lt + m2 * e2;
    for (int c = 3; c < 6; ++c) sig[c * n + v] = m2 * eps[c * n + v];
  }
}
cudaError_t launch_stress(double* sig, const double* eps, const int8_t* phase, const PhaseTab<double>& tab,
                          int sx, int sy, int sz, int nx, int ny, int nz, cudaStream_t s) {
  k_stress<<<8 * 152, 256, 0, s>>>(sig, eps, phase, tab, sx, sy, sz, nx, ny, nz);
  count_launches(1);
  return cudaGetLastError();
}

#define BFCS_INST(R)                                                                              \
  template cudaError_t launch_body_force<R>(R*, int, int, int, double, double, double, double,     \
                                            double*, cudaStream_t);                               \
  template cudaError_t launch_polarize<R>(R*, const R*, const int8_t*, const PhaseTab<R>&, long long,  \
                                          cudaStream_t);                                          \
  template cudaError_t launch_body_force_blocks<R>(R*, int, int, int, double, double, double,      \
                                                   double, int, double*, cudaStream_t);           \
  template cudaError_t launch_validate<R>(const int8_t*, const R*, long long, int*, double*,       \
                                          double*, cudaStream_t);                                 \
  template cudaError_t launch_bden<R>(const C2<R>*, const Geo&, ResidSlot*, IterState*,            \
                                      cudaStream_t, int, long long);                              \
  template cudaError_t launch_accumulate<R>(double*, int*, const R*, const R*, const R*,           \
                                            const int8_t*, int, int, int, int, int, int,          \
                                            cudaStream_t);                                        \
  template cudaError_t launch_moduli<R>(const ModArgs<R>&, int, double*, double*, cudaStream_t);   \
  template cudaError_t launch_radial_max<R>(const R*, int, int, int, int, const int*, int,           \
                                            unsigned long long*, unsigned long long*, cudaStream_t);
BFCS_INST(float)
BFCS_INST(double)
#undef BFCS_INST

}  // namespace bfcs
