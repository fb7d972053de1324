// Nonlocal kernel regression of Eqs. 6.5-6.6 (displacement operator, Gamma =
// -b): the operator L[u](x) = sum over offsets 0 < |xi| < delta of K(|xi|)
// (u(x + xi) - u(x)) with a radial kernel K(r) = sum_m c_m B_m(r / delta)
// (Bernstein basis of degree M) is linear in c and a periodic convolution, so
// F[L u](q) = (K_hat(q) - K_hat(0)) u_hat(q) with K_hat real (K is even).  The
// fit needs G_mn = sum_x A_m u . A_n u, g_m = sum_x A_m u . Gamma and s =
// sum_x |Gamma|^2 (A_m = L for c = e_m): by Parseval these are weighted sums
// over the stored half spectrum of products of the basis spectra W_m(q) -
// W_m(0) with |u_hat|^2, Re(u_hat . conj Gamma_hat) and |Gamma_hat|^2.  FP64.
#include "kernels.h"

namespace bfcs {

__device__ __forceinline__ double bern(int M, int m, double t) {
  double c = 1.0;                       // C(M, m)
  for (int i = 1; i <= m; ++i) c = c * (M - m + i) / i;
  double p = c;
  for (int i = 0; i < m; ++i) p *= t;
  for (int i = 0; i < M - m; ++i) p *= 1.0 - t;
  return p;
}

// minimum-image offset of voxel index i on an axis of length n
__device__ __forceinline__ int min_image(int i, int n) { return 2 * i <= n ? i : i - n; }

// w[(m - m0) * N + v] = B_m(|xi_v| / delta) for 0 < |xi_v| < delta, else 0
// (m0 <= m < m0 + nb), or, with coef != nullptr, one field sum_m coef_m B_m
__global__ void k_basis_fields(double* w, int nb, int M, int m0, NlCoef coef, double delta, int nx, int ny, int nz) {
  const int n = nx * ny * nz;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int x = min_image(v % nx, nx), y = min_image((v / nx) % ny, ny), z = min_image(v / (nx * ny), nz);
    const double d = sqrt((double)(x * x + y * y + z * z));
    const bool in = d > 0.0 && d < delta;
    const double t = d / delta;
    if (coef.use) {
      double k = 0.0;
      if (in)
        for (int m = 0; m <= M; ++m) k += coef.c[m] * bern(M, m, t);
      w[v] = k;
    } else {
      for (int j = 0; j < nb; ++j) w[(long long)j * n + v] = in ? bern(M, m0 + j, t) : 0.0;
    }
  }
}

// W[(m0 + c) * modes + i] = Re spec_c(mode i), compact mode index i = (kz ny + ky) mx + kx
__global__ void k_extract_real(const C2<double>* spec, int ncomp, Geo g, double* W, int m0) {
  const int modes = g.nz * g.ny * g.mx;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < modes; i += gridDim.x * blockDim.x) {
    const int kx = i % g.mx, r = i / g.mx;
    for (int c = 0; c < ncomp; ++c) W[(long long)(m0 + c) * modes + i] = spec[c * g.cs + (long long)r * g.p + kx].x;
  }
}

template <int NB>
__global__ void __launch_bounds__(128) k_kernel_gram(const double* W, const C2<double>* spec, Geo g, double* part) {
  constexpr int NG = NB * (NB + 1) / 2;
  constexpr int NACC = NG + NB + 1;
  __shared__ double red[4][NACC];
  double acc[NACC];
#pragma unroll
  for (int j = 0; j < NACC; ++j) acc[j] = 0.0;
  const int modes = g.nz * g.ny * g.mx;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < modes; i += gridDim.x * blockDim.x) {
    const int kx = i % g.mx, r = i / g.mx;
    const long long gi = (long long)r * g.p + kx;
    const double w = (kx == 0 || 2 * kx == g.nx) ? 1.0 : 2.0;
    double U = 0.0, X = 0.0, S = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const C2<double> u = spec[c * g.cs + gi], h = spec[(3 + c) * g.cs + gi];
      U += u.x * u.x + u.y * u.y;
      X += u.x * h.x + u.y * h.y;
      S += h.x * h.x + h.y * h.y;
    }
    double d[NB];
#pragma unroll
    for (int m = 0; m < NB; ++m) d[m] = W[(long long)m * modes + i] - W[(long long)m * modes];
    int j = 0;
#pragma unroll
    for (int a = 0; a < NB; ++a)
#pragma unroll
      for (int b = a; b < NB; ++b) acc[j++] += w * d[a] * d[b] * U;
#pragma unroll
    for (int a = 0; a < NB; ++a) acc[NG + a] += w * d[a] * X;
    acc[NG + NB] += w * S;
  }
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NACC; ++j) {
    double t = acc[j];
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    if (lane == 0) red[wp][j] = t;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < NACC; j += blockDim.x)
    part[(long long)blockIdx.x * NACC + j] = ((red[0][j] + red[1][j]) + red[2][j]) + red[3][j];
}

// acc[j] += (sum of the block partials in block order) * scale
__global__ void k_kernel_gram_final(const double* part, int nparts, int nacc, double scale, double* acc) {
  for (int j = threadIdx.x; j < nacc; j += blockDim.x) {
    double t = 0.0;
    for (int k = 0; k < nparts; ++k) t += part[(long long)k * nacc + j];
    acc[j] += t * scale;
  }
}

// Adam on J(c) = c.G.c - 2 g.c + s + lam |c|^2 from c = 0, then the exact
// minimiser of the same J (Gaussian elimination with partial pivoting of
// G + lam I).  acc holds the packed upper triangle of G, then g, then s.
// out: coef[nb], exact[nb], J(coef), J(exact), G[nb * nb], g[nb].
__global__ void k_kernel_adam(const double* acc, int nb, double lam, int iters, double lr, double b1, double b2,
                              double eps, double* out) {
  __shared__ double G[kNlMaxBasis][kNlMaxBasis], gv[kNlMaxBasis], c[kNlMaxBasis], grad[kNlMaxBasis];
  __shared__ double A[kNlMaxBasis][kNlMaxBasis + 1];
  const int t = threadIdx.x;
  if (t == 0) {
    int j = 0;
    for (int a = 0; a < nb; ++a)
      for (int b = a; b < nb; ++b) { G[a][b] = acc[j]; G[b][a] = acc[j]; ++j; }
    for (int a = 0; a < nb; ++a) gv[a] = acc[j + a];
  }
  __syncthreads();
  double m1 = 0.0, v = 0.0, p1 = 1.0, p2 = 1.0;
  if (t < nb) c[t] = 0.0;
  __syncthreads();
  for (int it = 1; it <= iters; ++it) {
    if (t < nb) {
      double s = 0.0;
      for (int b = 0; b < nb; ++b) s += G[t][b] * c[b];
      grad[t] = 2.0 * (s - gv[t] + lam * c[t]);
    }
    __syncthreads();
    if (t < nb) {
      p1 *= b1;
      p2 *= b2;
      m1 = b1 * m1 + (1.0 - b1) * grad[t];
      v = b2 * v + (1.0 - b2) * grad[t] * grad[t];
      const double mh = m1 / (1.0 - p1), vh = v / (1.0 - p2);
      c[t] = c[t] - lr * mh / (sqrt(vh) + eps);
    }
    __syncthreads();
  }
  if (t == 0) {
    const double s = acc[nb * (nb + 1) / 2 + nb];
    for (int a = 0; a < nb; ++a) {
      for (int b = 0; b < nb; ++b) A[a][b] = G[a][b] + (a == b ? lam : 0.0);
      A[a][nb] = gv[a];
    }
    for (int k = 0; k < nb; ++k) {
      int piv = k;
      for (int a = k + 1; a < nb; ++a)
        if (fabs(A[a][k]) > fabs(A[piv][k])) piv = a;
      if (piv != k)
        for (int b = k; b <= nb; ++b) { const double tmp = A[k][b]; A[k][b] = A[piv][b]; A[piv][b] = tmp; }
      for (int a = k + 1; a < nb; ++a) {
        const double f = A[k][k] != 0.0 ? A[a][k] / A[k][k] : 0.0;
        for (int b = k; b <= nb; ++b) A[a][b] -= f * A[k][b];
      }
    }
    double x[kNlMaxBasis];
    for (int a = nb - 1; a >= 0; --a) {
      double r = A[a][nb];
      for (int b = a + 1; b < nb; ++b) r -= A[a][b] * x[b];
      x[a] = A[a][a] != 0.0 ? r / A[a][a] : 0.0;
    }
    auto J = [&](const double* q) {
      double e = s;
      for (int a = 0; a < nb; ++a) {
        double gq = 0.0;
        for (int b = 0; b < nb; ++b) gq += G[a][b] * q[b];
        e += q[a] * gq - 2.0 * gv[a] * q[a] + lam * q[a] * q[a];
      }
      return e;
    };
    double cc[kNlMaxBasis];
    for (int a = 0; a < nb; ++a) { cc[a] = c[a]; out[a] = c[a]; out[nb + a] = x[a]; }
    out[2 * nb] = J(cc);
    out[2 * nb + 1] = J(x);
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b) out[2 * nb + 2 + a * nb + b] = G[a][b];
    for (int a = 0; a < nb; ++a) out[2 * nb + 2 + nb * nb + a] = gv[a];
  }
}

// spec_c(q) *= (K_hat(q) - K_hat(0)) * scale for c < ncomp; K_hat real, compact modes
__global__ void k_kernel_mult(C2<double>* spec, int ncomp, Geo g, const double* Kr, double scale) {
  const int modes = g.nz * g.ny * g.mx;
  const double k0 = Kr[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < modes; i += gridDim.x * blockDim.x) {
    const int kx = i % g.mx, r = i / g.mx;
    const double f = (Kr[i] - k0) * scale;
    for (int c = 0; c < ncomp; ++c) {
      C2<double>& z = spec[c * g.cs + (long long)r * g.p + kx];
      z.x *= f;
      z.y *= f;
    }
  }
}

cudaError_t launch_basis_fields(double* w, int nb, int M, int m0, const NlCoef& coef, double delta, const Geo& g,
                                cudaStream_t st) {
  k_basis_fields<<<8 * 152, 256, 0, st>>>(w, nb, M, m0, coef, delta, g.nx, g.ny, g.nz);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_extract_real(const C2<double>* spec, int ncomp, const Geo& g, double* W, int m0,
                                cudaStream_t st) {
  k_extract_real<<<8 * 152, 256, 0, st>>>(spec, ncomp, g, W, m0);
  count_launches(1);
  return cudaGetLastError();
}

template <int NB>
static cudaError_t gram_nb(const double* W, const C2<double>* spec, const Geo& g, double* part, double* acc,
                           cudaStream_t st) {
  constexpr int NACC = NB * (NB + 1) / 2 + NB + 1;
  k_kernel_gram<NB><<<kNlParts, 128, 0, st>>>(W, spec, g, part);
  k_kernel_gram_final<<<1, 256, 0, st>>>(part, kNlParts, NACC, 1.0 / (double)g.n, acc);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_kernel_gram(int nb, const double* W, const C2<double>* spec, const Geo& g, double* part,
                               double* acc, cudaStream_t st) {
  switch (nb) {
#define BFCS_NB(N) case N: return gram_nb<N>(W, spec, g, part, acc, st);
    BFCS_NB(1) BFCS_NB(2) BFCS_NB(3) BFCS_NB(4) BFCS_NB(5) BFCS_NB(6) BFCS_NB(7) BFCS_NB(8)
#undef BFCS_NB
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_kernel_adam(const double* acc, int nb, double lam, int iters, double lr, double* out,
                               cudaStream_t st) {
  k_kernel_adam<<<1, 32, 0, st>>>(acc, nb, lam, iters, lr, 0.9, 0.999, 1e-8, out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_kernel_mult(C2<double>* spec, int ncomp, const Geo& g, const double* Kr, double scale,
                               cudaStream_t st) {
  k_kernel_mult<<<8 * 152, 256, 0, st>>>(spec, ncomp, g, Kr, scale);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace bfcs
