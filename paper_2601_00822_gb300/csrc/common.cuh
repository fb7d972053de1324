// Shared device building blocks of the BFCS solver: complex arithmetic,
// register-resident small DFTs and the shared-memory four-step line FFT.
//
// Transform convention (Eqs. 4.3-4.5 of the paper): forward uses
// omega^{-kn} = exp(-2 pi i kn/N), inverse exp(+2 pi i kn/N); the 1/|N| of the
// inverse (Eq. 4.4) is folded into the Green-operator pass, so every transform
// here is unnormalised.  `dir` is -1 for forward, +1 for inverse.
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace bfcs {

template <typename R> struct alignas(2 * sizeof(R)) C2 { R x, y; };
// ------------------------------------------------------------------ float-float arithmetic
// A real number held as the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2: about 48 significant bits.  GB300 executes FP64
// arithmetic at a small fraction of its FP32 rate, so the FFT passes of the
// precision ladder's defect evaluation compute in this form on the FP32 pipes
// while their fields stay FP64 in memory.  Sums use the error-free TwoSum of
// Knuth (TAOCP vol. 2, 4.2.2, Theorem B) followed by Dekker's FastTwoSum
// renormalisation (Dekker 1971, "A floating-point technique for extending the
// available precision"); products take the rounding error of hi * hi from one
// fused multiply-add.  The _rn intrinsics keep the compiler from contracting
// the error terms into fused operations.
struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr ff(float f) : hi(f), lo(0.0f) {}
  __host__ __device__ constexpr ff(int i) : hi((float)i), lo(0.0f) {}   // exact for |i| < 2^24
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};
__host__ __device__ __forceinline__ ff ff_pair(float h, float l) { ff r; r.hi = h; r.lo = l; return r; }

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {   // requires |a| >= |b| (or a = 0)
  const float s = __fadd_rn(a, b);
  return ff_pair(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ ff operator+(ff a, ff b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));   // TwoSum error of hi + hi
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ff_fast_two_sum(s, e);
}
__device__ __forceinline__ ff operator-(ff a) { return ff_pair(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);               // exact rounding error of hi * hi
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff operator/(ff a, ff b) {    // two correction steps of the float quotient
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const ff r = a - b * ff(q1);
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return ff_fast_two_sum(q1, q2);
}
__device__ __forceinline__ bool operator==(ff a, ff b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(ff a, ff b) { return !(a == b); }

// FP64 <-> float-float conversions with integer bit operations (the FP64
// conversion instructions share GB300's slow FP64 pipe).  Both cover the
// normal-float range: magnitudes below 2^-126 become zero, above 2^128 infinite.
// float -> the equal double, exactly (binary32 fields widened into binary64)
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu, sgn = u & 0x80000000u;
  if (e == 0) return __hiloint2double((int)sgn, 0);
  const unsigned eh = e == 0xFFu ? 0x7FFu : e + (1023u - 127u);
  return __hiloint2double((int)(sgn | (eh << 20) | ((u & 0x7FFFFFu) >> 3)), (int)((u & 0x7u) << 29));
}
// double -> hi + lo: hi keeps the leading 24 significant bits (truncated), lo
// the next 24 of the remaining 29 (truncated): relative error below 2^-47
__device__ __forceinline__ ff d2ff_bits(double d) {
  const unsigned h32 = (unsigned)__double2hiint(d), l32 = (unsigned)__double2loint(d);
  const unsigned sgn = h32 & 0x80000000u;
  const int e = (int)((h32 >> 20) & 0x7FFu) - 1023;
  if (e < -126) return ff_pair(__uint_as_float(sgn), 0.0f);
  if (e > 127) {
    const bool nan = e == 1024 && (((h32 & 0xFFFFFu) | l32) != 0u);
    return ff_pair(__uint_as_float(nan ? 0x7FC00000u : (sgn | 0x7F800000u)), 0.0f);
  }
  const float h = __uint_as_float(sgn | ((unsigned)(e + 127) << 23) | ((h32 & 0xFFFFFu) << 3) | (l32 >> 29));
  const unsigned r = l32 & 0x1FFFFFFFu;               // weight of bit 0: 2^(e - 52)
  float l = 0.0f;
  if (r != 0u) {
    const int top = 31 - __clz((int)r);               // position of the leading one of r
    const int el = e - 52 + top;                      // exponent of lo
    if (el >= -126) {
      const unsigned mant = top >= 23 ? (r >> (top - 23)) : (r << (23 - top));
      l = __uint_as_float(sgn | ((unsigned)(el + 127) << 23) | (mant & 0x7FFFFFu));
    }
  }
  return ff_pair(h, l);
}

// Storage type of a real (non-spectral) field for arithmetic type R: the
// float-float passes read and write their real fields as FP64.
template <typename R> struct RealOf { using T = R; };
template <> struct RealOf<ff> { using T = double; };
template <typename R> __device__ __forceinline__ R ld_real(typename RealOf<R>::T v) { return R(v); }
template <typename R> __device__ __forceinline__ typename RealOf<R>::T st_real(R v) {
  return (typename RealOf<R>::T)v;
}
template <> __device__ __forceinline__ ff ld_real<ff>(double v) { return d2ff_bits(v); }
template <> __device__ __forceinline__ double st_real<ff>(ff v) { return f2d_bits(v.hi) + f2d_bits(v.lo); }
// warp shuffle of one real
template <typename R> __device__ __forceinline__ R shfl_real(R v, int src) { return __shfl_sync(0xffffffffu, v, src); }
template <> __device__ __forceinline__ ff shfl_real<ff>(ff v, int src) {
  return ff_pair(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
}


template <typename R> __host__ __device__ __forceinline__ C2<R> mk(R a, R b) { C2<R> c; c.x = a; c.y = b; return c; }
template <typename R> __device__ __forceinline__ C2<R> operator+(C2<R> a, C2<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
template <typename R> __device__ __forceinline__ C2<R> operator-(C2<R> a, C2<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
template <typename R> __device__ __forceinline__ C2<R> cmul(C2<R> a, C2<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R> __device__ __forceinline__ C2<R> conjg(C2<R> a) { return mk<R>(a.x, -a.y); }
template <typename R> __device__ __forceinline__ C2<R> scale(C2<R> a, R s) { return mk<R>(a.x * s, a.y * s); }
// multiply by dir * i, dir = +-1
template <typename R, int DIR> __device__ __forceinline__ C2<R> mul_di(C2<R> a) {
  return DIR > 0 ? mk<R>(-a.y, a.x) : mk<R>(a.y, -a.x);
}

// |z|^2 accumulated in FP64 (float-float: from the leading parts, which carry
// the 24 bits a norm needs)
template <typename R> __device__ __forceinline__ double norm2(C2<R> z) {
  return (double)z.x * (double)z.x + (double)z.y * (double)z.y;
}
template <> __device__ __forceinline__ double norm2<ff>(C2<ff> z) {
  return (double)__fmaf_rn(z.x.hi, z.x.hi, __fmul_rn(z.y.hi, z.y.hi));
}

// 1 / q rounded to nearest (FP32: the reciprocal intrinsic, without the
// general division's special-case path)
template <typename R> __device__ __forceinline__ R recip(R q) { return R(1) / q; }
template <> __device__ __forceinline__ float recip<float>(float q) { return __frcp_rn(q); }

// cos(2 pi j / 48), exact quarter-wave table extended by symmetry; every radix
// used below divides 48, so these are all the constants the register DFTs need.
__host__ __device__ constexpr double q48(int j) {
  return j == 0 ? 1.0 : j == 1 ? 0.9914448613738104 : j == 2 ? 0.9659258262890683
       : j == 3 ? 0.9238795325112867 : j == 4 ? 0.8660254037844386 : j == 5 ? 0.7933533402912352
       : j == 6 ? 0.7071067811865476 : j == 7 ? 0.6087614290087207 : j == 8 ? 0.5
       : j == 9 ? 0.3826834323650898 : j == 10 ? 0.25881904510252074 : j == 11 ? 0.1305261922200516
       : 0.0;
}
__host__ __device__ constexpr double cos48(int j) {
  return (j % 48 + 48) % 48 <= 12 ? q48((j % 48 + 48) % 48)
       : (j % 48 + 48) % 48 <= 24 ? -q48(24 - (j % 48 + 48) % 48)
       : (j % 48 + 48) % 48 <= 36 ? -q48((j % 48 + 48) % 48 - 24)
       : q48(48 - (j % 48 + 48) % 48);
}
__host__ __device__ constexpr double sin48(int j) { return cos48(j - 12); }

// ------------------------------------------------------------------ register DFTs
// X[k] = sum_n x[n] exp(DIR 2 pi i n k / RADIX), in place, natural order.
template <typename R, int RADIX, int DIR> struct Dft;

template <typename R, int DIR> struct Dft<R, 1, DIR> {
  static __device__ __forceinline__ void run(C2<R>*) {}
};
template <typename R, int DIR> struct Dft<R, 2, DIR> {
  static __device__ __forceinline__ void run(C2<R>* x) {
    C2<R> a = x[0], b = x[1];
    x[0] = a + b; x[1] = a - b;
  }
};
template <typename R, int DIR> struct Dft<R, 3, DIR> {
  static __device__ __forceinline__ void run(C2<R>* x) {
    const R h = R(0.8660254037844386);   // sin(2 pi / 3)
    C2<R> t1 = x[1] + x[2];
    C2<R> t2 = x[0] - scale(t1, R(0.5));
    C2<R> t3 = mul_di<R, DIR>(scale(x[1] - x[2], h));
    x[0] = x[0] + t1; x[1] = t2 + t3; x[2] = t2 - t3;
  }
};
template <typename R, int DIR> struct Dft<R, 4, DIR> {
  static __device__ __forceinline__ void run(C2<R>* x) {
    C2<R> a = x[0] + x[2], b = x[0] - x[2], c = x[1] + x[3];
    C2<R> d = mul_di<R, DIR>(x[1] - x[3]);
    x[0] = a + c; x[2] = a - c; x[1] = b + d; x[3] = b - d;
  }
};

// composite radix A*B by the four-step rule with constant twiddles:
// n = B n1 + n2, k = k1 + A k2
template <int RADIX> struct Split;
template <> struct Split<6> { static constexpr int A = 3, B = 2; };
template <> struct Split<8> { static constexpr int A = 4, B = 2; };
template <> struct Split<12> { static constexpr int A = 4, B = 3; };
template <> struct Split<16> { static constexpr int A = 4, B = 4; };

template <typename R, int RADIX, int DIR> struct Dft {
  static __device__ __forceinline__ void run(C2<R>* x) {
    constexpr int A = Split<RADIX>::A, B = Split<RADIX>::B;
    C2<R> u[B][A];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) {
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) u[n2][n1] = x[B * n1 + n2];
      Dft<R, A, DIR>::run(u[n2]);
#pragma unroll
      for (int k1 = 1; k1 < A; ++k1) {
        if (n2 * k1 == 0) continue;
        constexpr int S = 48 / RADIX;
        const int j = (S * n2 * k1) % 48;
        if (j % 12 == 0) {
          // exp(DIR i pi j / 24) is DIR i, -1 or -DIR i: an exact rotation (a
          // product by the constants 0 and 1 is not folded without fast math)
          const C2<R> v = u[n2][k1];
          u[n2][k1] = j == 12 ? mul_di<R, DIR>(v) : j == 24 ? mk<R>(-v.x, -v.y) : mul_di<R, -DIR>(v);
          continue;
        }
        const C2<R> w = mk<R>(R(cos48(S * n2 * k1)), R(DIR * sin48(S * n2 * k1)));
        u[n2][k1] = cmul(u[n2][k1], w);
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      C2<R> v[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) v[n2] = u[n2][k1];
      Dft<R, B, DIR>::run(v);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) x[k1 + A * k2] = v[k2];
    }
  }
};

// ------------------------------------------------------------------ line FFT factorisation
// L = R1 * R2, both register radices.  Supported lengths are the even
// 2^a 3^b up to 256 listed here.
template <int L> struct Fac;
template <> struct Fac<4> { static constexpr int R1 = 2, R2 = 2; };
template <> struct Fac<6> { static constexpr int R1 = 3, R2 = 2; };
template <> struct Fac<8> { static constexpr int R1 = 4, R2 = 2; };
template <> struct Fac<12> { static constexpr int R1 = 4, R2 = 3; };
template <> struct Fac<16> { static constexpr int R1 = 4, R2 = 4; };
template <> struct Fac<24> { static constexpr int R1 = 8, R2 = 3; };
template <> struct Fac<32> { static constexpr int R1 = 8, R2 = 4; };
template <> struct Fac<48> { static constexpr int R1 = 8, R2 = 6; };
template <> struct Fac<64> { static constexpr int R1 = 8, R2 = 8; };
template <> struct Fac<96> { static constexpr int R1 = 16, R2 = 6; };
template <> struct Fac<128> { static constexpr int R1 = 16, R2 = 8; };
template <> struct Fac<192> { static constexpr int R1 = 16, R2 = 12; };
template <> struct Fac<256> { static constexpr int R1 = 16, R2 = 16; };

template <int L> struct LineInfo {
  static constexpr int R1 = Fac<L>::R1, R2 = Fac<L>::R2;
  static constexpr int RMAX = R1 > R2 ? R1 : R2;
};

// Factored stage-1 twiddles.  With the first radix R1 (R1 % 4 == 0, R1 >= 8) a
// stage-1 thread n2 needs W^(n2 b) (b = 1..3) and W^(4 n2 a) (a = 1..R1/4-1); the
// twiddle table of a line of length L holds them after its L entries W^j, laid
// out [entry][n2] so that the threads of consecutive n2 read consecutive values
// (one 128-byte line per warp load, where the strided W^((4 n2 a) mod L) spans up
// to 12).  The values equal the entries W^((n2 b) mod L), W^((4 n2 a) mod L).
// One block per eligible radix of the line (Fac<L>::R1, then Fac<L>::R2 if it
// differs) in float and double tables.  Float-float tables, where a product costs
// more than a load, hold instead the block [k1 - 1][n2] = W^((n2 k1) mod L),
// k1 = 1..R1-1, n2 < L/R1, for R1 = Fac<L>::R1.
constexpr bool tw_factored(int r1) { return r1 % 4 == 0 && r1 >= 8; }
constexpr int tw_block(int L, int r1) { return tw_factored(r1) ? (r1 / 4 + 2) * (L / r1) : 0; }
template <int L, int R1> constexpr int tw_offset() {
  return L + (R1 == Fac<L>::R1 ? 0 : tw_block(L, Fac<L>::R1));
}

// Shared-memory four-step FFT over NCOL independent lines of length L stored
// column-wise: element n of line f at s[n * NCOL + f].  Needs at least
// NCOL * RMAX threads (one task per thread per stage so it can run in place);
// extra threads idle.  tw[j] = exp(-2 pi i j / L) (forward sign).
// Stage 1 (thread (f, n2)): DFT_R1 over n1 of x[R2 n1 + n2], twiddle W_L^{n2 k1}.
// Stage 2 (thread (f, k1)): DFT_R2 over n2, output X[k1 + R1 k2].
// Begins and ends with __syncthreads().
template <typename R, int L, int DIR>
__device__ __forceinline__ void fft_cols(C2<R>* s, int ncol, const C2<R>* __restrict__ tw) {
  constexpr int R1 = LineInfo<L>::R1, R2 = LineInfo<L>::R2;
  const int tid = threadIdx.x;
  __syncthreads();
  {
    const int f = tid % ncol, n2 = tid / ncol;
    const bool act = n2 < R2;
    C2<R> x[R1];
    if (act) {
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) x[n1] = s[(R2 * n1 + n2) * ncol + f];
      Dft<R, R1, DIR>::run(x);
#pragma unroll
      for (int k1 = 1; k1 < R1; ++k1) {
        C2<R> w = tw[(n2 * k1) % L];
        if (DIR > 0) w.y = -w.y;
        x[k1] = cmul(x[k1], w);
      }
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) s[(n2 * R1 + k1) * ncol + f] = x[k1];
    }
  }
  __syncthreads();
  {
    const int f = tid % ncol, k1 = tid / ncol;
    const bool act = k1 < R1;
    C2<R> y[R2];
    if (act) {
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) y[n2] = s[(n2 * R1 + k1) * ncol + f];
      Dft<R, R2, DIR>::run(y);
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) s[(k1 + R1 * k2) * ncol + f] = y[k2];
    }
  }
  __syncthreads();
}

// Register-staged pieces of the same four-step FFT.  A thread holding the R1
// inputs x[R2 n1 + n2] (n1 = 0..R1-1) of one line runs stage1(); after the
// exchange through shared memory a thread holding the R2 values Y[n2][k1]
// (n2 = 0..R2-1) runs stage2() and owns the outputs X[k1 + R1 k2].
// stage1f / stage2f take the factor R1 explicitly (L = R1 * (L / R1), either
// order of the two radices); stage1 / stage2 use the default order of Fac<L>.
template <typename R, int L, int R1, int DIR>
__device__ __forceinline__ void stage1f(C2<R>* x, int n2, const C2<R>* __restrict__ tw) {
  Dft<R, R1, DIR>::run(x);
  if constexpr (R1 % 4 == 0 && R1 >= 8 && sizeof(R) <= 8 && !std::is_same<R, ff>::value) {
    // W^(n2 k1) with k1 = 4 a + b as W^(4 n2 a) W^(n2 b): R1/4 - 1 + 3 table loads
    // and (R1/4 - 1) * 3 products instead of R1 - 1 loads (each product adds about
    // one rounding; float-float keeps the table, where a product costs more than a load)
    constexpr int A = R1 / 4, N2 = L / R1;
    const C2<R>* const f = tw + tw_offset<L, R1>() + n2;   // factored table, [entry][n2]
    C2<R> wb[4], wa[A];
#pragma unroll
    for (int b = 1; b < 4; ++b) wb[b] = f[(b - 1) * N2];
#pragma unroll
    for (int a = 1; a < A; ++a) wa[a] = f[(a + 2) * N2];
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) {
      const int a = k1 / 4, b = k1 % 4;
      C2<R> w = a == 0 ? wb[b] : b == 0 ? wa[a] : cmul(wa[a], wb[b]);
      if (DIR > 0) w.y = -w.y;
      x[k1] = cmul(x[k1], w);
    }
  } else if constexpr (std::is_same<R, ff>::value && R1 == Fac<L>::R1) {
    // float-float: W^((n2 k1) mod L) from the table's block [k1 - 1][n2] after its
    // L entries (consecutive threads read consecutive values; the strided look-ups
    // of 16-byte entries spanned up to 29 lines per warp load)
    constexpr int N2 = L / R1;
    const C2<R>* const f = tw + L + n2;
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) {
      C2<R> w = f[(k1 - 1) * N2];
      if (DIR > 0) w.y = -w.y;
      x[k1] = cmul(x[k1], w);
    }
  } else {
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) {
      C2<R> w = tw[(n2 * k1) % L];
      if (DIR > 0) w.y = -w.y;
      x[k1] = cmul(x[k1], w);
    }
  }
}
// Twiddle, then DFT: x[k1] *= W_L^(DIR-conjugated n2 k1), then DFT_R1 over k1.  The
// second step of an inverse (or forward) transform taken in the other order of the
// four-step rule: with k = k1 + R1 k2 and n = R2 n1 + n2, a first in-place step
// Y[k1][n2] = DFT_R2 over k2 of X[k1 + R1 k2] (rows k1 + R1 m read and written),
// then for each n2 this step on Y[k1][n2] (k1 = 0..R1-1) gives x[R2 n1 + n2].
template <typename R, int L, int R1, int DIR>
__device__ __forceinline__ void twiddle_then_dft(C2<R>* x, int n2, const C2<R>* __restrict__ tw) {
  if constexpr (R1 % 4 == 0 && R1 >= 8 && sizeof(R) <= 8 && !std::is_same<R, ff>::value) {
    constexpr int A = R1 / 4, N2 = L / R1;
    const C2<R>* const f = tw + tw_offset<L, R1>() + n2;   // factored table, [entry][n2]
    C2<R> wb[4], wa[A];
#pragma unroll
    for (int b = 1; b < 4; ++b) wb[b] = f[(b - 1) * N2];
#pragma unroll
    for (int a = 1; a < A; ++a) wa[a] = f[(a + 2) * N2];
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) {
      const int a = k1 / 4, b = k1 % 4;
      C2<R> w = a == 0 ? wb[b] : b == 0 ? wa[a] : cmul(wa[a], wb[b]);
      if (DIR > 0) w.y = -w.y;
      x[k1] = cmul(x[k1], w);
    }
  } else {
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) {
      C2<R> w = tw[(n2 * k1) % L];
      if (DIR > 0) w.y = -w.y;
      x[k1] = cmul(x[k1], w);
    }
  }
  Dft<R, R1, DIR>::run(x);
}

template <typename R, int R2, int DIR>
__device__ __forceinline__ void stage2f(C2<R>* y) {
  Dft<R, R2, DIR>::run(y);
}
template <typename R, int L, int DIR>
__device__ __forceinline__ void stage1(C2<R>* x, int n2, const C2<R>* __restrict__ tw) {
  stage1f<R, L, LineInfo<L>::R1, DIR>(x, n2, tw);
}
template <typename R, int L, int DIR>
__device__ __forceinline__ void stage2(C2<R>* y) {
  stage2f<R, LineInfo<L>::R2, DIR>(y);
}

// ------------------------------------------------------------------ async copies
// 16-byte global -> shared copy that does not pass through registers
// (cp.async, completion tracked per thread with commit/wait groups).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ------------------------------------------------------------------ problem descriptors
constexpr int kMaxPhases = 16;

template <typename R> struct PhaseTab {
  R lam[kMaxPhases], mu[kMaxPhases];     // L(x)
  R lam1[kMaxPhases], mu1[kMaxPhases];   // L1(x) = L(x) - L0
};

// Half-spectrum geometry: [comp][z][y][kx], kx in [0, nx/2], row pitch p.
struct Geo {
  int nx, ny, nz;
  int mx;           // nx/2 + 1 stored columns
  int p;            // row pitch (complex elements)
  long long cs;     // component stride of the spectrum (nz*ny*p)
  long long n;      // voxel count nx*ny*nz (component stride of real fields)
};

// Signed wavevector component of index k on an axis of length n (reading: zero
// on the Nyquist index), in units of 2 pi / n.
__device__ __forceinline__ int signed_k(int k, int n) {
  return (2 * k == n) ? 0 : (2 * k < n ? k : k - n);
}

// Residual bookkeeping written by the Green pass, reduced in FP64.
struct ResidSlot { double num; double pad; };

// Per-member descriptor of a batched solve (device memory, one per member).
// Field arrays are of the plan's real type.
struct Member {
  const int8_t* phase;    // phase ids of the untranslated microstructure
  int sx, sy, sz;         // translation chi: phase(x) = phase0(x - chi) (Eq. 3.3)
  int warm;               // 1: sweep 0 reads eps_init (its residual is not evaluated)
  double E[6];            // prescribed mean strain
  const void* b;          // 3 x N body force
  const void* eps_init;   // 6 x N or null
  void* eps_out;          // 6 x N
  void* sig_out;          // 6 x N or null
  void* u_out;            // 3 x N or null
  double tol;             // >= 0: this member's tolerance (overrides the launch's), < 0: the launch's
};

// Device-side iteration state of one solve.  Everything before resid_last is
// zeroed at the start of a solve.
struct IterState {
  int done;          // 1 once r <= tol, the iteration stalled or diverged (later sweeps are no-ops)
  int iters;         // sweeps executed
  int diverged;      // 1: NaN/Inf seen; 2: a bounded device wait of one of its passes expired
  int stalled;       // no 10% drop of the residual over the stall window
  int stall_at;      // sweep of the last stall checkpoint
  int next_check;    // sweep whose residual is evaluated next (sparse evaluation; else every sweep)
  int last_check;    // sweep of resid_last (valid once checks > 0)
  int checks;        // residual evaluations so far in this solve
  double stall_ref;  // residual at that checkpoint (0 = none yet)
  double resid_last;
  double bden;       // sqrt(sum |b_hat|^2) over modes with xi != 0
  double resid_final;
  double tau0[6];    // k = 0 mode of tau (unnormalised), current sweep
};

}  // namespace bfcs
