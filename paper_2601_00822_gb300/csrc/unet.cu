// Learned warm start / surrogate: a 3D U-net on periodic volumes, trained and
// run by the kernels in this file (BF16 activations and weights, FP32
// accumulation, FP32 master weights, gradients and Adam moments).  The paper
// motivates learned surrogates of the averaged response (Sec. 6, Eqs.
// 6.9-6.10, Fig. 5); the architecture is the project's:
//   widths 32, 32, 32, 48; two circular 3^3 convolutions per level with leaky
//   ReLU (slope 0.1); 2^3 average pooling; 2^3 stride-2 transposed
//   convolutions up (run as a 1^3 convolution to 8 C channels plus a pixel
//   shuffle); skip concatenation [upsampled, skip]; 1^3 head to the 6 strain
//   components.
//
// Activations are channels-last [b][z][y][x][c] BF16.  Convolutions are
// implicit GEMMs on the tensor cores (mma.sync m16n8k16 BF16 -> FP32):
// rows = voxels, columns = output channels, K = taps x input channels.  The
// weight gradient is a second GEMM (rows = output channels, columns = input
// channels, K = voxels) staged through shared memory with ldmatrix.trans,
// split over voxel chunks and reduced in a fixed order (deterministic).
#include "bfcs.h"
#include "kernels.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

namespace bfcs {
namespace net {

typedef __nv_bfloat16 bf16;

constexpr float kSlope = 0.1f;

struct Vol { int nx, ny, nz; };

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ unsigned ld32(const bf16* p) { return *reinterpret_cast<const unsigned*>(p); }

// fine voxel offset of sub-voxel o = 4 oz + 2 oy + ox on a grid of pitch (FX, FY)
__device__ __forceinline__ long long sub_off(int o, int FX, int FY) {
  return ((long long)(o >> 2) * FY + ((o >> 1) & 1)) * FX + (o & 1);
}

__device__ __forceinline__ void mma16816(float* c, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void ldsm_x4_trans(unsigned* r, const void* smem_row) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem_row);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// ------------------------------------------------------------------ convolution (forward / data gradient)
enum InMode : int { IN_CONV = 0, IN_GATHER_UP = 1 };
enum OutMode : int { OUT_BF16 = 0, OUT_SHUFFLE_UP = 1, OUT_F32 = 2 };

struct ConvArgs {
  const bf16* in;     // channels-last input: element (voxel, k) at in[voxel * ldi + offi + k]
  int ldi, offi;
  int cin;            // GEMM K per tap (multiple of 16)
  const bf16* w;      // [tap][cout_p][cin], K fastest
  const float* bias;  // bias[col % bias_mod], or null
  int bias_mod;
  int cout_p;         // GEMM columns (multiple of 8)
  int cout;           // columns stored (OUT_F32)
  int ksize;          // 1 or 3 (circular)
  Vol v;              // grid of the GEMM rows (coarse grid for the gather / shuffle modes)
  int batch;
  int act;            // 1: leaky ReLU
  int in_mode, out_mode;
  void* out;          // channels-last output, element (voxel, col) at out[voxel * ldo + offo + col]
  int ldo, offo;
  int up_c;           // gather / shuffle: channels per sub-voxel (multiple of 16)
};

constexpr int kConvWarps = 4;
constexpr int kConvNT = 8;   // n8 tiles per block (64 columns)

__global__ void __launch_bounds__(kConvWarps * 32) k_conv(ConvArgs a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const long long nvox = (long long)a.v.nx * a.v.ny * a.v.nz;
  const int b = blockIdx.z;
  const long long row0 = (long long)blockIdx.x * (kConvWarps * 32) + warp * 32;   // 2 m16 tiles per warp
  const int col0 = blockIdx.y * (kConvNT * 8);
  const int ntiles = min(kConvNT, (a.cout_p - col0) / 8);
  float acc[2][kConvNT][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < kConvNT; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  // fragment rows g and g + 8 of both m16 tiles (clamped; stores are guarded)
  int cx[4], cy[4], cz[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const long long r = min(row0 + (q >> 1) * 16 + (q & 1) * 8 + g, nvox - 1);
    cx[q] = (int)(r % a.v.nx);
    cy[q] = (int)((r / a.v.nx) % a.v.ny);
    cz[q] = (int)(r / ((long long)a.v.nx * a.v.ny));
  }
  const int taps = a.ksize == 3 ? 27 : 1;
  const int FX = 2 * a.v.nx, FY = 2 * a.v.ny;
  const long long in_batch = a.in_mode == IN_GATHER_UP ? nvox * 8 : nvox;
  const bf16* inb = a.in + (long long)b * in_batch * a.ldi + a.offi;
  for (int tap = 0; tap < taps; ++tap) {
    const int dz = a.ksize == 3 ? tap / 9 - 1 : 0, dy = a.ksize == 3 ? (tap / 3) % 3 - 1 : 0,
              dx = a.ksize == 3 ? tap % 3 - 1 : 0;
    const bf16* rp[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      long long vox;
      if (a.in_mode == IN_CONV)
        vox = ((long long)wrap(cz[q] + dz, a.v.nz) * a.v.ny + wrap(cy[q] + dy, a.v.ny)) * a.v.nx +
              wrap(cx[q] + dx, a.v.nx);
      else
        vox = ((long long)(2 * cz[q]) * FY + 2 * cy[q]) * FX + 2 * cx[q];
      rp[q] = inb + vox * a.ldi;
    }
    const bf16* wt = a.w + (long long)tap * a.cout_p * a.cin;
    for (int kc = 0; kc < a.cin; kc += 16) {
      long long koff = kc;
      if (a.in_mode == IN_GATHER_UP) {   // k = o * up_c + c -> fine voxel 2u + o, channel c
        const int o = kc / a.up_c;
        koff = sub_off(o, FX, FY) * a.ldi + (kc - o * a.up_c);
      }
      unsigned af[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        af[i][0] = ld32(rp[2 * i] + koff + 2 * t);
        af[i][1] = ld32(rp[2 * i + 1] + koff + 2 * t);
        af[i][2] = ld32(rp[2 * i] + koff + 2 * t + 8);
        af[i][3] = ld32(rp[2 * i + 1] + koff + 2 * t + 8);
      }
#pragma unroll
      for (int j = 0; j < kConvNT; ++j) {
        if (j < ntiles) {
          const bf16* wr = wt + (long long)(col0 + j * 8 + g) * a.cin + kc + 2 * t;
          const unsigned bfr[2] = {ld32(wr), ld32(wr + 8)};
          mma16816(acc[0][j], af[0], bfr);
          mma16816(acc[1][j], af[1], bfr);
        }
      }
    }
  }
  // epilogue: bias, activation, store
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = q >> 1, h = q & 1;
    const long long r = row0 + i * 16 + h * 8 + g;
    if (r >= nvox) continue;
#pragma unroll
    for (int j = 0; j < kConvNT; ++j) {
      if (j >= ntiles) continue;
      const int col = col0 + j * 8 + 2 * t;
      float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
      if (a.bias != nullptr) {
        v0 += a.bias[col % a.bias_mod];
        v1 += a.bias[(col + 1) % a.bias_mod];
      }
      if (a.act) {
        v0 = v0 > 0.f ? v0 : kSlope * v0;
        v1 = v1 > 0.f ? v1 : kSlope * v1;
      }
      if (a.out_mode == OUT_F32) {
        float* o = (float*)a.out + ((long long)b * nvox + r) * a.ldo + a.offo;
        if (col < a.cout) o[col] = v0;
        if (col + 1 < a.cout) o[col + 1] = v1;
      } else if (a.out_mode == OUT_BF16) {
        bf16* o = (bf16*)a.out + ((long long)b * nvox + r) * a.ldo + a.offo + col;
        *reinterpret_cast<__nv_bfloat162*>(o) = __floats2bfloat162_rn(v0, v1);
      } else {   // column o * up_c + c -> fine voxel 2u + o, channel c
        const int o = col / a.up_c, c = col - o * a.up_c;
        const long long fv = ((long long)(2 * cz[q]) * FY + 2 * cy[q]) * FX + 2 * cx[q] + sub_off(o, FX, FY);
        bf16* out = (bf16*)a.out + ((long long)b * nvox * 8 + fv) * a.ldo + a.offo + c;
        *reinterpret_cast<__nv_bfloat162*>(out) = __floats2bfloat162_rn(v0, v1);
      }
    }
  }
}

// Tiled 3^3 convolution (IN_CONV, OUT_BF16): a block computes a 16 x 8 x 2
// voxel tile for 32 output columns.  The tile's circular halo (18 x 10 x 4
// voxels, all cin channels) is staged once in shared memory with cp.async;
// A fragments come from it by ldmatrix (rows = 16 consecutive x voxels, one
// 16-byte chunk of 8 channels per row).  Chunk c of halo voxel v sits at
// chunk c ^ ((v >> sh) & (chunks - 1)): 8 consecutive voxels then hit 8
// distinct 16-byte bank groups (conflict-free ldmatrix) for cin = 16, 32, 64.
// B fragments (weights, at most 110 KB per layer) are read from L1/L2.
// Needs nx % 16 == 0, ny % 8 == 0, nz % 2 == 0, cin in {16, 32, 64}, ldi and
// offi multiples of 8.
constexpr int kTX = 16, kTY = 8, kTZ = 2;
constexpr int kHX = kTX + 2, kHY = kTY + 2, kHZ = kTZ + 2, kHalo = kHX * kHY * kHZ;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::);
}
__device__ __forceinline__ void ldsm_x4(unsigned* r, unsigned saddr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(saddr));
}

size_t conv3t_smem(int cin) { return (size_t)kHalo * cin * sizeof(bf16); }

__global__ void __launch_bounds__(128) k_conv3t(ConvArgs a) {
  extern __shared__ __align__(128) unsigned char smh[];
  const int chunks = a.cin >> 3;
  const int sh = chunks == 8 ? 0 : chunks == 4 ? 1 : 2;
  const int rowb = a.cin * 2;
  const int ntx = a.v.nx / kTX, nty = a.v.ny / kTY;
  int tb = blockIdx.x;
  const int x0 = (tb % ntx) * kTX;
  tb /= ntx;
  const int y0 = (tb % nty) * kTY, z0 = (tb / nty) * kTZ;
  const int b = blockIdx.z;
  const long long nvox = (long long)a.v.nx * a.v.ny * a.v.nz;
  const bf16* inb = a.in + (long long)b * nvox * a.ldi + a.offi;
  for (int i = threadIdx.x; i < kHalo * chunks; i += blockDim.x) {
    const int v = i / chunks, c = i - v * chunks;
    const int hx = v % kHX, hy = (v / kHX) % kHY, hz = v / (kHX * kHY);
    const int gx = wrap(x0 + hx - 1, a.v.nx), gy = wrap(y0 + hy - 1, a.v.ny), gz = wrap(z0 + hz - 1, a.v.nz);
    const bf16* src = inb + (((long long)gz * a.v.ny + gy) * a.v.nx + gx) * a.ldi + c * 8;
    cp_async16(smh + v * rowb + 16 * (c ^ ((v >> sh) & (chunks - 1))), src);
  }
  cp_async_wait_all();
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int col0 = blockIdx.y * 32;
  const int ntiles = min(4, (a.cout_p - col0) / 8);
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  int rowv[4];   // halo index of x = 0 of this warp's tile rows, plus the ldmatrix row of this lane
  const int lrow = (lane & 7) + ((lane >> 3) & 1) * 8, lk = lane >> 4;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = warp * 4 + q;
    rowv[q] = ((r / kTY + 1) * kHY + (r % kTY + 1)) * kHX + 1 + lrow;
  }
  const unsigned sbase = (unsigned)__cvta_generic_to_shared(smh);
  for (int tap = 0; tap < 27; ++tap) {
    const int doff = ((tap / 9 - 1) * kHY + ((tap / 3) % 3 - 1)) * kHX + (tap % 3 - 1);
    const bf16* wt = a.w + (long long)tap * a.cout_p * a.cin + (long long)(col0 + g) * a.cin + 2 * t;
    for (int kc = 0; kc < a.cin; kc += 16) {
      const int c = (kc >> 3) + lk;
      unsigned af[4][4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int v = rowv[q] + doff;
        ldsm_x4(af[q], sbase + v * rowb + 16 * (c ^ ((v >> sh) & (chunks - 1))));
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j < ntiles) {
          const bf16* wr = wt + (long long)j * 8 * a.cin + kc;
          const unsigned bfr[2] = {ld32(wr), ld32(wr + 8)};
#pragma unroll
          for (int q = 0; q < 4; ++q) mma16816(acc[q][j], af[q], bfr);
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = warp * 4 + q;
    const int y = y0 + r % kTY, z = z0 + r / kTY;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long vox = ((long long)z * a.v.ny + y) * a.v.nx + x0 + g + 8 * h;
      bf16* orow = (bf16*)a.out + ((long long)b * nvox + vox) * a.ldo + a.offo;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j >= ntiles) continue;
        const int col = col0 + j * 8 + 2 * t;
        float v0 = acc[q][j][2 * h], v1 = acc[q][j][2 * h + 1];
        if (a.bias != nullptr) {
          v0 += a.bias[col % a.bias_mod];
          v1 += a.bias[(col + 1) % a.bias_mod];
        }
        if (a.act) {
          v0 = v0 > 0.f ? v0 : kSlope * v0;
          v1 = v1 > 0.f ? v1 : kSlope * v1;
        }
        *reinterpret_cast<__nv_bfloat162*>(orow + col) = __floats2bfloat162_rn(v0, v1);
      }
    }
  }
}

bool conv3t_ok(const ConvArgs& a) {
  return a.ksize == 3 && a.in_mode == IN_CONV && a.out_mode == OUT_BF16 && a.v.nx % kTX == 0 &&
         a.v.ny % kTY == 0 && a.v.nz % kTZ == 0 && (a.cin == 16 || a.cin == 32 || a.cin == 64) &&
         a.ldi % 8 == 0 && a.offi % 8 == 0 && a.cout_p % 8 == 0;
}

// ------------------------------------------------------------------ tcgen05 convolution
// 3^3 circular convolution on the 5th-generation tensor cores (tcgen05.mma,
// kind::f16, BF16 operands, FP32 accumulator in tensor memory).  A persistent
// block of 4 warps keeps the layer's weights in shared memory and walks
// 128-voxel tiles (8 x-voxels x 16 y-rows x 1 z-slab).  Per tile the circular
// halo (10 x 18 x 3 voxels, all cin channels) is staged with cp.async in the
// canonical K-major no-swizzle layout: 8-channel chunk c of halo voxel v at
// byte (c * NV + v) * 16.  Eight consecutive x-voxels then form one 8 x 16 B
// core matrix, the next tile row (y + 1) sits HX voxels further (the stride
// between 8-row groups, SBO) and the next channel chunk NV voxels further
// (the stride along K, LBO) - so the A operand of every tap is the same
// descriptor at a different start address.  Weights: chunk c of output
// channel n of tap t at ((t * KC + c) * N + n) * 16 (SBO = 128 B, LBO = N * 16).
// One thread issues 27 * cin / 16 MMAs of 128 x N x 16 into the accumulator,
// tcgen05.commit arrives on an mbarrier, and the four warps read their 32
// TMEM lanes (= tile voxels) back for bias, activation and the BF16 store.
// Needs nx % 8 == 0, ny % 16 == 0, cin in {16, 32, 64}, cout_p in {32, 64},
// IN_CONV / OUT_BF16, ldi, offi, ldo, offo multiples of 8.
constexpr int kTcX = 8, kTcY = 16;
constexpr int kTcHX = kTcX + 2, kTcHY = kTcY + 2, kTcHZ = 3, kTcNV = kTcHX * kTcHY * kTcHZ;
constexpr unsigned kTcSpinLimit = 1u << 26;    // bounded wait on the MMA completion barrier

// nbuf halo buffers (each rounded to 1 KB) + weights
size_t conv3tc_smem(int cin, int n, int nbuf) {
  return nbuf * (((size_t)kTcNV * (cin / 8) * 16 + 1023) / 1024 * 1024) + (size_t)27 * (cin / 8) * n * 16;
}
// two halo buffers only where two blocks still fit on an SM (measured: two
// co-resident blocks beat one double-buffered block for the 32-channel layers)
int conv3tc_nbuf(int cin, int n) { return conv3tc_smem(cin, n, 2) <= 111 * 1024 ? 2 : 1; }

__device__ __forceinline__ uint64_t umma_sdesc(unsigned saddr, unsigned lbo, unsigned sbo) {
  // start address, leading (K) and stride (M/N) byte offsets in 16-byte units,
  // descriptor version 1 (bit 46), no swizzle, base offset 0
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 and 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ unsigned umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

// Pipelined: with two halo buffers (nbuf = 2) the halo of tile k+1 streams in
// and the epilogue of tile k-1 runs while the tensor cores work on tile k (two
// TMEM accumulators of N columns); with one buffer the next halo waits for
// the current tile's MMAs.
constexpr int kTcThreads = 256;   // 8 warps: warps w and w + 4 share TMEM lanes 32 (w % 4) .. + 31

__global__ void __launch_bounds__(kTcThreads, 2) k_conv3_tc(ConvArgs a, int* err, int nbuf) {
  extern __shared__ __align__(1024) unsigned char smt[];
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ unsigned tmem_base_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int KC = a.cin >> 3, N = a.cout_p;
  const unsigned h_stride = ((unsigned)kTcNV * KC * 16u + 1023u) & ~1023u;   // one halo buffer
  unsigned char* sw = smt + nbuf * h_stride;                                 // weights after the halos
  const unsigned sh_a = (unsigned)__cvta_generic_to_shared(smt);
  const unsigned sw_a = (unsigned)__cvta_generic_to_shared(sw);
  const unsigned mbar_a0 = (unsigned)__cvta_generic_to_shared(&mbar[0]);
  const long long nvox = (long long)a.v.nx * a.v.ny * a.v.nz;
  const int ntx = a.v.nx / kTcX, nty = a.v.ny / kTcY;
  const int tiles_ps = ntx * nty * a.v.nz;
  const int total = tiles_ps * a.batch;
  const int G = gridDim.x;
  // a network whose tensor-core wait once expired launches no more tensor-core
  // work: the flag is sticky until the context is destroyed (see the exit below)
  // (one thread reads it, so every thread of the block takes the same branch)
  if (__syncthreads_or(tid == 0 && *(volatile int*)err != 0)) return;

  if (warp == 0) {   // tensor memory: 2 accumulators of N FP32 columns x 128 lanes
    const unsigned dst = (unsigned)__cvta_generic_to_shared(&tmem_base_s);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst), "r"(2 * N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar_a0));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar_a0 + 8));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  for (int i = tid; i < 27 * N * KC; i += blockDim.x) {   // weights (core-matrix layout)
    const int c = i % KC, n = (i / KC) % N, tap = i / (KC * N);
    cp_async16(sw + ((tap * KC + c) * N + n) * 16, a.w + ((long long)tap * N + n) * a.cin + c * 8);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");

  struct TileXY { int b, x0, y0, z0; };
  auto tile_of = [&](int t) {
    TileXY r;
    r.b = t / tiles_ps;
    int tt = t - r.b * tiles_ps;
    r.x0 = (tt % ntx) * kTcX;
    tt /= ntx;
    r.y0 = (tt % nty) * kTcY;
    r.z0 = tt / nty;
    return r;
  };
  auto issue_halo = [&](int t, int buf) {
    const TileXY q = tile_of(t);
    unsigned char* sh = smt + buf * h_stride;
    const bf16* inb = a.in + (long long)q.b * nvox * a.ldi + a.offi;
    for (int i = tid; i < kTcNV * KC; i += blockDim.x) {
      const int v = i / KC, c = i - v * KC;
      const int hx = v % kTcHX, hy = (v / kTcHX) % kTcHY, hz = v / (kTcHX * kTcHY);
      const int gx = wrap(q.x0 + hx - 1, a.v.nx), gy = wrap(q.y0 + hy - 1, a.v.ny),
                gz = wrap(q.z0 + hz - 1, a.v.nz);
      cp_async16(sh + (c * kTcNV + v) * 16, inb + (((long long)gz * a.v.ny + gy) * a.v.nx + gx) * a.ldi + c * 8);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  bool ok = true;
  // bounded wait for the k-th commit on barrier k % 2 (its (k / 2)-th phase); one decision per block
  auto wait_mma = [&](int k) {
    const unsigned bar = mbar_a0 + 8u * (unsigned)(k & 1), parity = (unsigned)((k >> 1) & 1);
    unsigned done = 0, spins = 0;
    while (!done) {
      asm volatile(
          "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
          : "=r"(done)
          : "r"(bar), "r"(parity)
          : "memory");
      if (!done && ++spins > kTcSpinLimit) break;
    }
    if (__syncthreads_or(!done)) {
      if (tid == 0) atomicExch(err, 1);
      ok = false;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  };
  auto epilogue = [&](const TileXY& q, int slot) {
    const int quarter = warp & 3, half = warp >> 2;
    const int r = quarter * 32 + lane;   // TMEM lane = tile voxel (x = r % 8, y = r / 8)
    const long long vox = ((long long)q.z0 * a.v.ny + q.y0 + r / kTcX) * a.v.nx + q.x0 + r % kTcX;
    bf16* orow = (bf16*)a.out + ((long long)q.b * nvox + vox) * a.ldo + a.offo;
    for (int c0 = half * 16; c0 < N; c0 += 32) {   // this warp's 16-column slices
      unsigned v[16];
      const unsigned taddr = tmem_base_s + ((unsigned)(quarter * 32) << 16) + (unsigned)(slot * N + c0);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
      for (int q8 = 0; q8 < 16; q8 += 8) {
        __align__(16) __nv_bfloat162 o[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int col = c0 + q8 + 2 * u;
          float f0 = __uint_as_float(v[q8 + 2 * u]), f1 = __uint_as_float(v[q8 + 2 * u + 1]);
          if (a.bias != nullptr) {
            f0 += a.bias[col % a.bias_mod];
            f1 += a.bias[(col + 1) % a.bias_mod];
          }
          if (a.act) {
            f0 = f0 > 0.f ? f0 : kSlope * f0;
            f1 = f1 > 0.f ? f1 : kSlope * f1;
          }
          o[u] = __floats2bfloat162_rn(f0, f1);
        }
        *reinterpret_cast<uint4*>(orow + c0 + q8) = *reinterpret_cast<const uint4*>(o);
      }
    }
  };

  const unsigned idesc = umma_idesc_bf16(128, N);
  int t = blockIdx.x, k = 0;
  TileXY prev{};
  if (t < total) issue_halo(t, 0);
  for (; t < total && ok; t += G, ++k) {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");   // weights and halo of tile k
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const unsigned d_tmem = tmem_base_s + (unsigned)((k & 1) * N);
      // descriptors of tap 0, chunk 0; later MMAs only move the start address
      // (16-byte units in the low bits, which never carry past bit 13 here)
      const uint64_t ad0 = umma_sdesc(sh_a + (unsigned)(k % nbuf) * h_stride, kTcNV * 16, kTcHX * 16);
      const uint64_t bd0 = umma_sdesc(sw_a, N * 16, 128);
      int first = 1;
#pragma unroll 1
      for (int tap = 0; tap < 27; ++tap) {
        const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
        const unsigned aoff = (unsigned)((dz * kTcHY + dy) * kTcHX + dx);        // 16-byte units
#pragma unroll 4
        for (int kk = 0; kk < KC; kk += 2) {
          const uint64_t ad = ad0 + aoff + (unsigned)(kk * kTcNV);
          const uint64_t bd = bd0 + (unsigned)((tap * KC + kk) * N);
          asm volatile(
              "{\n.reg .pred p;\nsetp.eq.u32 p, %4, 0;\n"            // p: accumulate into D (not the first MMA)
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(first));
          first = 0;
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       mbar_a0 + 8u * (unsigned)(k & 1))
                   : "memory");
    }
    const TileXY cur = tile_of(t);
    if (k >= 1) {   // tile k-1: its MMAs are done, its accumulator is read while tile k's MMAs run
      wait_mma(k - 1);
      if (ok) epilogue(prev, (k - 1) & 1);
    }
    if (ok && t + G < total) {
      if (nbuf == 1) wait_mma(k);   // the only halo buffer is still being read by tile k's MMAs
      if (ok) issue_halo(t + G, (k + 1) % nbuf);
    }
    prev = cur;
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
  }
  if (ok && k >= 1) {
    wait_mma(k - 1);
    if (ok) epilogue(prev, (k - 1) & 1);
  }
  // After an expired wait (ok == false) the MMAs of the last commit may still be
  // in flight when the columns are released below: the contents of this CTA's
  // TMEM columns are then undefined, and so would be a later CTA's accumulator
  // placed in them.  The error flag is set before this point and is sticky, so
  // no later tensor-core launch of this network runs and bfcs_net_status
  // reports BFCS_ERR_TIMEOUT for every result from then on.
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem_base_s), "r"(2 * N));
}

bool conv3tc_ok(const ConvArgs& a) {
  return a.ksize == 3 && a.in_mode == IN_CONV && a.out_mode == OUT_BF16 && a.v.nx % kTcX == 0 &&
         a.v.ny % kTcY == 0 && (a.cin == 16 || a.cin == 32 || a.cin == 64) && (a.cout_p == 32 || a.cout_p == 64) &&
         a.ldi % 8 == 0 && a.offi % 8 == 0 && a.ldo % 8 == 0 && a.offo % 8 == 0 &&
         conv3tc_smem(a.cin, a.cout_p, 1) <= 225 * 1024;
}

// ------------------------------------------------------------------ weight gradient
// dW[tap][co][ci] = sum over (b, v) of dY[b][v][co] X[b][v + d_tap][ci]; for an
// up-convolution (up_c > 0) dW[o up_c + co][ci] = sum over (b, u) of
// dY[b][2u + o][co] X[b][u][ci] with dY read from the fine grid.
// Block (chunk, tap x mchunk): voxels [chunk * rows_per, ...), 64 output
// channels; partial[chunk][tap][cout_p][cin] in FP32.
struct WgArgs {
  const bf16* dy; int ldd, offd;   // output gradient (pre-activation)
  const bf16* x; int ldx, offx;    // layer input
  int cin, cout_p;                 // multiples of 16; cin <= 128; cout_p <= 64 or a multiple of 64
  int ksize;
  Vol v;                           // grid of the GEMM K index (coarse grid for the up mode)
  int batch;
  int up_c;
  long long chunk;                 // voxels per block (multiple of 64)
  float* part;
};

constexpr int kWgRows = 64;

__global__ void __launch_bounds__(128) k_wgrad(WgArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int mcols = min(64, a.cout_p);
  const int mchunks = a.cout_p / mcols;
  const int tap = blockIdx.y / mchunks, mc = blockIdx.y - tap * mchunks;
  const int taps = gridDim.y / mchunks;
  const int CP = mcols + 8, XP = a.cin + 8;         // row pitches: 16-byte multiples, conflict-free ldmatrix
  bf16* sD = reinterpret_cast<bf16*>(smraw);        // [64][CP]
  bf16* sX = sD + kWgRows * CP;                     // [64][XP]
  const int dz = a.ksize == 3 ? tap / 9 - 1 : 0, dy = a.ksize == 3 ? (tap / 3) % 3 - 1 : 0,
            dx = a.ksize == 3 ? tap % 3 - 1 : 0;
  const long long nvox = (long long)a.v.nx * a.v.ny * a.v.nz;
  const long long total = nvox * a.batch;
  const long long start = (long long)blockIdx.x * a.chunk;
  const long long stop = min(start + a.chunk, total);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = mcols / 16;
  const int FX = 2 * a.v.nx, FY = 2 * a.v.ny;
  float acc[4][4][4];                               // [m16 tile][n8 tile of this warp][4]
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  const int dvec = mcols / 8, xvec = a.cin / 8;
  for (long long r0 = start; r0 < stop; r0 += kWgRows) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < kWgRows * (dvec + xvec); idx += blockDim.x) {
      const int row = idx / (dvec + xvec), cv = idx - row * (dvec + xvec);
      const long long gr = r0 + row;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (gr < stop) {
        const long long b = gr / nvox;
        const long long vv = gr - b * nvox;
        const int x = (int)(vv % a.v.nx), y = (int)((vv / a.v.nx) % a.v.ny),
                  z = (int)(vv / ((long long)a.v.nx * a.v.ny));
        if (cv < dvec) {
          const int col = mc * mcols + cv * 8;
          if (a.up_c > 0) {
            const int o = col / a.up_c, c = col - o * a.up_c;
            const long long fv = ((long long)(2 * z) * FY + 2 * y) * FX + 2 * x + sub_off(o, FX, FY);
            val = *reinterpret_cast<const uint4*>(a.dy + (b * nvox * 8 + fv) * a.ldd + a.offd + c);
          } else {
            val = *reinterpret_cast<const uint4*>(a.dy + gr * a.ldd + a.offd + col);
          }
        } else {
          const long long nb = ((long long)wrap(z + dz, a.v.nz) * a.v.ny + wrap(y + dy, a.v.ny)) * a.v.nx +
                               wrap(x + dx, a.v.nx);
          val = *reinterpret_cast<const uint4*>(a.x + (b * nvox + nb) * a.ldx + a.offx + (cv - dvec) * 8);
        }
      }
      bf16* dst = cv < dvec ? sD + row * CP + cv * 8 : sX + row * XP + (cv - dvec) * 8;
      *reinterpret_cast<uint4*>(dst) = val;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kWgRows; ks += 16) {
      const int mi = lane >> 3, rr = lane & 7;
      unsigned bq[2][4];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int n0 = (warp + 4 * p) * 16;
        if (n0 < a.cin) ldsm_x4_trans(bq[p], sX + (ks + (mi & 1) * 8 + rr) * XP + n0 + (mi >> 1) * 8);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (i >= mt) continue;
        unsigned af[4];
        ldsm_x4_trans(af, sD + (ks + (mi >> 1) * 8 + rr) * CP + i * 16 + (mi & 1) * 8);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const int n0 = (warp + 4 * p) * 16;
          if (n0 < a.cin) {
            const unsigned b0[2] = {bq[p][0], bq[p][1]};
            const unsigned b1[2] = {bq[p][2], bq[p][3]};
            mma16816(acc[i][2 * p], af, b0);
            mma16816(acc[i][2 * p + 1], af, b1);
          }
        }
      }
    }
  }
  const int g = lane >> 2, t = lane & 3;
  float* out = a.part + ((long long)blockIdx.x * taps + tap) * a.cout_p * a.cin;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (i >= mt) continue;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int n0 = (warp + 4 * p) * 16 + h * 8;
        if (n0 >= a.cin) continue;
        const float* c = acc[i][2 * p + h];
        const int co = mc * mcols + i * 16 + g, ci = n0 + 2 * t;
        out[(long long)co * a.cin + ci] = c[0];
        out[(long long)co * a.cin + ci + 1] = c[1];
        out[(long long)(co + 8) * a.cin + ci] = c[2];
        out[(long long)(co + 8) * a.cin + ci + 1] = c[3];
      }
    }
  }
}

// Tiled weight gradient of a 3^3 convolution with 32 output channels:
// block (i, s) walks voxel tiles i, i + gridDim.x, ... (16 x 8 x 2 voxels of
// one sample); per tile it stages dY (256 x 32, row pitch 40 elements:
// conflict-free ldmatrix.trans) and the circular halo of X for the input
// channels [32 s, 32 s + 32) (swizzled as in k_conv3t), then warp w
// accumulates the taps 3w .. 3w + 2 in registers: dW[tap] += dY^T X_shifted,
// K = the 16 voxels of one tile row per step.  partial[i][tap][co][ci] FP32.
// Needs cout_p == 32, the tiled grid, cin in {16, 32, 64}.
constexpr int kWgtWarps = 9, kWgtDP = 40;

size_t wgrad3t_smem(int cin) {
  return (size_t)kTX * kTY * kTZ * kWgtDP * sizeof(bf16) + (size_t)kHalo * (cin < 32 ? cin : 32) * sizeof(bf16);
}

__global__ void __launch_bounds__(kWgtWarps * 32) k_wgrad3t(WgArgs a) {
  extern __shared__ __align__(128) unsigned char smw[];
  const int cs = min(a.cin, 32);
  const int c0 = blockIdx.y * cs;
  const int chunks = cs >> 3;
  const int sh = chunks == 4 ? 1 : 2;
  const int rowb = cs * 2;
  bf16* sD = reinterpret_cast<bf16*>(smw);
  unsigned char* sX = smw + kTX * kTY * kTZ * kWgtDP * sizeof(bf16);
  const unsigned sXb = (unsigned)__cvta_generic_to_shared(sX);
  const int ntx = a.v.nx / kTX, nty = a.v.ny / kTY, ntz = a.v.nz / kTZ;
  const int per_sample = ntx * nty * ntz;
  const long long nvox = (long long)a.v.nx * a.v.ny * a.v.nz;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mi = lane >> 3, rr = lane & 7;
  const int tap0 = warp * 3;
  const int np = cs / 16;     // n16 pairs
  float acc[3][2][4][4];
#pragma unroll
  for (int u = 0; u < 3; ++u)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[u][i][j][q] = 0.f;
  for (int tile = blockIdx.x; tile < per_sample * a.batch; tile += gridDim.x) {
    const int b = tile / per_sample;
    int tb = tile - b * per_sample;
    const int x0 = (tb % ntx) * kTX;
    tb /= ntx;
    const int y0 = (tb % nty) * kTY, z0 = (tb / nty) * kTZ;
    __syncthreads();   // the previous tile's shared-memory reads are done
    for (int i = threadIdx.x; i < kTX * kTY * kTZ * 4; i += blockDim.x) {
      const int v = i >> 2, c = i & 3;
      const long long vox = ((long long)(z0 + v / (kTX * kTY)) * a.v.ny + y0 + (v / kTX) % kTY) * a.v.nx + x0 + v % kTX;
      cp_async16(sD + v * kWgtDP + c * 8, a.dy + ((long long)b * nvox + vox) * a.ldd + a.offd + c * 8);
    }
    for (int i = threadIdx.x; i < kHalo * chunks; i += blockDim.x) {
      const int v = i / chunks, c = i - v * chunks;
      const int hx = v % kHX, hy = (v / kHX) % kHY, hz = v / (kHX * kHY);
      const int gx = wrap(x0 + hx - 1, a.v.nx), gy = wrap(y0 + hy - 1, a.v.ny), gz = wrap(z0 + hz - 1, a.v.nz);
      const bf16* src = a.x + ((long long)b * nvox + ((long long)gz * a.v.ny + gy) * a.v.nx + gx) * a.ldx + a.offx +
                        c0 + c * 8;
      cp_async16(sX + v * rowb + 16 * (c ^ ((v >> sh) & (chunks - 1))), src);
    }
    cp_async_wait_all();
    __syncthreads();
    if (tap0 >= 27) continue;
    for (int r = 0; r < kTY * kTZ; ++r) {
      const int yy = r % kTY, zz = r / kTY;
      unsigned af[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i)
        ldsm_x4_trans(af[i], sD + (r * kTX + (mi >> 1) * 8 + rr) * kWgtDP + i * 16 + (mi & 1) * 8);
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int tap = tap0 + u;
        const int hv0 = ((zz + 1 + tap / 9 - 1) * kHY + (yy + 1 + (tap / 3) % 3 - 1)) * kHX + 1 + (tap % 3 - 1) +
                        (mi & 1) * 8 + rr;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          if (p < np) {
            const int ch = 2 * p + (mi >> 1);
            unsigned bq[4];
            const unsigned addr = sXb + hv0 * rowb + 16 * (ch ^ ((hv0 >> sh) & (chunks - 1)));
            asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                         : "=r"(bq[0]), "=r"(bq[1]), "=r"(bq[2]), "=r"(bq[3])
                         : "r"(addr));
            const unsigned b0[2] = {bq[0], bq[1]};
            const unsigned b1[2] = {bq[2], bq[3]};
#pragma unroll
            for (int i = 0; i < 2; ++i) {
              mma16816(acc[u][i][2 * p], af[i], b0);
              mma16816(acc[u][i][2 * p + 1], af[i], b1);
            }
          }
        }
      }
    }
  }
  if (tap0 >= 27) return;
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    float* out = a.part + ((long long)blockIdx.x * 27 + tap0 + u) * 32 * a.cin + c0;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j >= 2 * np) continue;
        const int co = i * 16 + g, ci = j * 8 + 2 * t;
        out[(long long)co * a.cin + ci] = acc[u][i][j][0];
        out[(long long)co * a.cin + ci + 1] = acc[u][i][j][1];
        out[(long long)(co + 8) * a.cin + ci] = acc[u][i][j][2];
        out[(long long)(co + 8) * a.cin + ci + 1] = acc[u][i][j][3];
      }
  }
}

bool wgrad3t_ok(const WgArgs& a) {
  return a.ksize == 3 && a.up_c == 0 && a.cout_p == 32 && a.v.nx % kTX == 0 && a.v.ny % kTY == 0 &&
         a.v.nz % kTZ == 0 && (a.cin == 16 || a.cin == 32 || a.cin == 64) && a.ldd % 8 == 0 && a.offd % 8 == 0 &&
         a.ldx % 8 == 0 && a.offx % 8 == 0;
}

// out[i] = sum over c (in order) of part[c * per + i]
__global__ void k_sum_chunks(const float* part, int nchunks, long long per, float* out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < nchunks; ++c) s += part[c * per + i];
    out[i] = s;
  }
}

// ------------------------------------------------------------------ elementwise
// network input (B, 4, N) FP32 -> channels-last BF16 [B][N][16] (channels 4..15 zero)
__global__ void k_features_in(const float* x, bf16* out, long long n, int batch) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n * batch;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / n, v = i - b * n;
    __align__(16) bf16 o[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16(c < 4 ? x[(b * 4 + c) * n + v] : 0.f);
    reinterpret_cast<uint4*>(out + i * 16)[0] = reinterpret_cast<const uint4*>(o)[0];
    reinterpret_cast<uint4*>(out + i * 16)[1] = reinterpret_cast<const uint4*>(o)[1];
  }
}
// head output [B][N][6] FP32 -> (B, 6, N)
__global__ void k_features_out(const float* y, float* out, long long n, int batch) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n * batch;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / n, v = i - b * n;
#pragma unroll
    for (int c = 0; c < 6; ++c) out[(b * 6 + c) * n + v] = y[i * 6 + c];
  }
}
// 2^3 average pooling, fine -> coarse (channels-last views)
__global__ void k_pool(const bf16* in, int ldi, int offi, bf16* out, int ldo, int offo, int C, Vol coarse,
                       int batch) {
  const long long nc = (long long)coarse.nx * coarse.ny * coarse.nz;
  const int FX = 2 * coarse.nx, FY = 2 * coarse.ny;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nc * batch * C;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long r = i / C;
    const long long b = r / nc, u = r - b * nc;
    const int x = (int)(u % coarse.nx), y = (int)((u / coarse.nx) % coarse.ny),
              z = (int)(u / ((long long)coarse.nx * coarse.ny));
    const long long f0 = b * nc * 8 + ((long long)(2 * z) * FY + 2 * y) * FX + 2 * x;
    float s = 0.f;
#pragma unroll
    for (int o = 0; o < 8; ++o) s += __bfloat162float(in[(f0 + sub_off(o, FX, FY)) * ldi + offi + c]);
    out[r * ldo + offo + c] = __float2bfloat16(0.125f * s);
  }
}
// pooling gradient added into the fine gradient: dfine[2u + o][c] += dcoarse[u][c] / 8
__global__ void k_unpool_add(const bf16* dco, int ldc, int offc, bf16* dfine, int ldf, int offf, int C, Vol coarse,
                             int batch) {
  const long long nc = (long long)coarse.nx * coarse.ny * coarse.nz;
  const int FX = 2 * coarse.nx, FY = 2 * coarse.ny;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nc * batch * C * 8;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    long long r = i / C;
    const int o = (int)(r % 8);
    r /= 8;
    const long long b = r / nc, u = r - b * nc;
    const int x = (int)(u % coarse.nx), y = (int)((u / coarse.nx) % coarse.ny),
              z = (int)(u / ((long long)coarse.nx * coarse.ny));
    const long long fv = b * nc * 8 + ((long long)(2 * z) * FY + 2 * y) * FX + 2 * x + sub_off(o, FX, FY);
    bf16* d = dfine + fv * ldf + offf + c;
    *d = __float2bfloat16(__bfloat162float(*d) + 0.125f * __bfloat162float(dco[r * ldc + offc + c]));
  }
}
// dY *= act'(pre) in place; the sign of the saved post-activation output
// equals the sign of the pre-activation.  8 channels (16 bytes) per thread.
__global__ void k_act_bwd(bf16* dy, int ldd, int offd, const bf16* y, int ldy, int offy, int C, long long rows) {
  const int cv = C / 8;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < rows * cv;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / cv;
    const int c = (int)(i - r * cv) * 8;
    uint4* dp = reinterpret_cast<uint4*>(dy + r * ldd + offd + c);
    uint4 dv = *dp;
    const uint4 yv = *reinterpret_cast<const uint4*>(y + r * ldy + offy + c);
    bf16* d8 = reinterpret_cast<bf16*>(&dv);
    const bf16* y8 = reinterpret_cast<const bf16*>(&yv);
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (!(__bfloat162float(y8[k]) > 0.f)) d8[k] = __float2bfloat16(__bfloat162float(d8[k]) * kSlope);
    *dp = dv;
  }
}
// bias gradient partials: part[block][c] = sum over this block's rows of dY[r][c]
constexpr int kBiasThreads = 256;
__global__ void __launch_bounds__(kBiasThreads) k_bias_grad(const bf16* dy, int ldd, int offd, int C, long long rows,
                                                            long long per, float* part) {
  __shared__ float red[kBiasThreads];
  const int nr = kBiasThreads / C;
  const int c = threadIdx.x % C, j = threadIdx.x / C;
  const long long r0 = blockIdx.x * per, r1 = min(rows, r0 + per);
  float s = 0.f;
  if (j < nr)
    for (long long r = r0 + j; r < r1; r += nr) s += __bfloat162float(dy[r * ldd + offd + c]);
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < C) {
    float t = 0.f;
    for (int q = 0; q < nr; ++q) t += red[q * C + threadIdx.x];
    part[(long long)blockIdx.x * C + threadIdx.x] = t;
  }
}
// relative squared L2 loss: per (block, sample) sums of (p - t)^2 and t^2 in
// FP64; one voxel per thread (6 contiguous predictions, 6 coalesced targets)
constexpr int kLossBlocks = 64;
__global__ void k_loss(const float* pred, const float* target, long long n, double* num, double* den) {
  __shared__ double rn[32], rd[32];
  const int b = blockIdx.y;
  double sn = 0.0, sd = 0.0;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    const float* pr = pred + ((long long)b * n + v) * 6;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const double p = pr[c];
      const double t = target[((long long)b * 6 + c) * n + v];
      sn += (p - t) * (p - t);
      sd += t * t;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    sn += __shfl_down_sync(0xffffffffu, sn, off);
    sd += __shfl_down_sync(0xffffffffu, sd, off);
  }
  if ((threadIdx.x & 31) == 0) { rn[threadIdx.x >> 5] = sn; rd[threadIdx.x >> 5] = sd; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0;
    for (int w = 0; w < (int)blockDim.x / 32; ++w) { s0 += rn[w]; s1 += rd[w]; }
    num[b * gridDim.x + blockIdx.x] = s0;
    den[b * gridDim.x + blockIdx.x] = s1;
  }
}
// den_b[b], and loss = mean over b of num_b / den_b (written if loss != null)
__global__ void k_loss_final(const double* num, const double* den, int nblk, int batch, double* den_b, double* loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double l = 0.0;
  for (int b = 0; b < batch; ++b) {
    double s0 = 0, s1 = 0;
    for (int k = 0; k < nblk; ++k) { s0 += num[b * nblk + k]; s1 += den[b * nblk + k]; }
    den_b[b] = s1;
    l += s0 / s1;
  }
  if (loss != nullptr) *loss = l / batch;
}
// dL/dpred = 2 (p - t) / (den_b B), written as the head's output gradient
// [B][N][16] BF16 (channels 6..15 zero); one voxel per thread
__global__ void k_loss_grad(const float* pred, const float* target, const double* den_b, long long n, int batch,
                            bf16* dy) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n * batch;
       r += (long long)gridDim.x * blockDim.x) {
    const long long b = r / n, v = r - b * n;
    const double f = 2.0 / (den_b[b] * batch);
    __align__(16) bf16 o[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16(0.f);
#pragma unroll
    for (int c = 0; c < 6; ++c)
      o[c] = __float2bfloat16((float)(((double)pred[r * 6 + c] - (double)target[(b * 6 + c) * n + v]) * f));
    reinterpret_cast<uint4*>(dy + r * 16)[0] = reinterpret_cast<const uint4*>(o)[0];
    reinterpret_cast<uint4*>(dy + r * 16)[1] = reinterpret_cast<const uint4*>(o)[1];
  }
}
// Adam (Kingma and Ba 2014), bias-corrected, FP32 state
__global__ void k_adam(float* w, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// ------------------------------------------------------------------ weight layouts
// kind 0 conv3, 1 conv1, 2 up.  Forward layout [tap][cols][cin_p] with
// cols = cout_p (conv) or 8 cout (up, column o cout + co); data-gradient
// layout: conv [26 - tap][cin_p][cout_p] (flipped taps, transposed), up
// [cin_p][8 cout].  The flat vector holds PyTorch's shapes: conv
// W[co][ci][kz][ky][kx] (tap = 9 kz + 3 ky + kx), up W[ci][co][oz][oy][ox].
struct LayerDef { int kind, cin, cout, cin_p, cout_p; long long woff, boff; };

__global__ void k_pack(const float* flat, LayerDef L, bf16* fw, bf16* bw) {
  const int taps = L.kind == 0 ? 27 : 1;
  const int ocols = L.kind == 2 ? 8 * L.cout : L.cout_p;
  const long long nf = (long long)taps * ocols * L.cin_p;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += (long long)gridDim.x * blockDim.x) {
    const int ci = (int)(i % L.cin_p);
    const long long r = i / L.cin_p;
    const int col = (int)(r % ocols), tap = (int)(r / ocols);
    float w = 0.f;
    if (ci < L.cin) {
      if (L.kind == 2) {
        const int o = col / L.cout, co = col - o * L.cout;
        w = flat[L.woff + ((long long)ci * L.cout + co) * 8 + o];
      } else if (col < L.cout) {
        w = flat[L.woff + ((long long)col * L.cin + ci) * taps + tap];
      }
    }
    const bf16 wb = __float2bfloat16(w);
    fw[i] = wb;
    if (L.kind == 2) bw[(long long)ci * ocols + col] = wb;
    else bw[((long long)(taps == 27 ? 26 - tap : 0) * L.cin_p + ci) * L.cout_p + col] = wb;
  }
}

// summed weight gradient (layout of the forward weights) and bias gradient -> flat
__global__ void k_unpack_grad(const float* gw, const float* gb, LayerDef L, float* gflat) {
  const int taps = L.kind == 0 ? 27 : 1;
  const int ocols = L.kind == 2 ? 8 * L.cout : L.cout_p;
  const long long nw = (long long)taps * L.cout * L.cin * (L.kind == 2 ? 8 : 1);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nw + L.cout;
       i += (long long)gridDim.x * blockDim.x) {
    if (i >= nw) { gflat[L.boff + (i - nw)] = gb[i - nw]; continue; }
    if (L.kind == 2) {
      const int o = (int)(i % 8);
      const long long r = i / 8;
      const int co = (int)(r % L.cout), ci = (int)(r / L.cout);
      gflat[L.woff + i] = gw[(long long)(o * L.cout + co) * L.cin_p + ci];
    } else {
      const int tap = (int)(i % taps);
      const long long r = i / taps;
      const int ci = (int)(r % L.cin), co = (int)(r / L.cin);
      gflat[L.woff + i] = gw[((long long)tap * ocols + co) * L.cin_p + ci];
    }
  }
}

// ------------------------------------------------------------------ features / outputs
// max |b| over 3 N values as the bits of a non-negative float (order-independent)
template <typename R>
__global__ void k_absmax(const R* b, long long n3, unsigned* out) {
  float m = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf((float)b[i]));
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}
struct MuTab { float mu[BFCS_MAX_PHASES]; float mu_max; };
// x (4, N): b / s and mu / mu_max - 1/2; target (6, N) = eps mu_max / s (if eps)
template <typename R>
__global__ void k_prepare(const R* b, const int8_t* phase, MuTab mt, const unsigned* sbits, const R* eps, float* x,
                          float* target, long long n) {
  const float s = __uint_as_float(*sbits);
  const float inv = s > 0.f ? 1.f / s : 0.f;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c * n + v] = (float)b[c * n + v] * inv;
    x[3 * n + v] = mt.mu[phase[v]] / mt.mu_max - 0.5f;
    if (eps != nullptr) {
#pragma unroll
      for (int c = 0; c < 6; ++c) target[c * n + v] = (float)((double)eps[c * n + v] * mt.mu_max * inv);
    }
  }
}
// channels-last BF16 network input of one sample straight from b and phase
template <typename R>
__global__ void k_prepare_x0(const R* b, const int8_t* phase, MuTab mt, const unsigned* sbits, bf16* x0, long long n) {
  const float s = __uint_as_float(*sbits);
  const float inv = s > 0.f ? 1.f / s : 0.f;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    __align__(16) bf16 o[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16(0.f);
#pragma unroll
    for (int c = 0; c < 3; ++c) o[c] = __float2bfloat16((float)b[c * n + v] * inv);
    o[3] = __float2bfloat16(mt.mu[phase[v]] / mt.mu_max - 0.5f);
    reinterpret_cast<uint4*>(x0 + v * 16)[0] = reinterpret_cast<const uint4*>(o)[0];
    reinterpret_cast<uint4*>(x0 + v * 16)[1] = reinterpret_cast<const uint4*>(o)[1];
  }
}
// predicted strain (6, N) = y s / mu_max from the head output [N][6]
template <typename R>
__global__ void k_predict_out(const float* y, const unsigned* sbits, float mu_max, R* eps, long long n) {
  const double f = (double)__uint_as_float(*sbits) / mu_max;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 6; ++c) eps[c * n + v] = (R)(y[v * 6 + c] * f);
  }
}

}  // namespace net
}  // namespace bfcs

// ====================================================================== host side
using namespace bfcs::net;
using bfcs::count_launches;

namespace {

// (kind, cin, cout) in the order of the flat parameter vector
struct LayerSpec { int kind, cin, cout; };
constexpr int kNumLayers = 18;
constexpr LayerSpec kSpec[kNumLayers] = {
    {0, 4, 32},  {0, 32, 32},                 // e0a e0b
    {0, 32, 32}, {0, 32, 32},                 // e1a e1b
    {0, 32, 32}, {0, 32, 32},                 // e2a e2b
    {0, 32, 48}, {0, 48, 48},                 // e3a e3b
    {2, 48, 32}, {0, 64, 32}, {0, 32, 32},    // u2 d2a d2b
    {2, 32, 32}, {0, 64, 32}, {0, 32, 32},    // u1 d1a d1b
    {2, 32, 32}, {0, 64, 32}, {0, 32, 32},    // u0 d0a d0b
    {1, 32, 6},                               // head
};
enum { E0A, E0B, E1A, E1B, E2A, E2B, E3A, E3B, U2, D2A, D2B, U1, D1A, D1B, U0, D0A, D0B, HEAD };

long long param_count() {
  long long n = 0;
  for (const LayerSpec& s : kSpec) {
    const long long k = s.kind == 0 ? 27 : s.kind == 1 ? 1 : 8;
    n += k * s.cin * s.cout + s.cout;
  }
  return n;
}

int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
int grid_for(long long n, int threads = 256) { return std::max(1, std::min(ceil_div(n, threads), 152 * 16)); }

struct View { bf16* p; int ld, off; };

}  // namespace

struct bfcs_net_s {
  int nx, ny, nz, maxb, flags;
  cudaStream_t st;
  Vol vol[4];
  long long n[4];
  LayerDef def[kNumLayers];
  bf16* fw[kNumLayers];
  bf16* bw[kNumLayers];
  float* gw[kNumLayers];     // summed weight gradients (forward layout)
  float* gb[kNumLayers];
  char* base = nullptr;
  // activations
  bf16 *X0, *A0, *C0, *D0a, *D0b, *P0, *A1, *C1, *D1a, *D1b, *P1, *A2, *C2, *D2a, *D2b, *P2, *A3, *H3;
  float* OUT;
  // gradients (training only)
  bf16 *dOUT = nullptr, *dA0, *dC0, *dD0a, *dD0b, *dP0, *dA1, *dC1, *dD1a, *dD1b, *dP1, *dA2, *dC2, *dD2a, *dD2b,
       *dP2, *dA3, *dH3;
  float* part = nullptr;     // weight / bias gradient partials
  long long part_cap = 0;
  double* lnum;              // loss partials
  double* lden;
  double* den_b;
  unsigned* sbits;           // per-sample max |b|
  int* err;                  // set by a kernel whose bounded wait expired
};

namespace {

cudaError_t pack_all(bfcs_net_s* N, const float* params) {
  for (int l = 0; l < kNumLayers; ++l) {
    const LayerDef& L = N->def[l];
    const long long nf = (long long)(L.kind == 0 ? 27 : 1) * (L.kind == 2 ? 8 * L.cout : L.cout_p) * L.cin_p;
    k_pack<<<grid_for(nf), 256, 0, N->st>>>(params, L, N->fw[l], N->bw[l]);
  }
  count_launches(kNumLayers);
  return cudaGetLastError();
}

// forward GEMM of layer l: in -> out on the grid of level lv (coarse level for an up layer)
int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || n < 1)
      n = 1;
  }
  return n;
}

// BFCS_NET_TCGEN05=0 keeps the convolutions on the mma.sync kernels
bool tcgen05_enabled() {
  const char* e = std::getenv("BFCS_NET_TCGEN05");
  return !(e != nullptr && std::atoi(e) == 0);
}

cudaError_t launch_conv(const ConvArgs& a, long long nvox, int* err, cudaStream_t st) {
  if (tcgen05_enabled() && conv3tc_ok(a)) {
    const long long tiles = (long long)(a.v.nx / kTcX) * (a.v.ny / kTcY) * a.v.nz * a.batch;
    const int nbuf = conv3tc_nbuf(a.cin, a.cout_p);
    const size_t smem = conv3tc_smem(a.cin, a.cout_p, nbuf);
    const int per_sm = std::max(1, std::min(2, (int)((227 * 1024) / (smem + 2048))));
    const int blocks = (int)std::min<long long>(tiles, (long long)sm_count() * per_sm);
    k_conv3_tc<<<blocks, kTcThreads, smem, st>>>(a, err, nbuf);
  } else if (conv3t_ok(a)) {
    const int tiles = (a.v.nx / kTX) * (a.v.ny / kTY) * (a.v.nz / kTZ);
    k_conv3t<<<dim3(tiles, ceil_div(a.cout_p, 32), a.batch), 128, conv3t_smem(a.cin), st>>>(a);
  } else {
    k_conv<<<dim3(ceil_div(nvox, kConvWarps * 32), ceil_div(a.cout_p, kConvNT * 8), a.batch), kConvWarps * 32, 0,
             st>>>(a);
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t conv_fwd(bfcs_net_s* N, int l, const float* params, int B, View in, int lv, int out_mode, void* out,
                     int ldo, int offo) {
  const LayerDef& L = N->def[l];
  ConvArgs a{};
  a.in = in.p; a.ldi = in.ld; a.offi = in.off;
  a.cin = L.cin_p;
  a.w = N->fw[l];
  a.bias = params + L.boff;
  a.bias_mod = L.cout;
  a.cout_p = L.kind == 2 ? 8 * L.cout : L.cout_p;
  a.cout = L.kind == 1 ? L.cout : a.cout_p;
  a.ksize = L.kind == 0 ? 3 : 1;
  a.v = N->vol[lv];
  a.batch = B;
  a.act = L.kind == 0 ? 1 : 0;
  a.in_mode = IN_CONV;
  a.out_mode = out_mode;
  a.out = out; a.ldo = ldo; a.offo = offo;
  a.up_c = L.cout;
  return launch_conv(a, N->n[lv], N->err, N->st);
}

cudaError_t pool(bfcs_net_s* N, View in, View out, int C, int coarse_lv, int B) {
  const long long tot = N->n[coarse_lv] * B * C;
  k_pool<<<grid_for(tot), 256, 0, N->st>>>(in.p, in.ld, in.off, out.p, out.ld, out.off, C, N->vol[coarse_lv], B);
  count_launches(1);
  return cudaGetLastError();
}

#define NET_TRY(x) \
  if ((e = (x)) != cudaSuccess) return e

cudaError_t forward(bfcs_net_s* N, const float* params, int B) {
  cudaError_t e;
  const int F = OUT_BF16;
  NET_TRY(conv_fwd(N, E0A, params, B, {N->X0, 16, 0}, 0, F, N->A0, 32, 0));
  NET_TRY(conv_fwd(N, E0B, params, B, {N->A0, 32, 0}, 0, F, N->C0, 64, 32));
  NET_TRY(pool(N, {N->C0, 64, 32}, {N->P0, 32, 0}, 32, 1, B));
  NET_TRY(conv_fwd(N, E1A, params, B, {N->P0, 32, 0}, 1, F, N->A1, 32, 0));
  NET_TRY(conv_fwd(N, E1B, params, B, {N->A1, 32, 0}, 1, F, N->C1, 64, 32));
  NET_TRY(pool(N, {N->C1, 64, 32}, {N->P1, 32, 0}, 32, 2, B));
  NET_TRY(conv_fwd(N, E2A, params, B, {N->P1, 32, 0}, 2, F, N->A2, 32, 0));
  NET_TRY(conv_fwd(N, E2B, params, B, {N->A2, 32, 0}, 2, F, N->C2, 64, 32));
  NET_TRY(pool(N, {N->C2, 64, 32}, {N->P2, 32, 0}, 32, 3, B));
  NET_TRY(conv_fwd(N, E3A, params, B, {N->P2, 32, 0}, 3, F, N->A3, 48, 0));
  NET_TRY(conv_fwd(N, E3B, params, B, {N->A3, 48, 0}, 3, F, N->H3, 48, 0));
  NET_TRY(conv_fwd(N, U2, params, B, {N->H3, 48, 0}, 3, OUT_SHUFFLE_UP, N->C2, 64, 0));
  NET_TRY(conv_fwd(N, D2A, params, B, {N->C2, 64, 0}, 2, F, N->D2a, 32, 0));
  NET_TRY(conv_fwd(N, D2B, params, B, {N->D2a, 32, 0}, 2, F, N->D2b, 32, 0));
  NET_TRY(conv_fwd(N, U1, params, B, {N->D2b, 32, 0}, 2, OUT_SHUFFLE_UP, N->C1, 64, 0));
  NET_TRY(conv_fwd(N, D1A, params, B, {N->C1, 64, 0}, 1, F, N->D1a, 32, 0));
  NET_TRY(conv_fwd(N, D1B, params, B, {N->D1a, 32, 0}, 1, F, N->D1b, 32, 0));
  NET_TRY(conv_fwd(N, U0, params, B, {N->D1b, 32, 0}, 1, OUT_SHUFFLE_UP, N->C0, 64, 0));
  NET_TRY(conv_fwd(N, D0A, params, B, {N->C0, 64, 0}, 0, F, N->D0a, 32, 0));
  NET_TRY(conv_fwd(N, D0B, params, B, {N->D0a, 32, 0}, 0, F, N->D0b, 32, 0));
  NET_TRY(conv_fwd(N, HEAD, params, B, {N->D0b, 32, 0}, 0, OUT_F32, N->OUT, 6, 0));
  return cudaSuccess;
}

// Backward of layer l.  dout: gradient w.r.t. the layer output (post-activation;
// turned into the pre-activation gradient in place); out: saved output; in:
// saved input; din: where the input gradient goes (p == null: not needed).
// lv: level of the GEMM rows (coarse level for an up layer).
cudaError_t layer_bwd(bfcs_net_s* N, int l, int B, View dout, View out, View in, View din, int lv) {
  const LayerDef& L = N->def[l];
  const bool up = L.kind == 2;
  const int taps = L.kind == 0 ? 27 : 1;
  const long long rows = N->n[lv] * B;                  // GEMM K rows of the weight gradient
  const long long orows = up ? rows * 8 : rows;         // rows of the output gradient
  const int dch = up ? L.cout : L.cout_p;               // channels of the output gradient view
  if (L.kind == 0) {
    k_act_bwd<<<grid_for(orows * dch / 8), 256, 0, N->st>>>(dout.p, dout.ld, dout.off, out.p, out.ld, out.off, dch,
                                                            orows);
    count_launches(1);
  }
  // weight gradient
  WgArgs w{};
  w.dy = dout.p; w.ldd = dout.ld; w.offd = dout.off;
  w.x = in.p; w.ldx = in.ld; w.offx = in.off;
  w.cin = L.cin_p;
  w.cout_p = up ? 8 * L.cout : L.cout_p;
  w.ksize = L.kind == 0 ? 3 : 1;
  w.v = N->vol[lv];
  w.batch = B;
  w.up_c = up ? L.cout : 0;
  const int mchunks = w.cout_p > 64 ? w.cout_p / 64 : 1;
  const int want = 152 * 8;
  int nchunks = std::max(1, std::min(ceil_div(want, taps * mchunks), ceil_div(rows, kWgRows)));
  w.chunk = (long long)ceil_div(ceil_div(rows, nchunks), kWgRows) * kWgRows;
  nchunks = ceil_div(rows, w.chunk);
  const long long per = (long long)taps * w.cout_p * w.cin;
  const int bc = dch;
  const int nblk = std::max(1, std::min(1024, ceil_div(orows, 512)));
  if ((long long)nchunks * per + (long long)nblk * bc > N->part_cap) return cudaErrorInvalidValue;
  w.part = N->part;
  if (wgrad3t_ok(w)) {
    const long long tiles = (long long)(w.v.nx / kTX) * (w.v.ny / kTY) * (w.v.nz / kTZ) * B;
    nchunks = (int)std::min<long long>(tiles, 152);
    if ((long long)nchunks * per + (long long)nblk * bc > N->part_cap) return cudaErrorInvalidValue;
    k_wgrad3t<<<dim3(nchunks, w.cin > 32 ? w.cin / 32 : 1), kWgtWarps * 32, wgrad3t_smem(w.cin), N->st>>>(w);
  } else {
    const int mcols = std::min(64, w.cout_p);
    const size_t smem = (size_t)kWgRows * (mcols + 8 + w.cin + 8) * sizeof(bf16);
    k_wgrad<<<dim3(nchunks, taps * mchunks), 128, smem, N->st>>>(w);
  }
  k_sum_chunks<<<grid_for(per), 256, 0, N->st>>>(N->part, nchunks, per, N->gw[l]);
  // bias gradient (over the rows of the output gradient)
  const long long bper = (orows + nblk - 1) / nblk;
  float* bpart = N->part + (long long)nchunks * per;
  k_bias_grad<<<nblk, kBiasThreads, 0, N->st>>>(dout.p, dout.ld, dout.off, bc, orows, bper, bpart);
  k_sum_chunks<<<grid_for(bc), 256, 0, N->st>>>(bpart, nblk, bc, N->gb[l]);
  count_launches(4);
  // input gradient: a convolution with the data-gradient weights
  if (din.p != nullptr) {
    ConvArgs a{};
    a.in = dout.p; a.ldi = dout.ld; a.offi = dout.off;
    a.cin = up ? 8 * L.cout : L.cout_p;
    a.w = N->bw[l];
    a.bias = nullptr; a.bias_mod = 1;
    a.cout_p = L.cin_p; a.cout = L.cin_p;
    a.ksize = L.kind == 0 ? 3 : 1;
    a.v = N->vol[lv];
    a.batch = B;
    a.act = 0;
    a.in_mode = up ? IN_GATHER_UP : IN_CONV;
    a.out_mode = OUT_BF16;
    a.out = din.p; a.ldo = din.ld; a.offo = din.off;
    a.up_c = L.cout;
    const cudaError_t e = launch_conv(a, N->n[lv], N->err, N->st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t unpool_add(bfcs_net_s* N, View dco, View dfine, int C, int coarse_lv, int B) {
  const long long tot = N->n[coarse_lv] * B * C * 8;
  k_unpool_add<<<grid_for(tot), 256, 0, N->st>>>(dco.p, dco.ld, dco.off, dfine.p, dfine.ld, dfine.off, C,
                                                 N->vol[coarse_lv], B);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t backward(bfcs_net_s* N, int B) {
  cudaError_t e;
  const View none{nullptr, 0, 0};
  NET_TRY(layer_bwd(N, HEAD, B, {N->dOUT, 16, 0}, none, {N->D0b, 32, 0}, {N->dD0b, 32, 0}, 0));
  NET_TRY(layer_bwd(N, D0B, B, {N->dD0b, 32, 0}, {N->D0b, 32, 0}, {N->D0a, 32, 0}, {N->dD0a, 32, 0}, 0));
  NET_TRY(layer_bwd(N, D0A, B, {N->dD0a, 32, 0}, {N->D0a, 32, 0}, {N->C0, 64, 0}, {N->dC0, 64, 0}, 0));
  NET_TRY(layer_bwd(N, U0, B, {N->dC0, 64, 0}, none, {N->D1b, 32, 0}, {N->dD1b, 32, 0}, 1));
  NET_TRY(layer_bwd(N, D1B, B, {N->dD1b, 32, 0}, {N->D1b, 32, 0}, {N->D1a, 32, 0}, {N->dD1a, 32, 0}, 1));
  NET_TRY(layer_bwd(N, D1A, B, {N->dD1a, 32, 0}, {N->D1a, 32, 0}, {N->C1, 64, 0}, {N->dC1, 64, 0}, 1));
  NET_TRY(layer_bwd(N, U1, B, {N->dC1, 64, 0}, none, {N->D2b, 32, 0}, {N->dD2b, 32, 0}, 2));
  NET_TRY(layer_bwd(N, D2B, B, {N->dD2b, 32, 0}, {N->D2b, 32, 0}, {N->D2a, 32, 0}, {N->dD2a, 32, 0}, 2));
  NET_TRY(layer_bwd(N, D2A, B, {N->dD2a, 32, 0}, {N->D2a, 32, 0}, {N->C2, 64, 0}, {N->dC2, 64, 0}, 2));
  NET_TRY(layer_bwd(N, U2, B, {N->dC2, 64, 0}, none, {N->H3, 48, 0}, {N->dH3, 48, 0}, 3));
  NET_TRY(layer_bwd(N, E3B, B, {N->dH3, 48, 0}, {N->H3, 48, 0}, {N->A3, 48, 0}, {N->dA3, 48, 0}, 3));
  NET_TRY(layer_bwd(N, E3A, B, {N->dA3, 48, 0}, {N->A3, 48, 0}, {N->P2, 32, 0}, {N->dP2, 32, 0}, 3));
  NET_TRY(unpool_add(N, {N->dP2, 32, 0}, {N->dC2, 64, 32}, 32, 3, B));
  NET_TRY(layer_bwd(N, E2B, B, {N->dC2, 64, 32}, {N->C2, 64, 32}, {N->A2, 32, 0}, {N->dA2, 32, 0}, 2));
  NET_TRY(layer_bwd(N, E2A, B, {N->dA2, 32, 0}, {N->A2, 32, 0}, {N->P1, 32, 0}, {N->dP1, 32, 0}, 2));
  NET_TRY(unpool_add(N, {N->dP1, 32, 0}, {N->dC1, 64, 32}, 32, 2, B));
  NET_TRY(layer_bwd(N, E1B, B, {N->dC1, 64, 32}, {N->C1, 64, 32}, {N->A1, 32, 0}, {N->dA1, 32, 0}, 1));
  NET_TRY(layer_bwd(N, E1A, B, {N->dA1, 32, 0}, {N->A1, 32, 0}, {N->P0, 32, 0}, {N->dP0, 32, 0}, 1));
  NET_TRY(unpool_add(N, {N->dP0, 32, 0}, {N->dC0, 64, 32}, 32, 1, B));
  NET_TRY(layer_bwd(N, E0B, B, {N->dC0, 64, 32}, {N->C0, 64, 32}, {N->A0, 32, 0}, {N->dA0, 32, 0}, 0));
  NET_TRY(layer_bwd(N, E0A, B, {N->dA0, 32, 0}, {N->A0, 32, 0}, {N->X0, 16, 0}, none, 0));
  return cudaSuccess;
}

cudaError_t loss_and_grad(bfcs_net_s* N, int B, const float* target, double* loss_dev) {
  k_loss<<<dim3(kLossBlocks, B), 256, 0, N->st>>>(N->OUT, target, N->n[0], N->lnum, N->lden);
  k_loss_final<<<1, 32, 0, N->st>>>(N->lnum, N->lden, kLossBlocks, B, N->den_b, loss_dev);
  k_loss_grad<<<grid_for(N->n[0] * B), 256, 0, N->st>>>(N->OUT, target, N->den_b, N->n[0], B, N->dOUT);
  count_launches(3);
  return cudaGetLastError();
}

cudaError_t grads_to_flat(bfcs_net_s* N, float* grad) {
  for (int l = 0; l < kNumLayers; ++l) {
    const LayerDef& L = N->def[l];
    const long long nw = (long long)(L.kind == 0 ? 27 : 1) * L.cout * L.cin * (L.kind == 2 ? 8 : 1) + L.cout;
    k_unpack_grad<<<grid_for(nw), 256, 0, N->st>>>(N->gw[l], N->gb[l], L, grad);
  }
  count_launches(kNumLayers);
  return cudaGetLastError();
}

int status_of(cudaError_t e) { return e == cudaSuccess ? BFCS_OK : BFCS_ERR_CUDA; }

void free_net(bfcs_net_s* N) {
  if (N->base) cudaFree(N->base);
  delete N;
}

float mu_table(int nphases, const bfcs_lame* phases, MuTab* mt) {
  float mx = 0.f;
  for (int p = 0; p < BFCS_MAX_PHASES; ++p) mt->mu[p] = 0.f;
  for (int p = 0; p < nphases; ++p) {
    mt->mu[p] = (float)phases[p].mu;
    mx = std::max(mx, mt->mu[p]);
  }
  mt->mu_max = mx;
  return mx;
}

bool valid_phases(int nphases, const bfcs_lame* phases) {
  if (nphases < 1 || nphases > BFCS_MAX_PHASES || phases == nullptr) return false;
  for (int p = 0; p < nphases; ++p)
    if (!(phases[p].mu > 0.0) || !std::isfinite(phases[p].mu)) return false;
  return true;
}

}  // namespace

extern "C" {

long long bfcs_net_param_count(void) { return param_count(); }

int bfcs_net_create(bfcs_net* out, int nx, int ny, int nz, int max_batch, int flags, void* stream) {
  if (out == nullptr) return BFCS_ERR_INVALID_ARG;
  *out = nullptr;
  if (nx < 8 || ny < 8 || nz < 8 || nx % 8 || ny % 8 || nz % 8 || max_batch < 1 || max_batch > 1024 ||
      (flags & ~BFCS_NET_TRAIN) != 0)
    return BFCS_ERR_INVALID_ARG;
  if ((long long)nx * ny * nz * max_batch > (1LL << 31)) return BFCS_ERR_INVALID_ARG;
  bfcs_net_s* N = new (std::nothrow) bfcs_net_s();
  if (N == nullptr) return BFCS_ERR_OOM;
  N->nx = nx; N->ny = ny; N->nz = nz; N->maxb = max_batch; N->flags = flags;
  N->st = (cudaStream_t)stream;
  for (int l = 0; l < 4; ++l) {
    N->vol[l] = {nx >> l, ny >> l, nz >> l};
    N->n[l] = (long long)(nx >> l) * (ny >> l) * (nz >> l);
  }
  long long off = 0;
  for (int l = 0; l < kNumLayers; ++l) {
    const LayerSpec& s = kSpec[l];
    LayerDef& L = N->def[l];
    L.kind = s.kind; L.cin = s.cin; L.cout = s.cout;
    L.cin_p = (s.cin + 15) / 16 * 16;
    L.cout_p = s.kind == 1 ? (s.cout + 15) / 16 * 16 : s.cout;
    L.woff = off;
    off += (long long)(s.kind == 0 ? 27 : s.kind == 1 ? 1 : 8) * s.cin * s.cout;
    L.boff = off;
    off += s.cout;
  }
  // one allocation, carved in 256-byte aligned pieces
  const long long B = max_batch;
  const bool train = (flags & BFCS_NET_TRAIN) != 0;
  std::vector<std::pair<void**, size_t>> req;
  auto add = [&](void* p, size_t bytes) { req.push_back({(void**)p, bytes}); };
  const long long* n = N->n;
  auto act = [&](bf16** p, int lv, int C) { add(p, (size_t)(B * n[lv] * C) * sizeof(bf16)); };
  act(&N->X0, 0, 16); act(&N->A0, 0, 32); act(&N->C0, 0, 64); act(&N->D0a, 0, 32); act(&N->D0b, 0, 32);
  act(&N->P0, 1, 32); act(&N->A1, 1, 32); act(&N->C1, 1, 64); act(&N->D1a, 1, 32); act(&N->D1b, 1, 32);
  act(&N->P1, 2, 32); act(&N->A2, 2, 32); act(&N->C2, 2, 64); act(&N->D2a, 2, 32); act(&N->D2b, 2, 32);
  act(&N->P2, 3, 32); act(&N->A3, 3, 48); act(&N->H3, 3, 48);
  add(&N->OUT, (size_t)(B * n[0] * 6) * sizeof(float));
  for (int l = 0; l < kNumLayers; ++l) {
    const LayerDef& L = N->def[l];
    const size_t nw = (size_t)(L.kind == 0 ? 27 : 1) * (L.kind == 2 ? 8 * L.cout : L.cout_p) * L.cin_p;
    add(&N->fw[l], nw * sizeof(bf16));
    add(&N->bw[l], nw * sizeof(bf16));
    N->gw[l] = nullptr;
    N->gb[l] = nullptr;
    if (train) {
      add(&N->gw[l], nw * sizeof(float));
      add(&N->gb[l], (size_t)L.cout * sizeof(float));
    }
  }
  add(&N->lnum, (size_t)kLossBlocks * B * sizeof(double));
  add(&N->lden, (size_t)kLossBlocks * B * sizeof(double));
  add(&N->den_b, (size_t)B * sizeof(double));
  add(&N->sbits, (size_t)B * sizeof(unsigned));
  add(&N->err, sizeof(int));
  if (train) {
    act(&N->dOUT, 0, 16); act(&N->dA0, 0, 32); act(&N->dC0, 0, 64); act(&N->dD0a, 0, 32); act(&N->dD0b, 0, 32);
    act(&N->dP0, 1, 32); act(&N->dA1, 1, 32); act(&N->dC1, 1, 64); act(&N->dD1a, 1, 32); act(&N->dD1b, 1, 32);
    act(&N->dP1, 2, 32); act(&N->dA2, 2, 32); act(&N->dC2, 2, 64); act(&N->dD2a, 2, 32); act(&N->dD2b, 2, 32);
    act(&N->dP2, 3, 32); act(&N->dA3, 3, 48); act(&N->dH3, 3, 48);
    // weight-gradient partials: at most 152*8 blocks' worth of one layer's weights, plus bias partials
    N->part_cap = 0;
    for (int l = 0; l < kNumLayers; ++l) {
      const LayerDef& L = N->def[l];
      const long long taps = L.kind == 0 ? 27 : 1;
      const long long per = taps * (L.kind == 2 ? 8 * L.cout : L.cout_p) * L.cin_p;
      const long long mch = L.kind == 2 ? 8 * L.cout / 64 : 1;
      const long long nch = std::max<long long>(1, ceil_div(152 * 8, taps * mch));
      N->part_cap = std::max(N->part_cap, std::max(nch, 152LL) * per + 1024LL * 64);
    }
    add(&N->part, (size_t)N->part_cap * sizeof(float));
  }
  size_t total = 0;
  for (auto& r : req) total += (r.second + 255) / 256 * 256;
  if (cudaMalloc((void**)&N->base, total) != cudaSuccess) {
    cudaGetLastError();
    delete N;
    return BFCS_ERR_OOM;
  }
  size_t pos = 0;
  for (auto& r : req) {
    *r.first = N->base + pos;
    pos += (r.second + 255) / 256 * 256;
  }
  if (cudaFuncSetAttribute(k_conv3t, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv3t_smem(64)) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_conv3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024) != cudaSuccess ||
      cudaFuncSetAttribute(k_wgrad3t, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wgrad3t_smem(64)) !=
          cudaSuccess) {
    cudaGetLastError();
    free_net(N);
    return BFCS_ERR_CUDA;
  }
  // zero everything once: padded input channels stay zero
  if (cudaMemsetAsync(N->base, 0, total, N->st) != cudaSuccess) { free_net(N); return BFCS_ERR_CUDA; }
  *out = N;
  return BFCS_OK;
}

int bfcs_net_status(bfcs_net N) {
  if (N == nullptr) return BFCS_ERR_INVALID_ARG;
  int h = 0;
  if (cudaMemcpyAsync(&h, N->err, sizeof(int), cudaMemcpyDeviceToHost, N->st) != cudaSuccess ||
      cudaStreamSynchronize(N->st) != cudaSuccess)
    return BFCS_ERR_CUDA;
  return h ? BFCS_ERR_TIMEOUT : BFCS_OK;
}

int bfcs_net_destroy(bfcs_net N) {
  if (N == nullptr) return BFCS_ERR_INVALID_ARG;
  cudaStreamSynchronize(N->st);
  free_net(N);
  return BFCS_OK;
}

int bfcs_net_prepare(bfcs_net N, int precision, const void* b, const int8_t* phase, int nphases,
                     const bfcs_lame* phases, const void* eps, float* x_out, float* target_out) {
  if (N == nullptr || b == nullptr || phase == nullptr || x_out == nullptr || (eps != nullptr && target_out == nullptr) ||
      (precision != BFCS_FP32 && precision != BFCS_FP64) || !valid_phases(nphases, phases))
    return BFCS_ERR_INVALID_ARG;
  MuTab mt;
  mu_table(nphases, phases, &mt);
  const long long n = N->n[0];
  cudaMemsetAsync(N->sbits, 0, sizeof(unsigned), N->st);
  if (precision == BFCS_FP64) {
    k_absmax<double><<<grid_for(3 * n), 256, 0, N->st>>>((const double*)b, 3 * n, N->sbits);
    k_prepare<double><<<grid_for(n), 256, 0, N->st>>>((const double*)b, phase, mt, N->sbits, (const double*)eps, x_out,
                                                      target_out, n);
  } else {
    k_absmax<float><<<grid_for(3 * n), 256, 0, N->st>>>((const float*)b, 3 * n, N->sbits);
    k_prepare<float><<<grid_for(n), 256, 0, N->st>>>((const float*)b, phase, mt, N->sbits, (const float*)eps, x_out,
                                                     target_out, n);
  }
  count_launches(2);
  return status_of(cudaGetLastError());
}

int bfcs_net_forward(bfcs_net N, const float* params, int batch, const float* x, float* y) {
  if (N == nullptr || params == nullptr || x == nullptr || y == nullptr || batch < 1 || batch > N->maxb)
    return BFCS_ERR_INVALID_ARG;
  cudaError_t e = pack_all(N, params);
  if (e == cudaSuccess) {
    k_features_in<<<grid_for(N->n[0] * batch), 256, 0, N->st>>>(x, N->X0, N->n[0], batch);
    count_launches(1);
    e = forward(N, params, batch);
  }
  if (e == cudaSuccess) {
    k_features_out<<<grid_for(N->n[0] * batch), 256, 0, N->st>>>(N->OUT, y, N->n[0], batch);
    count_launches(1);
    e = cudaGetLastError();
  }
  return status_of(e);
}

int bfcs_net_grad(bfcs_net N, const float* params, int batch, const float* x, const float* target, float* grad,
                  double* loss_dev) {
  if (N == nullptr || params == nullptr || x == nullptr || target == nullptr || grad == nullptr || batch < 1 ||
      batch > N->maxb || (N->flags & BFCS_NET_TRAIN) == 0)
    return BFCS_ERR_INVALID_ARG;
  cudaError_t e = pack_all(N, params);
  if (e == cudaSuccess) {
    k_features_in<<<grid_for(N->n[0] * batch), 256, 0, N->st>>>(x, N->X0, N->n[0], batch);
    count_launches(1);
    e = forward(N, params, batch);
  }
  if (e == cudaSuccess) e = loss_and_grad(N, batch, target, loss_dev);
  if (e == cudaSuccess) e = backward(N, batch);
  if (e == cudaSuccess) e = grads_to_flat(N, grad);
  return status_of(e);
}

int bfcs_net_adam(bfcs_net N, float* params, const float* grad, float* m, float* v, long long t, float lr) {
  if (N == nullptr || params == nullptr || grad == nullptr || m == nullptr || v == nullptr || t < 1 ||
      !(lr > 0.f) || !std::isfinite(lr))
    return BFCS_ERR_INVALID_ARG;
  const float c1 = (float)(1.0 - std::pow(0.9, (double)t)), c2 = (float)(1.0 - std::pow(0.999, (double)t));
  const long long n = param_count();
  k_adam<<<grid_for(n), 256, 0, N->st>>>(params, grad, m, v, n, lr, 0.9f, 0.999f, 1e-8f, c1, c2);
  count_launches(1);
  return status_of(cudaGetLastError());
}

int bfcs_net_train_step(bfcs_net N, float* params, float* grad, float* m, float* v, long long t, float lr, int batch,
                        const float* x, const float* target, double* loss_dev) {
  const int s = bfcs_net_grad(N, params, batch, x, target, grad, loss_dev);
  if (s != BFCS_OK) return s;
  return bfcs_net_adam(N, params, grad, m, v, t, lr);
}

int bfcs_net_predict(bfcs_net N, const float* params, int precision, int batch, const void* const* b,
                     const int8_t* const* phase, int nphases, const bfcs_lame* phases, void* const* eps_out) {
  if (N == nullptr || params == nullptr || batch < 1 || b == nullptr || phase == nullptr || eps_out == nullptr ||
      (precision != BFCS_FP32 && precision != BFCS_FP64) || !valid_phases(nphases, phases))
    return BFCS_ERR_INVALID_ARG;
  for (int i = 0; i < batch; ++i)
    if (b[i] == nullptr || phase[i] == nullptr || eps_out[i] == nullptr) return BFCS_ERR_INVALID_ARG;
  MuTab mt;
  const float mu_max = mu_table(nphases, phases, &mt);
  const long long n = N->n[0];
  cudaError_t e = pack_all(N, params);
  for (int i0 = 0; i0 < batch && e == cudaSuccess; i0 += N->maxb) {
    const int B = std::min(N->maxb, batch - i0);
    cudaMemsetAsync(N->sbits, 0, B * sizeof(unsigned), N->st);
    for (int i = 0; i < B; ++i) {
      if (precision == BFCS_FP64) {
        k_absmax<double><<<grid_for(3 * n), 256, 0, N->st>>>((const double*)b[i0 + i], 3 * n, N->sbits + i);
        k_prepare_x0<double><<<grid_for(n), 256, 0, N->st>>>((const double*)b[i0 + i], phase[i0 + i], mt,
                                                             N->sbits + i, N->X0 + i * n * 16, n);
      } else {
        k_absmax<float><<<grid_for(3 * n), 256, 0, N->st>>>((const float*)b[i0 + i], 3 * n, N->sbits + i);
        k_prepare_x0<float><<<grid_for(n), 256, 0, N->st>>>((const float*)b[i0 + i], phase[i0 + i], mt,
                                                            N->sbits + i, N->X0 + i * n * 16, n);
      }
    }
    count_launches(2 * B);
    e = forward(N, params, B);
    for (int i = 0; i < B && e == cudaSuccess; ++i) {
      if (precision == BFCS_FP64)
        k_predict_out<double><<<grid_for(n), 256, 0, N->st>>>(N->OUT + i * n * 6, N->sbits + i, mu_max,
                                                              (double*)eps_out[i0 + i], n);
      else
        k_predict_out<float><<<grid_for(n), 256, 0, N->st>>>(N->OUT + i * n * 6, N->sbits + i, mu_max,
                                                             (float*)eps_out[i0 + i], n);
      count_launches(1);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  return status_of(e);
}

}  // extern "C"
