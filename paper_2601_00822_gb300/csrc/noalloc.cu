// Allocation-free form of the body-force generator (bfcs_body_force_noalloc).
//
// Who needs it: code that must not allocate device memory while it runs --
// for example a host application whose device memory is entirely owned by its
// own pool or caching allocator, a real-time loop in which an allocation could
// stall on a device synchronisation, or a caller that has pre-sized its memory
// budget and treats any extra allocation as an error.  bfcs_body_force obtains
// its small FP64 scratch with cudaMallocAsync on every call; this variant uses
// a fixed array in the library's own device memory instead.
//
// The scratch is a file-scope __device__ array, so every GPU that loads the
// library holds it (16 KiB) until the process exits.  Host code cannot use the
// array's name as a device address, so the first call on each device looks
// the address up with cudaGetSymbolAddress while that device is current and
// caches it per device.
#include "bfcs.h"
#include "kernels.h"

#include <cmath>
#include <mutex>

namespace {

// one FP64 partial sum per block plus the mean
constexpr int kNoAllocBlocks = 2048;
constexpr long long kVoxelsPerBlock = 65536;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_bf_scratch[kNoAllocBlocks + 1];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

// Device address of g_bf_scratch on the current device (set-up on first use).
int scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BFCS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_bf_scratch) != cudaSuccess || p == nullptr) return BFCS_ERR_CUDA;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return BFCS_OK;
}

}  // namespace

extern "C" int bfcs_body_force_noalloc(int nx, int ny, int nz, double cx, double cy, double cz, double a,
                                       int precision, void* b_out, void* stream) {
  if (nx < 1 || ny < 1 || nz < 1 || !(a > 0) || b_out == nullptr ||
      (precision != BFCS_FP32 && precision != BFCS_FP64) || !std::isfinite(cx) || !std::isfinite(cy) ||
      !std::isfinite(cz))
    return BFCS_ERR_INVALID_ARG;
  const long long n = (long long)nx * ny * nz;
  if (n > (long long)kNoAllocBlocks * kVoxelsPerBlock) return BFCS_ERR_INVALID_ARG;   // beyond the scratch
  const int blocks = (int)((n + kVoxelsPerBlock - 1) / kVoxelsPerBlock);
  double* scratch = nullptr;
  const int e = scratch_address(&scratch);
  if (e != BFCS_OK) return e;
  cudaStream_t st = (cudaStream_t)stream;
  const cudaError_t c =
      precision == BFCS_FP64
          ? bfcs::launch_body_force_blocks<double>((double*)b_out, nx, ny, nz, cx, cy, cz, a, blocks, scratch, st)
          : bfcs::launch_body_force_blocks<float>((float*)b_out, nx, ny, nz, cx, cy, cz, a, blocks, scratch, st);
  return c == cudaSuccess ? BFCS_OK : BFCS_ERR_CUDA;
}
