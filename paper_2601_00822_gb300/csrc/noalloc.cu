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
// caches it for that device's context.  The cache is keyed by the context's
// unique id as well: after a cudaDeviceReset the runtime creates a new context
// and loads the library's device code again (possibly at another address), and
// the first call in the new context repeats the look-up.
#include "bfcs.h"
#include "kernels.h"

#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <mutex>

namespace {

// one FP64 partial sum per block plus the mean
constexpr int kNoAllocBlocks = 2048;
constexpr int kThreads = 256;                    // threads per block of the body-force kernels
constexpr long long kMaxVoxels = 134217728;      // the stated limit of this entry point (512^3)
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_bf_scratch[kNoAllocBlocks + 1];

using CtxGetCurrent = CUresult (*)(CUcontext*);
using CtxGetId = CUresult (*)(CUcontext, unsigned long long*);

std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};
unsigned long long g_ctx[kMaxDevices] = {0};
CtxGetCurrent g_get_current = nullptr;
CtxGetId g_get_id = nullptr;

// Unique id of the calling thread's current context (0 when none is current).
// The driver functions are reached through the runtime, so the library does
// not link the driver library itself.
bool current_context_id(unsigned long long* id) {
  if (g_get_current == nullptr || g_get_id == nullptr) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || f1 == nullptr)
      return false;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess || f2 == nullptr)
      return false;
    g_get_current = reinterpret_cast<CtxGetCurrent>(f1);
    g_get_id = reinterpret_cast<CtxGetId>(f2);
  }
  CUcontext ctx = nullptr;
  if (g_get_current(&ctx) != CUDA_SUCCESS) return false;
  *id = 0;
  if (ctx != nullptr && g_get_id(ctx, id) != CUDA_SUCCESS) return false;
  return true;
}

// Device address of g_bf_scratch in the current device's context (set-up on
// the first call per device and context).
int scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BFCS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long id = 0;
  if (!current_context_id(&id)) return BFCS_ERR_CUDA;
  if (g_addr[dev] == nullptr || id == 0 || id != g_ctx[dev]) {
    void* p = nullptr;
    // the look-up makes the device's primary context current if none is
    if (cudaGetSymbolAddress(&p, g_bf_scratch) != cudaSuccess || p == nullptr) return BFCS_ERR_CUDA;
    if (!current_context_id(&id) || id == 0) return BFCS_ERR_CUDA;
    g_addr[dev] = static_cast<double*>(p);
    g_ctx[dev] = id;
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
  if (n > kMaxVoxels) return BFCS_ERR_INVALID_ARG;
  // one thread per voxel up to the scratch's 2048 partial sums (the kernels
  // loop over the grid, so larger grids take several voxels per thread)
  const int blocks = (int)std::min<long long>(kNoAllocBlocks, (n + kThreads - 1) / kThreads);
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
