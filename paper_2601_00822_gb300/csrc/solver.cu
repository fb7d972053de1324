// Host side of the C ABI: plans, the sweep driver of the modified basic scheme
// (Algorithm 1) with device-side convergence flags and bounded host waits, the
// batched and translated-averaging drivers (Eqs. 3.3-3.6) and the utilities.
#include <cuda.h>
#include "bfcs.h"
#include "kernels.h"

#include <chrono>
#include <cmath>
#include <cstdlib>
#include <array>
#include <cstring>
#include <thread>
#include <vector>

using namespace bfcs;

struct bfcs_plan_s {
  int nx, ny, nz, max_batch, flags;
  bool fp64;                  // sweeps in FP64 (BFCS_FP64)
  bool mixed;                 // FP32 sweeps + FP64 defect correction (BFCS_MIXED)
  cudaStream_t st;
  Geo g;
  size_t csz;                 // bytes of one complex value
  size_t rsz;                 // bytes of one real value
  void* spec = nullptr;       // 6 x cs complex
  void* bhat = nullptr;       // 3 x cs complex
  void* dprev = nullptr;      // 3 x cs complex
  void* tw[3] = {nullptr, nullptr, nullptr};
  ResidSlot* part = nullptr;
  int npart = 0;              // slots allocated (>= every writer's block count)
  int ngreen = 0;             // blocks of the fused z/Green pass = residual partials per sweep
  int stall_window = 100;     // sweeps without a 10% residual drop that end a solve
  IterState* ist = nullptr;        // max_batch members
  IterState* ist_host = nullptr;   // pinned, 3 slots x max_batch
  Member* mem_dev = nullptr;       // max_batch member descriptors
  Member* mem_host = nullptr;      // pinned staging of the descriptors
  int graph_sweeps = 8;            // sweeps per captured graph (0: no graphs)
  int resid_max = 1;               // BFCS_SPARSE_RESID: most sweeps between residual evaluations (1: every sweep)
  unsigned long long* io_dev = nullptr;   // profiled z/Green launches: d_prev reads, d writes
  cudaStream_t loop_st = nullptr;  // private stream of the sweep loop (capturable), ordered with st
  cudaEvent_t order_ev[2];
  cudaEvent_t ev[2];
  double* hist = nullptr;
  int hist_cap = 0;
  int last_iters = 0;
  int last_batch = 0;
  int* ival = nullptr;             // device: phase min/max, 2 per member
  double* dval = nullptr;          // device: b sums, 6 per member
  double* dscratch = nullptr;      // device scratch for reductions
  int* ival_host = nullptr;        // pinned
  double* dval_host = nullptr;     // pinned
  void* tmp = nullptr;             // 15 x N real: eps, sig, u for averaging members
  int* tmp_hits = nullptr;         // N int
  double* mod_buf = nullptr;       // effective-moduli partial sums and totals
  unsigned long long* prof_buf = nullptr;   // shell maxima and counts of bfcs_radial_profile
  // measurement hook: CUDA events around the launches of one kernel kind
  int prof_kind = 0;
  std::vector<cudaEvent_t> prof_ev;   // start/end pairs
  std::vector<int> prof_sweep;        // sweep index of each pair
  int prof_used = 0;
  long long prof_launches = 0;
  double prof_ms = 0.0;
  // precision ladder (BFCS_MIXED): FP64 transform workspace and FP32 real scratch
  void* spec64 = nullptr;          // max_batch x 6 x cs: complex128 (bfcs_fft3d) or float-float (ladder)
  void* bhat64 = nullptr;          // max_batch x 3 x cs float-float complex: the ladder's load spectra
  void* tw64[3] = {nullptr, nullptr, nullptr};
  void* twff[3] = {nullptr, nullptr, nullptr};   // float-float twiddles of the ladder's passes
  IterState* ist64 = nullptr;      // max_batch FP64 residual states
  float* r32 = nullptr;            // max_batch x 12 x N floats: (unused 3) | eps32 (6) | u32 (3)
  double* u64 = nullptr;           // max_batch x 3 x N doubles: FP64 displacements when the caller passes none
  int max_rounds = 8;              // defect-correction rounds
  double switch_tol = 1e-4;        // FP32 phase stops here (or at the stall)
  bfcs_net net = nullptr;          // inference context of bfcs_surrogate_infer (created on first use)
  bool use_cg = false;             // BFCS_CG: conjugate gradients (Algorithm 2) drive the sweeps
  bool use_cd = false;             // BFCS_CD / BFCS_CD_PRECOND: displacement-based CG (Algorithm 3)
  int cd_precond = 0;              // 1: G0 preconditioner (BFCS_CD_PRECOND)
  double* cd_part = nullptr;       // 2 x kCdParts per member
  CdState* cd_state = nullptr;     // max_batch
  CdState* cd_host = nullptr;      // pinned
  void* cg_vec = nullptr;          // c, r, p, q: 4 x max_batch x 6 x cs complex (sweep precision)
  double* cg_part = nullptr;       // kCgParts per member
  CgState* cg_state = nullptr;     // max_batch
  IterState* cg_skip = nullptr;    // max_batch done flags for the FFT passes of A p
  CgState* cg_host = nullptr;      // pinned copy
  int col_variant = 0;             // y-pass tile / factor order of the FP32 sweeps (autotuned or default)
  double col_variant_ms[kColVariants] = {};   // tuning times (ms per y forward+inverse pair)
  CUtensorMap tmap_y[2];           // FP32 spectra as a 3D tensor for the tensor-copy y passes (8, 16 columns)
  bool tmap_ok = false;
};

namespace {

int severity(int s) { return s < 0 ? 1000 - s : s; }

constexpr int kHistCap = 1 << 14;   // residual history entries kept per member
constexpr double kIncStrainTol = 1e-9;   // ladder: strain increments at or above this tolerance
constexpr int kSparseResidMax = 8;  // BFCS_SPARSE_RESID: most sweeps between residual evaluations

double wait_limit_s() {
  const char* e = std::getenv("BFCS_WAIT_TIMEOUT_S");
  if (e != nullptr) {
    const double v = std::atof(e);
    if (v > 0) return v;
  }
  return 900.0;
}

// Bounded wait for an event: BFCS_ERR_TIMEOUT once the limit passes.
int wait_event(cudaEvent_t ev) {
  const auto t0 = std::chrono::steady_clock::now();
  const double lim = wait_limit_s();
  for (long it = 0;; ++it) {
    const cudaError_t q = cudaEventQuery(ev);
    if (q == cudaSuccess) return BFCS_OK;
    if (q != cudaErrorNotReady) return BFCS_ERR_CUDA;
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > lim) return BFCS_ERR_TIMEOUT;
    if (it < 2000) std::this_thread::yield();
    else std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

int sync_stream(bfcs_plan P) {
  if (cudaEventRecord(P->ev[0], P->st) != cudaSuccess) return BFCS_ERR_CUDA;
  return wait_event(P->ev[0]);
}

#define CK(x)                                   \
  do {                                          \
    if ((x) != cudaSuccess) return BFCS_ERR_CUDA; \
  } while (0)

// Small reads of a solve's state into the plan's pinned host buffers.  With
// unified addressing a kernel writes them directly (no copy engine: a user's
// large host<->device copies on other streams do not hold the solve up); else an
// ordinary asynchronous copy.
bool host_writable_from_device() {
  static int v = -1;
  if (v < 0) {
    int dev = 0, ua = 0;
    v = (cudaGetDevice(&dev) == cudaSuccess &&
         cudaDeviceGetAttribute(&ua, cudaDevAttrUnifiedAddressing, dev) == cudaSuccess && ua == 1) ? 1 : 0;
  }
  return v == 1;
}
cudaError_t read_small(void* host, const void* dev, size_t bytes, cudaStream_t st) {
  if (bytes % sizeof(unsigned) == 0 && host_writable_from_device()) return launch_copy_words(host, dev, bytes, st);
  return cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, st);
}

// The radices (R1, R2) of Fac<n>, on the host.
static void line_radices(int n, int& r1, int& r2) {
  switch (n) {
    case 4: r1 = 2; r2 = 2; break;    case 6: r1 = 3; r2 = 2; break;    case 8: r1 = 4; r2 = 2; break;
    case 12: r1 = 4; r2 = 3; break;   case 16: r1 = 4; r2 = 4; break;   case 24: r1 = 8; r2 = 3; break;
    case 32: r1 = 8; r2 = 4; break;   case 48: r1 = 8; r2 = 6; break;   case 64: r1 = 8; r2 = 8; break;
    case 96: r1 = 16; r2 = 6; break;  case 128: r1 = 16; r2 = 8; break; case 192: r1 = 16; r2 = 12; break;
    case 256: r1 = 16; r2 = 16; break;
    default: r1 = r2 = 0; break;
  }
}

// Twiddles W^j = exp(-2 pi i j / n), j < n, then (FP32 and FP64 tables) the
// factored stage-1 blocks that tw_offset / stage1f read: for each eligible
// first radix r (Fac<n>::R1, then Fac<n>::R2 if it differs), entries
// [b - 1][n2] = W^((n2 b) mod n), b = 1..3, and [a + 2][n2] = W^((4 n2 a) mod n),
// a = 1..r/4-1, for n2 < n / r; float-float tables instead [k1 - 1][n2] =
// W^((n2 k1) mod n), k1 = 1..r1-1, for the first radix r1.
template <typename R>
std::vector<C2<R>> twiddle_table(int n) {
  auto w = [&](long long j) {
    const double t = 2.0 * 3.14159265358979323846 * (double)(j % n) / n;
    C2<R> c;
    c.x = (R)std::cos(t);
    c.y = (R)(-std::sin(t));
    return c;
  };
  std::vector<C2<R>> h(n);
  for (int j = 0; j < n; ++j) h[j] = w(j);
  if (std::is_same<R, ff>::value) {     // float-float: [k1 - 1][n2] = W^(n2 k1), k1 < r1
    int r1 = 0, r2 = 0;
    line_radices(n, r1, r2);
    for (int k1 = 1; k1 < r1; ++k1)
      for (int n2 = 0; n2 < n / r1; ++n2) h.push_back(w((long long)n2 * k1));
  } else {
    int r1 = 0, r2 = 0;
    line_radices(n, r1, r2);
    for (int k = 0; k < 2; ++k) {
      const int r = k == 0 ? r1 : r2;
      if (!tw_factored(r) || (k == 1 && r2 == r1)) continue;   // one block per distinct radix
      const int n2s = n / r;
      for (int b = 1; b < 4; ++b)
        for (int n2 = 0; n2 < n2s; ++n2) h.push_back(w((long long)n2 * b));
      for (int a = 1; a < r / 4; ++a)
        for (int n2 = 0; n2 < n2s; ++n2) h.push_back(w(4LL * n2 * a));
    }
  }
  return h;
}

template <typename R>
void* make_twiddles(int n) {
  const std::vector<C2<R>> h = twiddle_table<R>(n);
  void* d = nullptr;
  if (cudaMalloc(&d, sizeof(C2<R>) * h.size()) != cudaSuccess) return nullptr;
  if (cudaMemcpy(d, h.data(), sizeof(C2<R>) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return nullptr;
  }
  return d;
}

void free_plan(bfcs_plan P) {
  if (P == nullptr) return;
  cudaFree(P->spec); cudaFree(P->bhat); cudaFree(P->dprev);
  for (int i = 0; i < 3; ++i) cudaFree(P->tw[i]);
  cudaFree(P->part); cudaFree(P->ist); cudaFree(P->hist); cudaFree(P->mem_dev); cudaFree(P->io_dev);
  if (P->mem_host) cudaFreeHost(P->mem_host);
  cudaFree(P->ival); cudaFree(P->dval); cudaFree(P->dscratch);
  cudaFree(P->tmp); cudaFree(P->tmp_hits); cudaFree(P->mod_buf); cudaFree(P->prof_buf);
  cudaFree(P->spec64); cudaFree(P->bhat64); cudaFree(P->ist64); cudaFree(P->r32); cudaFree(P->u64);
  for (int i = 0; i < 3; ++i) { cudaFree(P->tw64[i]); cudaFree(P->twff[i]); }
  if (P->ist_host) cudaFreeHost(P->ist_host);
  if (P->ival_host) cudaFreeHost(P->ival_host);
  if (P->dval_host) cudaFreeHost(P->dval_host);
  cudaEventDestroy(P->ev[0]);
  cudaEventDestroy(P->ev[1]);
  for (cudaEvent_t e : P->prof_ev) cudaEventDestroy(e);
  if (P->loop_st) cudaStreamDestroy(P->loop_st);
  if (P->order_ev[0]) cudaEventDestroy(P->order_ev[0]);
  if (P->order_ev[1]) cudaEventDestroy(P->order_ev[1]);
  if (P->net) bfcs_net_destroy(P->net);
  cudaFree(P->cg_vec); cudaFree(P->cg_part); cudaFree(P->cg_state); cudaFree(P->cg_skip);
  cudaFree(P->cd_part); cudaFree(P->cd_state);
  if (P->cd_host) cudaFreeHost(P->cd_host);
  if (P->cg_host) cudaFreeHost(P->cg_host);
  delete P;
}

// Tensor map of the plan's FP32 spectra for the tensor-copy y passes: floats
// along kx (extent 2 mx: columns past mx read as zeros), rows of pitch p (ny),
// planes (member, component, z) of ny p complex values; one box is 2T floats x
// ny rows x 1 plane (T = 8 or 16 columns: 64 or 128 bytes, 16-byte multiples;
// every tile starts at a multiple of 16 floats).  The encoder is reached through
// the runtime, so the library does not link the driver library.  Returns false
// (no tensor-copy variants) when it is unavailable or rejects the layout.
bool encode_spectrum_map(bfcs_plan P) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  const Geo& g = P->g;
  if (g.ny > 256 || g.ny < 32) return false;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || fn == nullptr) {
    cudaGetLastError();
    return false;
  }
  const cuuint64_t dims[3] = {(cuuint64_t)(2 * g.mx), (cuuint64_t)g.ny, (cuuint64_t)P->max_batch * 6 * g.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)g.p * sizeof(C2<float>), (cuuint64_t)g.ny * g.p * sizeof(C2<float>)};
  const cuuint32_t estr[3] = {1, 1, 1};
  for (int k = 0; k < 2; ++k) {       // box widths of the two tile variants: 8 and 16 columns
    const cuuint32_t box[3] = {k == 0 ? 16u : 32u, (cuuint32_t)g.ny, 1};
    const CUresult r = reinterpret_cast<Encode>(fn)(&P->tmap_y[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, P->spec, dims,
                                                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
  }
  return true;
}

// Autotuner of the FP32 sweep's y passes: every valid column-pass variant
// (tile width, factor order) runs a y forward + inverse pair over the plan's
// own spectrum buffer (max_batch members, zeroed), CUDA events on the plan's
// stream, 2 untimed + 5 timed pairs; the fastest is kept.  All variants
// compute the same transform (the factor order changes the rounding only).
int autotune(bfcs_plan P) {
  cudaStream_t st = P->st;
  const size_t bytes = (size_t)P->max_batch * 6 * P->g.cs * sizeof(C2<float>);
  if (cudaMemsetAsync(P->spec, 0, bytes, st) != cudaSuccess) return BFCS_ERR_CUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return BFCS_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return BFCS_ERR_CUDA; }
  CArgs<float> ca{};
  ca.data = (C2<float>*)P->spec;
  ca.g = P->g;
  ca.axis = 1;
  ca.ncomp = 6;
  ca.tw = (const C2<float>*)P->tw[1];
  ca.ms = 6 * P->g.cs;
  ca.tmap = P->tmap_ok ? P->tmap_y : nullptr;
  ca.tmap_data = P->spec;
  double best = INFINITY;
  int bestv = 0, status = BFCS_OK;
  for (int v = 0; v < kColVariants && status == BFCS_OK; ++v) {
    P->col_variant_ms[v] = 0.0;
    if (!col_variant_valid(v, P->g.ny) || (col_variant_tma(v) && !P->tmap_ok)) continue;
    ca.variant = v;
    bool ok = true;
    for (int k = 0; k < 7 && ok; ++k) {
      if (k == 2) ok = cudaEventRecord(e0, st) == cudaSuccess;
      ok = ok && launch_colpass_b<float>(ca, -1, P->max_batch, st) == cudaSuccess &&
           launch_colpass_b<float>(ca, +1, P->max_batch, st) == cudaSuccess;
    }
    ok = ok && cudaEventRecord(e1, st) == cudaSuccess;
    if (!ok) { status = BFCS_ERR_CUDA; break; }
    const int w = wait_event(e1);
    if (w != BFCS_OK) { status = w; break; }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { status = BFCS_ERR_CUDA; break; }
    P->col_variant_ms[v] = ms / 5.0;
    if (ms / 5.0 < best) { best = ms / 5.0; bestv = v; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  P->col_variant = bestv;
  return status;
}

template <typename R>
PhaseTab<R> make_tab(int nph, const bfcs_lame* phases, bfcs_lame C0) {
  PhaseTab<R> t{};
  for (int p = 0; p < kMaxPhases; ++p) {
    const bfcs_lame q = phases[p < nph ? p : nph - 1];
    t.lam[p] = (R)q.lambda;
    t.mu[p] = (R)q.mu;
    t.lam1[p] = (R)(q.lambda - C0.lambda);
    t.mu1[p] = (R)(q.mu - C0.mu);
  }
  return t;
}

int check_material(int nph, const bfcs_lame* phases, bfcs_lame C0) {
  if (phases == nullptr || nph < 1 || nph > BFCS_MAX_PHASES) return BFCS_ERR_INVALID_ARG;
  auto ok = [](bfcs_lame l) {
    return std::isfinite(l.lambda) && std::isfinite(l.mu) && l.mu > 0 && 3 * l.lambda + 2 * l.mu > 0;
  };
  if (!ok(C0)) return BFCS_ERR_INVALID_ARG;
  for (int p = 0; p < nph; ++p)
    if (!ok(phases[p])) return BFCS_ERR_INVALID_ARG;
  return BFCS_OK;
}

// Phase ids in [0, nph) and a self-equilibrated load (Eq. 2.5), for members
// whose phase maps and loads are given in the host arrays.
template <typename R>
int validate_members(bfcs_plan P, int B, const int8_t* const* phase, const void* const* b, int nph) {
  for (int m = 0; m < B; ++m)
    CK(launch_validate<R>(phase[m], (const R*)b[m], P->g.n, P->ival + 2 * m, P->dval + 6 * m, P->dscratch,
                          P->st));
  CK(read_small(P->ival_host, P->ival, 2 * B * sizeof(int), P->st));
  CK(read_small(P->dval_host, P->dval, 6 * B * sizeof(double), P->st));
  const int w = sync_stream(P);
  if (w != BFCS_OK) return w;
  const double thr = sizeof(R) == 4 ? 1e-6 : 1e-12;
  for (int m = 0; m < B; ++m) {
    if (P->ival_host[2 * m] < 0 || P->ival_host[2 * m + 1] >= nph) return BFCS_ERR_INVALID_ARG;
    for (int c = 0; c < 3; ++c) {
      const double sm = P->dval_host[6 * m + c], sa = P->dval_host[6 * m + 3 + c];
      if (!std::isfinite(sm) || !std::isfinite(sa)) return BFCS_ERR_INVALID_ARG;
      if (std::fabs(sm) > thr * sa) return BFCS_ERR_NONZERO_MEAN;
    }
  }
  return BFCS_OK;
}

template <typename R>
int validate_inputs(bfcs_plan P, const int8_t* phase, const void* b, int nph) {
  return validate_members<R>(P, 1, &phase, &b, nph);
}

// b_hat = F(b): x R2C, then y and z forward, into `dst` (3 components).
template <typename R>
int transform_into(bfcs_plan P, const void* b, void* dst, void* const* tw) {
  XArgs<R> xa{};
  xa.g = P->g;
  xa.real_in = (const R*)b;
  xa.spec_out = (C2<R>*)dst;
  xa.ncomp = 3;
  xa.mode = XM_R2C;
  xa.tw = (const C2<R>*)tw[0];
  CK(launch_xpass<R>(xa, P->st));
  CArgs<R> ca{};
  ca.data = (C2<R>*)dst;
  ca.g = P->g;
  ca.ncomp = 3;
  ca.axis = 1;
  ca.tw = (const C2<R>*)tw[1];
  CK(launch_colpass<R>(ca, -1, P->st));
  ca.axis = 2;
  ca.tw = (const C2<R>*)tw[2];
  CK(launch_colpass<R>(ca, -1, P->st));
  return BFCS_OK;
}

template <typename R>
int transform_load(bfcs_plan P, const void* b) {
  return transform_into<R>(P, b, P->bhat, P->tw);
}

struct SolveOut {
  void* eps;
  void* sig;
  void* u;
};

// x-pass member fields (launch arguments) from the host-side descriptors.
template <typename R>
void fill_xm(XArgs<R>& xa, const Member* m, int B, int in_sel, int out_sel) {
  xa.use_xm = 1;
  for (int k = 0; k < B; ++k) {
    XMember& x = xa.xm[k];
    x.phase = m[k].phase;
    x.sx = m[k].sx; x.sy = m[k].sy; x.sz = m[k].sz;
    x.warm = m[k].warm;
    x.real_in = in_sel == XIN_B ? m[k].b : (in_sel == XIN_EPS_INIT || m[k].warm) ? m[k].eps_init : nullptr;
    x.eps_out = (out_sel & XOUT_EPS) ? m[k].eps_out : nullptr;
    x.sig_out = (out_sel & XOUT_SIG) ? m[k].sig_out : nullptr;
    x.real_out = (out_sel & XOUT_U) ? m[k].u_out : nullptr;
  }
}

// Upload B member descriptors (host array) to the plan.
int upload_members(bfcs_plan P, int B, const Member* m) {
  std::memcpy(P->mem_host, m, B * sizeof(Member));
  CK(cudaMemcpyAsync(P->mem_dev, P->mem_host, B * sizeof(Member), cudaMemcpyHostToDevice, P->st));
  return BFCS_OK;
}

// b_hat of every member: x R2C of mem[m].b, then y and z forward; and its norm.
template <typename R>
int transform_members(bfcs_plan P, int B) {
  XArgs<R> xa{};
  xa.g = P->g;
  xa.spec_out = (C2<R>*)P->bhat;
  xa.spec_ms = 3 * P->g.cs;
  fill_xm(xa, P->mem_host, B, XIN_B, 0);
  xa.ncomp = 3;
  xa.mode = XM_R2C;
  xa.tw = (const C2<R>*)P->tw[0];
  CK(launch_xpass_b<R>(xa, B, P->st));
  CArgs<R> ca{};
  ca.data = (C2<R>*)P->bhat;
  ca.ms = 3 * P->g.cs;
  ca.g = P->g;
  ca.ncomp = 3;
  ca.axis = 1;
  ca.tw = (const C2<R>*)P->tw[1];
  CK(launch_colpass_b<R>(ca, -1, B, P->st));
  ca.axis = 2;
  ca.tw = (const C2<R>*)P->tw[2];
  CK(launch_colpass_b<R>(ca, -1, B, P->st));
  CK(launch_bden<R>((const C2<R>*)P->bhat, P->g, P->part, P->ist, P->st, B, 3 * P->g.cs));
  return BFCS_OK;
}

// One plan's batch of B members advancing together (Algorithm 1): the kernel
// arguments of one sweep, the INIT step, the sweep enqueue and the
// finalisation.  Needs the member descriptors, b_hat and bden in place;
// outputs go through the descriptors' eps_out / sig_out / u_out.
template <typename R>
struct SweepSet {
  bfcs_plan P = nullptr;
  int B = 0;
  double tol = 0.0;
  bfcs_lame C0{};
  const double* E0 = nullptr;
  int maxdim = 0;
  GArgs<R> ga{};
  CArgs<R> cy{};
  XArgs<R> xa{};

  void prepare(bfcs_plan plan, int batch, const PhaseTab<R>& tab, bfcs_lame c0, const double* e0, double t) {
    P = plan; B = batch; tol = t; C0 = c0; E0 = e0;
    const Geo g = P->g;
    maxdim = std::max(g.nx, std::max(g.ny, g.nz));
    const long long sms = 6 * g.cs;
    ga.spec = (C2<R>*)P->spec;
    ga.bhat = (const C2<R>*)P->bhat;
    ga.dprev = (C2<R>*)P->dprev;
    ga.g = g;
    ga.lam0 = (R)C0.lambda;
    ga.mu0 = (R)C0.mu;
    for (int c = 0; c < 6; ++c) ga.E[c] = (R)E0[c];
    ga.inv_n = (R)(1.0 / (double)g.n);
    ga.tw = (const C2<R>*)P->tw[2];
    ga.part = P->part;
    ga.st = P->ist;
    ga.use_me = 1;
    for (int m = 0; m < B; ++m)
      for (int c = 0; c < 6; ++c) ga.mE[m][c] = (R)P->mem_host[m].E[c];
    ga.sparse = P->resid_max > 1 ? 1 : 0;
    ga.maxit = 0;                  // set by run_sets for its call
    ga.spec_ms = sms;
    ga.b_ms = 3 * g.cs;
    ga.d_ms = 3 * g.cs;
    ga.part_ms = P->ngreen;
    cy.data = (C2<R>*)P->spec;
    cy.ms = sms;
    cy.g = g;
    cy.ncomp = 6;
    cy.axis = 1;
    cy.tw = (const C2<R>*)P->tw[1];
    cy.variant = P->col_variant;
    cy.tmap = P->tmap_ok ? P->tmap_y : nullptr;
    cy.tmap_data = P->spec;
    xa.g = g;
    xa.spec_in = (C2<R>*)P->spec;
    xa.spec_out = (C2<R>*)P->spec;
    xa.spec_ms = sms;
    xa.tab = tab;
    xa.tw = (const C2<R>*)P->tw[0];
    xa.ncomp = 6;
    fill_xm(xa, P->mem_host, B, XIN_NONE, 0);
  }

  // eps^0 = eps^{b(0)} + E for every member, d_prev = 0; a warm-started member
  // instead starts from its eps_init: the state kept between sweeps is the
  // x-transform of eps scaled by 1/nx (y, z in real space).  On the plan's stream.
  int init(bool any_warm) {
    cudaStream_t st = P->st;
    for (int m = 0; m < B; ++m)
      CK(cudaMemsetAsync(P->ist + m, 0, offsetof(IterState, resid_last), st));
    ga.mode = GM_INIT;
    ga.skip_done = 0;
    CK(launch_zgreen_b<R>(ga, B, st));
    cy.st = nullptr;
    cy.ncomp = 6;
    CK(launch_colpass_b<R>(cy, +1, B, st));
    if (any_warm) {
      for (int m = 0; m < B; ++m) {
        if (!P->mem_host[m].warm) continue;
        XArgs<R> xw{};
        xw.g = P->g;
        xw.real_in = (const R*)P->mem_host[m].eps_init;
        xw.spec_out = (C2<R>*)P->spec + m * 6 * P->g.cs;
        xw.out_scale = (R)(1.0 / P->g.nx);
        xw.ncomp = 6;
        xw.mode = XM_R2C;
        xw.tw = (const C2<R>*)P->tw[0];
        CK(launch_xpass<R>(xw, st));
      }
    }
    P->prof_used = 0;
    return BFCS_OK;
  }

  // one sweep for all members on stream q; identical launches every sweep
  // (graph-capturable); `sweep` labels profiled launches (-1: not profiled)
  int enqueue(cudaStream_t q, int sweep) {
    const int prof_cap = (int)P->prof_sweep.size();
    auto timed = [&](int kind, auto&& fn) -> cudaError_t {
      const bool t = P->prof_kind == kind && P->prof_used < prof_cap && sweep >= 0;
      if (t && cudaEventRecord(P->prof_ev[2 * P->prof_used], q) != cudaSuccess) return cudaErrorUnknown;
      const cudaError_t e = fn();
      if (t) {
        if (cudaEventRecord(P->prof_ev[2 * P->prof_used + 1], q) != cudaSuccess) return cudaErrorUnknown;
        P->prof_sweep[P->prof_used++] = sweep;
      }
      return e;
    };
    xa.mode = XM_SWEEP;
    xa.st = P->ist;
    CK(timed(1, [&] { return launch_xpass_b<R>(xa, B, q); }));
    cy.st = P->ist;
    cy.ncomp = 6;
    CK(timed(2, [&] { return launch_colpass_b<R>(cy, -1, B, q); }));
    ga.mode = GM_SWEEP;
    ga.skip_done = 1;
    CK(timed(3, [&] { return launch_zgreen_b<R>(ga, B, q); }));
    CK(timed(2, [&] { return launch_colpass_b<R>(cy, +1, B, q); }));
    // (the persistent form of the z pass does not run with sparse evaluation)
    const int nparts = ga.sparse ? green_nparts<R>(P->g) : green_sweep_parts<R>(P->g);
    unsigned long long* io = (P->prof_kind == 3 && sweep >= 0) ? P->io_dev : nullptr;
    CK(launch_resid_reduce(P->part, nparts, P->ist, P->mem_dev, P->hist, P->hist_cap, tol, C0.lambda, C0.mu, E0,
                           P->g.n, maxdim, GM_SWEEP, 0, P->stall_window, P->resid_max, ga.maxit, io, B, q));
    return BFCS_OK;
  }

  // eps^S, sigma^S in real space; residual of eps^S; u^S; per-member infos.
  // On the plan's stream; ends with a bounded wait.
  // u_only (no member wants sigma): eps^S by the x-direction C2R of the state and
  // u^S from the d_prev of the last sweep (launch_uhat), without the final pass's
  // forward transforms and residual; infos then report the last evaluated residual.
  bool u_only = false;
  int finalize(bfcs_info* infos) {
    cudaStream_t st = P->st;
    const long long sms = 6 * P->g.cs;
    if (u_only) return finalize_u(infos);
    xa.mode = XM_SWEEP;
    fill_xm(xa, P->mem_host, B, XIN_NONE, XOUT_EPS | XOUT_SIG);
    xa.st = nullptr;
    CK(launch_xpass_b<R>(xa, B, st));
    cy.st = nullptr;
    cy.ncomp = 6;
    CK(launch_colpass_b<R>(cy, -1, B, st));
    ga.mode = GM_FINAL;
    ga.skip_done = 0;
    CK(launch_zgreen_b<R>(ga, B, st));
    CK(launch_resid_reduce(P->part, P->ngreen, P->ist, P->mem_dev, P->hist, P->hist_cap, tol, C0.lambda, C0.mu,
                           E0, P->g.n, maxdim, GM_FINAL, 0, 0, P->resid_max, 0, nullptr, B, st));
    cy.ncomp = 3;
    CK(launch_colpass_b<R>(cy, +1, B, st));
    XArgs<R> xu{};
    xu.g = P->g;
    xu.spec_in = (C2<R>*)P->spec;
    xu.spec_ms = sms;
    fill_xm(xu, P->mem_host, B, XIN_NONE, XOUT_U);
    xu.ncomp = 3;
    xu.mode = XM_C2R;
    xu.tw = (const C2<R>*)P->tw[0];
    CK(launch_xpass_b<R>(xu, B, st));   // members without u_out write nothing
    return report(infos);
  }

  int finalize_u(bfcs_info* infos) {
    cudaStream_t st = P->st;
    const long long sms = 6 * P->g.cs;
    XArgs<R> xe{};
    xe.g = P->g;
    xe.spec_in = (C2<R>*)P->spec;
    xe.spec_ms = sms;
    xe.use_xm = 1;
    bool any_eps = false;
    for (int m = 0; m < B; ++m) {
      XMember& x = xe.xm[m];
      x.phase = P->mem_host[m].phase;
      x.real_out = P->mem_host[m].eps_out;
      any_eps = any_eps || x.real_out != nullptr;
    }
    xe.ncomp = 6;
    xe.mode = XM_C2R;
    xe.tw = (const C2<R>*)P->tw[0];
    if (any_eps) CK(launch_xpass_b<R>(xe, B, st));      // eps^S, before u_hat overwrites the state
    CK(launch_uhat<R>(ga, B, st));
    CArgs<R> cz = cy;
    cz.st = nullptr;
    cz.axis = 2;
    cz.ncomp = 3;
    cz.tw = (const C2<R>*)P->tw[2];
    cz.variant = 0;
    cz.tmap = nullptr;
    CK(launch_colpass_b<R>(cz, +1, B, st));             // z inverse
    cy.st = nullptr;
    cy.ncomp = 3;
    CK(launch_colpass_b<R>(cy, +1, B, st));             // y inverse
    XArgs<R> xu{};
    xu.g = P->g;
    xu.spec_in = (C2<R>*)P->spec;
    xu.spec_ms = sms;
    fill_xm(xu, P->mem_host, B, XIN_NONE, XOUT_U);
    xu.ncomp = 3;
    xu.mode = XM_C2R;
    xu.tw = (const C2<R>*)P->tw[0];
    CK(launch_xpass_b<R>(xu, B, st));
    return report(infos);
  }

  // per-member infos from the device states (bounded wait)
  int report(bfcs_info* infos) {
    cudaStream_t st = P->st;
    IterState* hf = P->ist_host + 2 * P->max_batch;
    CK(read_small(hf, P->ist, B * sizeof(IterState), st));
    const int w = sync_stream(P);
    if (w != BFCS_OK) return w;
    P->last_iters = hf[0].iters;
    P->last_batch = B;
    for (int k = 0; k < P->prof_used; ++k) {
      if (P->prof_sweep[k] >= hf[0].iters) continue;     // launches of sweeps skipped on device
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, P->prof_ev[2 * k], P->prof_ev[2 * k + 1]) != cudaSuccess)
        return BFCS_ERR_CUDA;
      P->prof_ms += ms;
      P->prof_launches += 1;
    }
    P->prof_used = 0;
    int worst = BFCS_OK;
    for (int m = 0; m < B; ++m) {
      const IterState& h = hf[m];
      int status = BFCS_OK;
      const double rf = u_only ? h.resid_last : h.resid_final;
      if (h.diverged == 2) status = BFCS_ERR_TIMEOUT;     // a bounded device wait expired
      else if (h.diverged || (!u_only && !std::isfinite(rf))) status = BFCS_ERR_DIVERGED;
      else if (tol > 0 && (!h.done || h.stalled)) status = BFCS_NOT_CONVERGED;
      if (infos != nullptr) {
        infos[m].iters = h.iters;
        infos[m].status = status;
        infos[m].resid = rf;
        infos[m].resid_prev = h.resid_last;
        infos[m].precision_path = sizeof(R) == 8 ? 1 : 0;
        infos[m].stalled = h.stalled;
      }
      if (severity(status) > severity(worst)) worst = status;
    }
    return worst;
  }
};

// The sweep loop of one or more sweep sets (plans of possibly different grid
// sizes), after their init().  It runs on the first plan's private stream
// (capturable even when a caller's stream is the legacy default stream); every
// other plan's private stream forks from it and joins it again, so one CUDA
// graph launch advances every set by graph_sweeps sweeps, the sets running
// side by side on the GPU.  The host reads the device states of chunk k-1
// while chunk k runs; the contraction rate of two observed residuals gives the
// sweeps still needed by the slowest member of any set, which sizes the next
// chunk; once the chunk in flight is expected to finish every member, the host
// waits for it before sending more (sweeps enqueued past convergence are
// skipped on the device, but still cost their launches).  Each set's own
// stream waits for the loop before its finalize().
template <typename R>
int run_sets(std::vector<SweepSet<R>*>& sets, int maxit) {
  const int S = (int)sets.size();
  bfcs_plan P0 = sets[0]->P;
  cudaStream_t const main = P0->loop_st;
  std::vector<cudaEvent_t> evs;                      // fork/join events of this call
  struct EvGuard {
    std::vector<cudaEvent_t>& v;
    ~EvGuard() { for (cudaEvent_t e : v) cudaEventDestroy(e); }
  } evguard{evs};
  auto new_event = [&](cudaEvent_t* e) -> bool {
    if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return false;
    evs.push_back(*e);
    return true;
  };
  // the loop stream starts after every set's stream (their INIT work)
  for (auto* ss : sets) {
    cudaEvent_t e;
    if (!new_event(&e)) return BFCS_ERR_CUDA;
    CK(cudaEventRecord(e, ss->P->st));
    CK(cudaStreamWaitEvent(main, e, 0));
  }
  // enqueue k sweeps of every set: set 0 on the main stream, the others forked
  auto enqueue_all = [&](int k, int label0) -> int {
    cudaEvent_t fork;
    if (S > 1) {
      if (!new_event(&fork)) return BFCS_ERR_CUDA;
      CK(cudaEventRecord(fork, main));
    }
    for (int i = 1; i < S; ++i) {
      cudaStream_t q = sets[i]->P->loop_st;
      CK(cudaStreamWaitEvent(q, fork, 0));
      for (int j = 0; j < k; ++j) {
        const int e = sets[i]->enqueue(q, label0 < 0 ? -1 : label0 + j);
        if (e != BFCS_OK) return e;
      }
    }
    for (int j = 0; j < k; ++j) {
      const int e = sets[0]->enqueue(main, label0 < 0 ? -1 : label0 + j);
      if (e != BFCS_OK) return e;
    }
    for (int i = 1; i < S; ++i) {
      cudaEvent_t join;
      if (!new_event(&join)) return BFCS_ERR_CUDA;
      CK(cudaEventRecord(join, sets[i]->P->loop_st));
      CK(cudaStreamWaitEvent(main, join, 0));
    }
    return BFCS_OK;
  };

  for (auto* ss : sets) ss->ga.maxit = maxit;     // the last sweep of this call stores d for the final step
  bool profiling = false;
  for (auto* ss : sets) profiling = profiling || ss->P->prof_kind != 0;
  const int G = profiling ? 0 : P0->graph_sweeps;
  cudaGraphExec_t gexec = nullptr;
  if (G > 0 && maxit >= G) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal));
    const int e = enqueue_all(G, -1);
    const cudaError_t ce = cudaStreamEndCapture(main, &graph);
    if (e != BFCS_OK || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return e != BFCS_OK ? e : BFCS_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return BFCS_ERR_CUDA;
  }
  struct GraphGuard {
    cudaGraphExec_t g;
    ~GraphGuard() { if (g) cudaGraphExecDestroy(g); }
  } guard{gexec};

  // all members of all sets, in order
  int total = 0;
  for (auto* ss : sets) total += ss->B;
  std::vector<int> obs_it(total, -1);
  std::vector<double> obs_r(total, 0.0);
  cudaEvent_t ev[2];
  if (!new_event(&ev[0]) || !new_event(&ev[1])) return BFCS_ERR_CUDA;
  auto host_state = [&](int slot, int i) { return sets[i]->P->ist_host + slot * sets[i]->P->max_batch; };
  auto all_done = [&](int slot) {
    for (int i = 0; i < S; ++i) {
      const IterState* h = host_state(slot, i);
      for (int m = 0; m < sets[i]->B; ++m)
        if (!h[m].done) return false;
    }
    return true;
  };
  // sweeps still needed by the slowest member after the observed state (<0: unknown)
  auto predict = [&](int slot) {
    double worst = 0.0;
    bool known = true;
    int gm = 0;
    for (int i = 0; i < S; ++i) {
      const IterState* h = host_state(slot, i);
      const SweepSet<R>& ss = *sets[i];
      for (int m = 0; m < ss.B; ++m, ++gm) {
        if (h[m].done) continue;
        // the residual observed is of sweep last_check (every sweep's, unless sparse)
        const double r = h[m].resid_last;
        const int at = h[m].last_check;
        const double tl = ss.P->mem_host[m].tol >= 0 ? ss.P->mem_host[m].tol : ss.tol;
        if (!(tl > 0) || !(h[m].checks > 0) || !std::isfinite(r) || !(r > 0) || obs_it[gm] < 0 ||
            !(at > obs_it[gm]) || !(r < obs_r[gm])) {
          known = false;
        } else {
          const double rate = std::pow(r / obs_r[gm], 1.0 / (at - obs_it[gm]));
          worst = std::max(worst, std::log(tl / r) / std::log(rate) - (h[m].iters - 1 - at));
        }
        if (h[m].checks > 0 && std::isfinite(r) && r > 0) { obs_it[gm] = at; obs_r[gm] = r; }
      }
    }
    return known ? worst : -1.0;
  };
  auto read_states = [&](int slot) -> int {
    for (int i = 0; i < S; ++i)
      CK(read_small(host_state(slot, i), sets[i]->P->ist, sets[i]->B * sizeof(IterState), main));
    CK(cudaEventRecord(ev[slot], main));
    return BFCS_OK;
  };
  int s = 0, chunk = 4, slot = 0;
  bool pending = false;
  int last_c = 0;
  while (s < maxit) {
    int c;
    if (gexec != nullptr && maxit - s >= G) {
      // whole graphs, never past maxit (the remainder runs as single sweeps)
      c = G * std::max(1, std::min(chunk, maxit - s) / G);
      for (int k = 0; k < c; k += G) CK(cudaGraphLaunch(gexec, main));
    } else {
      c = std::min(chunk, maxit - s);
      const int e = enqueue_all(c, s);
      if (e != BFCS_OK) return e;
    }
    s += c;
    int e = read_states(slot);
    if (e != BFCS_OK) return e;
    int next = std::min(chunk * 2, 64);
    bool drain = false;
    if (pending) {
      const int w = wait_event(ev[slot ^ 1]);
      if (w != BFCS_OK) return w;
      if (all_done(slot ^ 1)) break;
      const double need = predict(slot ^ 1);
      if (need >= 0) {
        const double left = need - last_c;
        if (left <= 0.5) drain = true;
        else next = std::max(1, std::min(64, (int)std::ceil(left) + 1));
      }
    }
    pending = true;
    slot ^= 1;
    last_c = c;
    chunk = next;
    if (drain) {
      const int w = wait_event(ev[slot ^ 1]);
      if (w != BFCS_OK) return w;
      if (all_done(slot ^ 1)) break;
      pending = false;
      chunk = 2;
      predict(slot ^ 1);
    }
  }
  // back on every set's own stream
  cudaEvent_t done;
  if (!new_event(&done)) return BFCS_ERR_CUDA;
  CK(cudaEventRecord(done, main));
  for (auto* ss : sets) CK(cudaStreamWaitEvent(ss->P->st, done, 0));
  return BFCS_OK;
}

// Chunk sizing of the Krylov loops, which read the members' device states after
// each chunk of iterations (iterations enqueued past a member's stop are skipped
// on the device but still cost their launches).  predict_left: from the residual r
// at iteration `it` and the one observed before (r_obs at it_obs), the iterations
// still needed to reach tol at the observed contraction rate, raised into `need`;
// false when unknown (no earlier observation, no decrease, no tolerance).
// next_chunk: that many plus one (2..64), else twice the last chunk.
static bool predict_left(double r, double tol, int it, double r_obs, int it_obs, double& need) {
  if (!(tol > 0) || !(r > 0) || !std::isfinite(r) || it_obs < 0 || it <= it_obs || !(r < r_obs)) return false;
  const double rate = std::pow(r / r_obs, 1.0 / (it - it_obs));
  need = std::max(need, std::log(tol / r) / std::log(rate));
  return true;
}
static int next_chunk(bool known, double need, int chunk) {
  if (!known) return std::min(chunk * 2, 64);
  return std::max(2, std::min(64, (int)std::ceil(need) + 1));
}

// Conjugate gradients (Algorithm 2, operator of Eq. 5.13) from the current
// state of every member of the set: c = the state, one standard sweep gives
// s, r = p = s - c (the fixed-point residual is the CG residual), then
// iterations of A p = p - F^-1 U0 F L1 p (the sweep's passes with the load
// switched off) until <r, r>_C0 <= rel_m^2 <r0, r0>_C0 or `maxit` iterations
// (or stagnation); the state becomes c.  rel_m = 0.5 tol_m / req_m, clamped to
// [floor, 0.5] (floor: 1e-6 in FP32, 1e-13 in FP64), with req_m the member's
// last measured residual of Eq. 5.11 (req_m <= 0: unknown; then the first
// sweep's residual is used for a cold start, else rel_m = 0.1).  Adds the
// operator applications to `applied`.
template <typename R>
int run_cg(SweepSet<R>& ss, std::vector<double>& req, int maxit, std::vector<int>& applied,
           const std::vector<char>& finished) {
  bfcs_plan P = ss.P;
  const int B = ss.B;
  cudaStream_t st = P->st;
  const Geo g = P->g;
  const long long sms = 6 * g.cs;
  const size_t vbytes = (size_t)B * sms * sizeof(C2<R>);
  C2<R>* base = (C2<R>*)P->cg_vec;
  const long long vstride = (long long)P->max_batch * sms;
  CgArgs<R> ca{};
  ca.c = base;
  ca.r = base + vstride;
  ca.p = base + 2 * vstride;
  ca.q = base + 3 * vstride;
  ca.ms = sms;
  ca.g = g;
  ca.lam0 = ss.C0.lambda;
  ca.mu0 = ss.C0.mu;
  ca.part = P->cg_part;
  ca.cg = P->cg_state;
  ca.skip = P->cg_skip;
  // c = state; s = one sweep of it (the standard pass, load included)
  CK(cudaMemcpyAsync(ca.c, P->spec, vbytes, cudaMemcpyDeviceToDevice, st));
  int e = ss.enqueue(st, -1);
  if (e != BFCS_OK) return e;
  bool unknown = false;
  for (int m = 0; m < B; ++m) unknown = unknown || (!(req[m] > 0) && !P->mem_host[m].warm);
  if (unknown) {   // cold start: the sweep just run evaluated r(eps^0)
    CK(read_small(P->ist_host, P->ist, B * sizeof(IterState), st));
    const int w = sync_stream(P);
    if (w != BFCS_OK) return w;
    for (int m = 0; m < B; ++m)
      if (!(req[m] > 0) && !P->mem_host[m].warm && std::isfinite(P->ist_host[m].resid_last))
        req[m] = P->ist_host[m].resid_last;
  }
  const double floor = sizeof(R) == 4 ? 1e-6 : 1e-13;
  for (int m = 0; m < B; ++m) {
    CgState& h = P->cg_host[m];
    h = CgState{};
    const double tl = P->mem_host[m].tol >= 0 ? P->mem_host[m].tol : ss.tol;
    const double rel = req[m] > 0 ? std::min(0.5, std::max(floor, 0.5 * tl / req[m])) : 0.1;
    h.tol2 = rel * rel;
    h.maxit = std::max(1, maxit);
  }
  CK(cudaMemcpyAsync(P->cg_state, P->cg_host, B * sizeof(CgState), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(P->cg_skip, 0, B * sizeof(IterState), st));
  ca.s = (const C2<R>*)P->spec;
  CK(launch_cg_vec<R>(ca, 0, B, st));
  ca.s = nullptr;
  // A p through the sweep's passes: x (tau = L1 p, forward x) -> y -> z/Green (operator only) -> y
  XArgs<R> xa = ss.xa;
  xa.mode = XM_SWEEP;
  xa.spec_in = ca.p;
  xa.spec_out = ca.q;
  xa.st = P->cg_skip;
  CArgs<R> cy = ss.cy;
  cy.data = ca.q;   // not the mapped spectrum: the same tile with direct loads (tmap_data != data)
  cy.st = P->cg_skip;
  cy.ncomp = 6;
  GArgs<R> ga = ss.ga;
  ga.spec = ca.q;
  ga.st = P->cg_skip;
  ga.mode = GM_APPLY;
  ga.skip_done = 1;
  auto iteration = [&]() -> int {
    CK(launch_xpass_b<R>(xa, B, st));
    CK(launch_colpass_b<R>(cy, -1, B, st));
    CK(launch_zgreen_b<R>(ga, B, st));
    CK(launch_colpass_b<R>(cy, +1, B, st));
    CK(launch_cg_vec<R>(ca, 1, B, st));
    CK(launch_cg_vec<R>(ca, 2, B, st));
    CK(launch_cg_vec<R>(ca, 3, B, st));
    return BFCS_OK;
  };
  int done_all = 0, it = 0, chunk = 8;
  std::vector<double> obs_r(B, -1.0);
  std::vector<int> obs_it(B, -1);
  while (!done_all && it < maxit) {
    const int c = std::min(chunk, maxit - it);
    for (int k = 0; k < c; ++k) {
      e = iteration();
      if (e != BFCS_OK) return e;
    }
    it += c;
    CK(read_small(P->cg_host, P->cg_state, B * sizeof(CgState), st));
    const int w = sync_stream(P);
    if (w != BFCS_OK) return w;
    done_all = 1;
    double need = 0.0;
    bool known = true;
    for (int m = 0; m < B; ++m) {
      const CgState& h = P->cg_host[m];
      if (h.done) continue;
      done_all = 0;
      // the stop test compares <r, r> with tol2 <r0, r0>: norms, squared
      const double r = h.rr > 0 ? std::sqrt(h.rr) : -1.0;
      known = known && predict_left(r, std::sqrt(h.tol2 * h.rr0), h.iters, obs_r[m], obs_it[m], need);
      obs_r[m] = r;
      obs_it[m] = h.iters;
    }
    chunk = next_chunk(known, need, chunk);
  }
  for (int m = 0; m < B; ++m)
    if (!finished[m]) applied[m] += 1 + P->cg_host[m].iters;   // finished members skipped both
  CK(cudaMemcpyAsync(P->spec, ca.c, vbytes, cudaMemcpyDeviceToDevice, st));
  return BFCS_OK;
}

// Displacement-based CG (Algorithm 3) for the B members of ss, after its init()
// (state: eps^{b(0)} + E, x transformed).  b^A = i xi . F[L1 eps^{b(0)}] comes from
// one x pass (polarization) and the forward y and z passes; every iteration
// applies the operator to p with the strain spectrum sym(i xi (x) p) / N (the
// direction step writes it), the inverse z and y passes, the x pass that forms
// sigma = L eps and transforms it forward, the forward y and z passes and the
// divergence (PQ step), then updates u1, r and z (UPDATE) and p (DIR).  The host
// reads the members' states after chunks of iterations.  Finally the strain
// eps^{b(0)} + grad^s u1 and the displacement u^{b(0)} + u1 are transformed back
// (with sigma = L eps when wanted) and the residual of Eq. 5.11 of the returned
// strain is formed.  A warm start is not taken (Algorithm 3 starts from u1 = 0).
template <typename R>
int run_cd(SweepSet<R>& ss, int maxit, bfcs_info* infos) {
  bfcs_plan P = ss.P;
  const int B = ss.B;
  cudaStream_t st = P->st;
  const Geo g = P->g;
  const long long vs = 3 * g.cs;
  const long long vstride = (long long)P->max_batch * vs;
  C2<R>* base = (C2<R>*)P->cg_vec;                 // 4 x max_batch x 3 cs of the 4 x max_batch x 6 cs
  CdArgs<R> a{};
  a.u = base;
  a.r = base + vstride;
  a.p = base + 2 * vstride;
  a.q = base + 3 * vstride;
  a.s = (C2<R>*)P->spec;
  a.ms = vs;
  a.sms = 6 * g.cs;
  a.bhat = (const C2<R>*)P->bhat;
  a.b_ms = 3 * g.cs;
  a.g = g;
  a.lam0 = ss.C0.lambda;
  a.mu0 = ss.C0.mu;
  a.part = P->cd_part;
  a.cd = P->cd_state;
  a.skip = P->cg_skip;
  a.mem = P->mem_dev;
  a.precond = P->cd_precond;
  a.tw = (const C2<R>*)P->tw[2];
  const int maxdim = std::max(g.nx, std::max(g.ny, g.nz));
  for (int m = 0; m < B; ++m) {
    CdState& h = P->cd_host[m];
    h = CdState{};
    h.tol = P->mem_host[m].tol >= 0 ? P->mem_host[m].tol : ss.tol;
    h.maxit = maxit;
  }
  CK(cudaMemcpyAsync(P->cd_state, P->cd_host, B * sizeof(CdState), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(P->cg_skip, 0, B * sizeof(IterState), st));
  // b^A from the state eps^{b(0)} (+ E): tau = L1 eps, forward x, y, z
  XArgs<R> xa = ss.xa;
  xa.mode = XM_SWEEP;
  fill_xm(xa, P->mem_host, B, XIN_NONE, 0);
  xa.st = nullptr;
  CK(launch_xpass_b<R>(xa, B, st));
  CArgs<R> cy = ss.cy;
  cy.st = nullptr;
  cy.ncomp = 6;
  CArgs<R> cz = ss.cy;
  cz.st = nullptr;
  cz.axis = 2;
  cz.ncomp = 6;
  cz.tw = (const C2<R>*)P->tw[2];
  cz.variant = 0;
  cz.tmap = nullptr;
  CK(launch_colpass_b<R>(cy, -1, B, st));
  CK(launch_colpass_b<R>(cz, -1, B, st));
  CK(launch_cd_vec<R>(a, CdMode::INIT, B, P->ist, P->mem_dev, maxdim, st));
  CK(launch_zcd<R>(a, false, B, P->ist, P->mem_dev, maxdim, st));      // p = z, its strain, inverse z
  // iterations: inverse y, x (sigma = L eps), forward y, then the fused forward z
  // pass with the divergence and <p, A p>, the update, and the fused direction step
  // with the inverse z transform of the next operator input
  XArgs<R> xs = ss.xa;
  xs.mode = XM_SWEEPSIG;
  fill_xm(xs, P->mem_host, B, XIN_NONE, 0);
  xs.st = P->cg_skip;
  cy.st = P->cg_skip;
  cz.st = P->cg_skip;
  int it = 0, chunk = 8;
  std::vector<double> obs_r(B, -1.0);
  std::vector<int> obs_it(B, -1);
  while (it < maxit) {
    const int c = std::min(chunk, maxit - it);
    for (int k = 0; k < c; ++k) {
      CK(launch_colpass_b<R>(cy, +1, B, st));
      CK(launch_xpass_b<R>(xs, B, st));
      CK(launch_colpass_b<R>(cy, -1, B, st));
      CK(launch_zcd<R>(a, true, B, P->ist, P->mem_dev, maxdim, st));
      CK(launch_cd_vec<R>(a, CdMode::UPDATE, B, P->ist, P->mem_dev, maxdim, st));
      CK(launch_zcd<R>(a, false, B, P->ist, P->mem_dev, maxdim, st));
    }
    it += c;
    CK(read_small(P->cd_host, P->cd_state, B * sizeof(CdState), st));
    const int w = sync_stream(P);
    if (w != BFCS_OK) return w;
    bool all = true;
    double need = 0.0;
    bool known = true;
    for (int m = 0; m < B; ++m) {
      const CdState& h = P->cd_host[m];
      if (h.done) continue;
      all = false;
      known = known && predict_left(h.resid, h.tol, h.iters, obs_r[m], obs_it[m], need);
      obs_r[m] = h.resid;
      obs_it[m] = h.iters;
    }
    if (all) break;
    chunk = next_chunk(known, need, chunk);
  }
  // the returned strain eps^{b(0)} + grad^s u1 (and sigma), its residual, the displacement
  cy.st = nullptr;
  cz.st = nullptr;
  CK(launch_cd_vec<R>(a, CdMode::FINAL, B, P->ist, P->mem_dev, maxdim, st));
  CK(launch_colpass_b<R>(cz, +1, B, st));
  CK(launch_colpass_b<R>(cy, +1, B, st));
  XArgs<R> xf = ss.xa;
  xf.mode = XM_SWEEPSIG;
  fill_xm(xf, P->mem_host, B, XIN_NONE, XOUT_EPS | XOUT_SIG);
  xf.st = nullptr;
  CK(launch_xpass_b<R>(xf, B, st));
  CK(launch_colpass_b<R>(cy, -1, B, st));
  CK(launch_colpass_b<R>(cz, -1, B, st));
  CK(launch_cd_vec<R>(a, CdMode::RESID, B, P->ist, P->mem_dev, maxdim, st));
  CK(launch_cd_vec<R>(a, CdMode::FINAL_U, B, P->ist, P->mem_dev, maxdim, st));
  cz.ncomp = 3;
  cy.ncomp = 3;
  CK(launch_colpass_b<R>(cz, +1, B, st));
  CK(launch_colpass_b<R>(cy, +1, B, st));
  XArgs<R> xu{};
  xu.g = P->g;
  xu.spec_in = (C2<R>*)P->spec;
  xu.spec_ms = 6 * g.cs;
  fill_xm(xu, P->mem_host, B, XIN_NONE, XOUT_U);
  xu.ncomp = 3;
  xu.mode = XM_C2R;
  xu.tw = (const C2<R>*)P->tw[0];
  CK(launch_xpass_b<R>(xu, B, st));
  ss.u_only = false;                               // the residual of the returned strain was formed
  return ss.report(infos);
}

// Algorithm 1 for B members of one grid, advancing together: each sweep is
// one launch per pass for all members; converged members skip on the device.
// With BFCS_CG the sweeps are driven by conjugate gradients (Algorithm 2):
// rounds of CG, each aimed at 0.5 tol relative to the last measured residual
// of Eq. 5.11 and followed by two verifying sweeps (the first one as a warm
// start, whose residual is not evaluated); rounds repeat while they at least
// halve the residual, then plain sweeps finish the job.
template <typename R>
int run_batch(bfcs_plan P, int B, const PhaseTab<R>& tab, bfcs_lame C0, const double* E0, double tol,
              int maxit, bfcs_info* infos, bool any_warm, bool u_only = false) {
  SweepSet<R> ss;
  ss.prepare(P, B, tab, C0, E0, tol);
  ss.u_only = u_only;
  if (P->use_cd && any_warm) return BFCS_ERR_INVALID_ARG;   // Algorithm 3 starts from u1 = 0
  int e = ss.init(any_warm);
  if (e != BFCS_OK) return e;
  if (P->use_cd) return run_cd<R>(ss, maxit, infos);
  std::vector<SweepSet<R>*> sets{&ss};
  if (P->use_cg && tol > 0 && maxit > 2) {
    std::vector<int> applied(B, 0), verify(B, 0);
    std::vector<double> req(B, -1.0);
    int left = maxit;
    if (any_warm) {               // a warm start need not be compatible: one plain sweep makes it so
      e = ss.enqueue(P->st, -1);
      if (e != BFCS_OK) return e;
      for (int m = 0; m < B; ++m) applied[m] += 1;
      left -= 1;
    }
    bool all = false;
    std::vector<char> finished(B, 0);      // met the tolerance in a verification: left alone afterwards
    for (int round = 0; round < 30 && !all && left > 2; ++round) {
      const std::vector<double> before = req;
      e = run_cg<R>(ss, req, left - 2, applied, finished);   // finished members skip (iteration state done)
      if (e != BFCS_OK) return e;
      // verify: the CG iterate is the warm start of two sweeps
      for (int m = 0; m < B; ++m) P->mem_host[m].warm = 1;
      e = upload_members(P, B, P->mem_host);
      if (e != BFCS_OK) return e;
      for (int m = 0; m < B; ++m)
        if (!finished[m]) CK(cudaMemsetAsync(P->ist + m, 0, offsetof(IterState, resid_last), P->st));
      e = run_sets<R>(sets, 2);
      if (e != BFCS_OK) return e;
      CK(read_small(P->ist_host, P->ist, B * sizeof(IterState), P->st));
      const int w = sync_stream(P);
      if (w != BFCS_OK) return w;
      all = true;
      bool progress = false;
      int most = 0;
      for (int m = 0; m < B; ++m) {
        const IterState& h = P->ist_host[m];
        if (!finished[m]) {
          verify[m] = h.iters;
          applied[m] += verify[m];
          if (h.done) {
            finished[m] = 1;
          } else {
            all = false;
            if (std::isfinite(h.resid_last) && h.resid_last > 0) {
              progress = progress || !(before[m] > 0) || h.resid_last < 0.5 * before[m];
              req[m] = h.resid_last;
            }
          }
        }
        most = std::max(most, applied[m]);
      }
      left = maxit - most;
      if (!all && !progress) break;          // CG no longer helps (e.g. the FP32 floor): plain sweeps finish
    }
    if (!all && left > 0) {        // plain sweeps from the last state (same iteration state)
      e = run_sets<R>(sets, left);
      if (e != BFCS_OK) return e;
    }
    e = ss.finalize(infos);       // infos[m].iters = sweeps since the last verification started
    if (infos != nullptr)
      for (int m = 0; m < B; ++m) infos[m].iters += applied[m] - verify[m];
    return e;
  }
  e = run_sets<R>(sets, maxit);
  if (e != BFCS_OK) return e;
  return ss.finalize(infos);
}

Member make_member(const int8_t* phase, const int shift[3], const double* E, const void* b,
                   const void* eps_init, SolveOut out) {
  Member m{};
  m.phase = phase;
  m.sx = shift[0]; m.sy = shift[1]; m.sz = shift[2];
  m.warm = eps_init != nullptr ? 1 : 0;
  for (int c = 0; c < 6; ++c) m.E[c] = E[c];
  m.b = b;
  m.eps_init = eps_init;
  m.eps_out = out.eps;
  m.sig_out = out.sig;
  m.u_out = out.u;
  m.tol = -1.0;
  return m;
}

// One solve whose b_hat and bden are already in the plan (member 0).
template <typename R>
int solve_core(bfcs_plan P, const int8_t* phase, const PhaseTab<R>& tab, bfcs_lame C0, const double* E,
               double tol, int maxit, const void* eps_init, SolveOut out, const int shift[3],
               bfcs_info* info) {
  const Member m = make_member(phase, shift, E, nullptr, eps_init, out);
  int e = upload_members(P, 1, &m);
  if (e != BFCS_OK) return e;
  return run_batch<R>(P, 1, tab, C0, E, tol, maxit, info, eps_init != nullptr);
}

template <typename R>
int solve_impl(bfcs_plan P, const int8_t* phase, int nph, const bfcs_lame* phases, bfcs_lame C0,
               const void* b, const double* E, double tol, int maxit, const void* eps_init, SolveOut out,
               const int shift[3], bfcs_info* info) {
  int e = check_material(nph, phases, C0);
  if (e != BFCS_OK) return e;
  if (phase == nullptr || b == nullptr || E == nullptr || out.eps == nullptr) return BFCS_ERR_INVALID_ARG;
  if (!(tol >= 0) || maxit < 0 || (eps_init != nullptr && maxit < 1)) return BFCS_ERR_INVALID_ARG;
  for (int c = 0; c < 6; ++c)
    if (!std::isfinite(E[c])) return BFCS_ERR_INVALID_ARG;
  e = validate_inputs<R>(P, phase, b, nph);
  if (e != BFCS_OK) return e;
  const Member m = make_member(phase, shift, E, b, eps_init, out);
  e = upload_members(P, 1, &m);
  if (e != BFCS_OK) return e;
  e = transform_members<R>(P, 1);
  if (e != BFCS_OK) return e;
  return run_batch<R>(P, 1, make_tab<R>(nph, phases, C0), C0, E, tol, maxit, info, eps_init != nullptr);
}

// bfcs_solve_batched on FP32/FP64 plans: groups of up to max_batch members
// advance together (one launch per pass per sweep for the whole group).
template <typename R>
int solve_batch_impl(bfcs_plan P, int batch, const bfcs_problem* pr, int nph, const bfcs_lame* phases,
                     bfcs_lame C0, double tol, int maxit, bfcs_info* infos) {
  int e = check_material(nph, phases, C0);
  if (e != BFCS_OK) return e;
  if (!(tol >= 0) || maxit < 0) return BFCS_ERR_INVALID_ARG;
  for (int m = 0; m < batch; ++m) {
    if (pr[m].phase == nullptr || pr[m].b == nullptr || pr[m].eps_out == nullptr) return BFCS_ERR_INVALID_ARG;
    if (pr[m].eps_init != nullptr && maxit < 1) return BFCS_ERR_INVALID_ARG;
    for (int c = 0; c < 6; ++c)
      if (!std::isfinite(pr[m].E[c])) return BFCS_ERR_INVALID_ARG;
  }
  const PhaseTab<R> tab = make_tab<R>(nph, phases, C0);
  int worst = BFCS_OK;
  std::vector<Member> mem;
  std::vector<const int8_t*> ph;
  std::vector<const void*> bs;
  for (int start = 0; start < batch; start += P->max_batch) {
    const int B = std::min(P->max_batch, batch - start);
    mem.clear(); ph.clear(); bs.clear();
    bool warm = false;
    for (int m = start; m < start + B; ++m) {
      mem.push_back(make_member(pr[m].phase, pr[m].shift, pr[m].E, pr[m].b, pr[m].eps_init,
                                SolveOut{pr[m].eps_out, pr[m].sig_out, pr[m].u_out}));
      ph.push_back(pr[m].phase);
      bs.push_back(pr[m].b);
      warm = warm || pr[m].eps_init != nullptr;
    }
    e = validate_members<R>(P, B, ph.data(), bs.data(), nph);
    if (e != BFCS_OK) return e;
    e = upload_members(P, B, mem.data());
    if (e != BFCS_OK) return e;
    e = transform_members<R>(P, B);
    if (e != BFCS_OK) return e;
    const int s = run_batch<R>(P, B, tab, C0, pr[start].E, tol, maxit, infos != nullptr ? infos + start : nullptr,
                               warm);
    if (s < 0) return s;
    if (severity(s) > severity(worst)) worst = s;
  }
  return worst;
}

// bfcs_solve_group: batches of different grids (one plan each) advancing
// together; one graph launch per chunk runs every plan's sweeps side by side.
template <typename R>
int solve_group_impl(int n, const bfcs_group_item* items, int nph, const bfcs_lame* phases, bfcs_lame C0,
                     double tol, int maxit) {
  int e = check_material(nph, phases, C0);
  if (e != BFCS_OK) return e;
  if (!(tol >= 0) || maxit < 0) return BFCS_ERR_INVALID_ARG;
  const PhaseTab<R> tab = make_tab<R>(nph, phases, C0);
  std::vector<SweepSet<R>> sets(n);
  std::vector<SweepSet<R>*> ptrs;
  for (int i = 0; i < n; ++i) {
    bfcs_plan P = items[i].plan;
    const bfcs_problem* pr = items[i].problems;
    const int B = items[i].batch;
    std::vector<Member> mem;
    std::vector<const int8_t*> ph;
    std::vector<const void*> bs;
    bool warm = false;
    for (int m = 0; m < B; ++m) {
      if (pr[m].phase == nullptr || pr[m].b == nullptr || pr[m].eps_out == nullptr) return BFCS_ERR_INVALID_ARG;
      if (pr[m].eps_init != nullptr && maxit < 1) return BFCS_ERR_INVALID_ARG;
      for (int c = 0; c < 6; ++c)
        if (!std::isfinite(pr[m].E[c])) return BFCS_ERR_INVALID_ARG;
      mem.push_back(make_member(pr[m].phase, pr[m].shift, pr[m].E, pr[m].b, pr[m].eps_init,
                                SolveOut{pr[m].eps_out, pr[m].sig_out, pr[m].u_out}));
      ph.push_back(pr[m].phase);
      bs.push_back(pr[m].b);
      warm = warm || pr[m].eps_init != nullptr;
    }
    e = validate_members<R>(P, B, ph.data(), bs.data(), nph);
    if (e != BFCS_OK) return e;
    e = upload_members(P, B, mem.data());
    if (e != BFCS_OK) return e;
    e = transform_members<R>(P, B);
    if (e != BFCS_OK) return e;
    sets[i].prepare(P, B, tab, C0, pr[0].E, tol);
    e = sets[i].init(warm);
    if (e != BFCS_OK) return e;
    ptrs.push_back(&sets[i]);
  }
  e = run_sets<R>(ptrs, maxit);
  if (e != BFCS_OK) return e;
  int worst = BFCS_OK;
  for (int i = 0; i < n; ++i) {
    const int s = sets[i].finalize(items[i].infos);
    if (s < 0) return s;
    if (severity(s) > severity(worst)) worst = s;
  }
  return worst;
}

// FP64 strain and defect from the FP64 displacements (precision ladder) of k
// members in one launch per pass (from_eps: from the FP64 strains instead, see
// below).  The passes compute in float-float (about
// 48 bits, on the FP32 pipes) with float-float spectra; the real fields (u64
// in, eps64 out) are FP64.  Slot j holds member idx[j]; dm[j] (host)
// carries its phase, shift, E, the displacement u64 (as `b`, the real input
// of the x transform) and eps_out.  eps64 = E + sym grad u64 (spectral,
// exactly compatible), sigma = L eps64, its transform, R_hat = i xi .
// sigma_hat + b_hat64[m], the FP64 residual r(eps64) into
// ist64[m].resid_final, and R_hat rounded to complex64 into the member's FP32
// load spectrum (slot m of the plan's b_hat: the load of its correction
// problem, already transformed).  eps64 goes to eps_out.
// from_eps: eps64 is already in dm[j].eps_init (FP64), the strain a previous
// round returned plus the FP32 strain of the correction added since; sigma =
// L eps64 and its transform are formed from it directly (the displacement
// transforms, the symmetric gradient and their inverse are skipped) and no
// strain is written.
int defect_spectrum(bfcs_plan P, int k, const int* idx);
int defect64(bfcs_plan P, int k, const Member* dm, const int* idx, const PhaseTab<ff>& tab, bool from_eps) {
  const Geo g = P->g;
  cudaStream_t st = P->st;
  const long long sms = 6 * g.cs;
  C2<ff>* spec = (C2<ff>*)P->spec64;
  int e = upload_members(P, k, dm);
  if (e != BFCS_OK) return e;
  CArgs<ff> ca{};
  ca.data = spec;
  ca.ms = sms;
  ca.g = g;
  if (from_eps) {
    XArgs<ff> xs{};                                              // sigma = L eps64, R2C
    xs.g = g;
    xs.spec_out = spec;
    xs.spec_ms = sms;
    fill_xm(xs, dm, k, XIN_EPS_INIT, 0);
    xs.tab = tab;
    xs.tw = (const C2<ff>*)P->twff[0];
    xs.ncomp = 6;
    xs.mode = XM_REALSIG;
    CK(launch_xpass_b<ff>(xs, k, st));
    ca.ncomp = 6;
    ca.axis = 1; ca.tw = (const C2<ff>*)P->twff[1];
    CK(launch_colpass_b<ff>(ca, -1, k, st));                    // y forward
    ca.axis = 2; ca.tw = (const C2<ff>*)P->twff[2];
    CK(launch_colpass_b<ff>(ca, -1, k, st));                    // z forward
    return defect_spectrum(P, k, idx);
  }
  XArgs<ff> xa{};                                                // u_hat, x direction
  xa.g = g;
  xa.spec_out = spec;
  xa.spec_ms = sms;
  fill_xm(xa, dm, k, XIN_B, 0);
  xa.ncomp = 3;
  xa.mode = XM_R2C;
  xa.tw = (const C2<ff>*)P->twff[0];
  CK(launch_xpass_b<ff>(xa, k, st));
  ca.ncomp = 3;
  ca.axis = 1; ca.tw = (const C2<ff>*)P->twff[1];
  CK(launch_colpass_b<ff>(ca, -1, k, st));
  ca.axis = 2; ca.tw = (const C2<ff>*)P->twff[2];
  CK(launch_colpass_b<ff>(ca, -1, k, st));
  CK(launch_symgrad<ff>(spec, sms, g, P->mem_dev, k, st));     // eps_hat / N (6 components)
  ca.ncomp = 6;
  CK(launch_colpass_b<ff>(ca, +1, k, st));                      // z inverse
  ca.axis = 1; ca.tw = (const C2<ff>*)P->twff[1];
  CK(launch_colpass_b<ff>(ca, +1, k, st));                      // y inverse
  XArgs<ff> xs{};                                                // eps out, sigma = L eps, R2C
  xs.g = g;
  xs.spec_in = spec;
  xs.spec_out = spec;
  xs.spec_ms = sms;
  fill_xm(xs, dm, k, XIN_NONE, XOUT_EPS);
  xs.tab = tab;
  xs.tw = (const C2<ff>*)P->twff[0];
  xs.ncomp = 6;
  xs.mode = XM_SWEEPSIG;
  CK(launch_xpass_b<ff>(xs, k, st));
  CK(launch_colpass_b<ff>(ca, -1, k, st));                      // y forward
  ca.axis = 2; ca.tw = (const C2<ff>*)P->twff[2];
  CK(launch_colpass_b<ff>(ca, -1, k, st));                      // z forward
  return defect_spectrum(P, k, idx);
}

// R_hat = i xi . sigma_hat + b_hat64 of slot j's member idx[j] from the float-float
// stress spectra in spec64 (slot-major), its residual into ist64, R_hat as complex64
// into the member's slot of the plan's b_hat.
int defect_spectrum(bfcs_plan P, int k, const int* idx) {
  const Geo g = P->g;
  cudaStream_t st = P->st;
  const long long sms = 6 * g.cs;
  C2<ff>* spec = (C2<ff>*)P->spec64;
  DArgs<ff> da{};
  da.spec = spec;
  da.spec_ms = sms;
  da.bhat = (const C2<ff>*)P->bhat64;
  da.b_ms = 3 * g.cs;
  da.out32 = (C2<float>*)P->bhat;
  da.o_ms = 3 * g.cs;
  da.g = g;
  da.part = P->part;
  da.st = P->ist64;
  for (int j = 0; j < k; ++j) da.idx[j] = idx[j];
  const int blocks = 512;
  CK(launch_defect<ff>(da, blocks, k, st));
  const int maxdim = std::max(g.nx, std::max(g.ny, g.nz));
  CK(launch_defect_final(P->part, blocks, P->ist64, idx, k, maxdim, st));
  return BFCS_OK;
}

// FP32 sweeps with FP64 defect correction for B <= max_batch members of one
// grid; every field at the API is FP64 (Member pointers).  The FP64 state of a
// member is its displacement u64, so eps64 = E + sym grad u64 stays exactly
// compatible.
//  Phase 1: one batched FP32 solve of all members to max(tol, switch_tol) (or
//  their stall), cold members from eps^{b(0)} + E, warm members from their
//  eps_init rounded to FP32; u64 = its displacement.
//  Rounds: every unfinished member gets eps64 and its FP64 residual r64 (one
//  batched set of FP64 passes); a member stops when r64 <= tol (or after
//  max_rounds / maxit); the others solve their correction problems (load = the
//  FP64 defect rounded to FP32, E = 0) together in one batched FP32 solve, each
//  to its own relative tolerance 0.5 tol / r64 (at least switch_tol, so that no
//  FP32 solve is asked to go near its rounding floor), and add the correction's
//  displacement (and, at tol >= kIncStrainTol, its strain to eps64, from which
//  the next round's defect is evaluated without re-forming eps64 from u64).
int solve_mixed_batch(bfcs_plan P, int B, const Member* in, int nph, const bfcs_lame* phases, bfcs_lame C0,
                      double tol, int maxit, bfcs_info* infos) {
  int e = check_material(nph, phases, C0);
  if (e != BFCS_OK) return e;
  if (B < 1 || B > P->max_batch || !(tol >= 0) || maxit < 0) return BFCS_ERR_INVALID_ARG;
  std::vector<const int8_t*> phs(B);
  std::vector<const void*> bs(B);
  for (int m = 0; m < B; ++m) {
    if (in[m].phase == nullptr || in[m].b == nullptr || in[m].eps_out == nullptr) return BFCS_ERR_INVALID_ARG;
    for (int c = 0; c < 6; ++c)
      if (!std::isfinite(in[m].E[c])) return BFCS_ERR_INVALID_ARG;
    phs[m] = in[m].phase;
    bs[m] = in[m].b;
  }
  e = validate_members<double>(P, B, phs.data(), bs.data(), nph);
  if (e != BFCS_OK) return e;
  const Geo g = P->g;
  const long long n = g.n;
  const size_t cs = (size_t)g.cs;
  cudaStream_t st = P->st;
  C2<float>* bhat32 = (C2<float>*)P->bhat;
  C2<ff>* bhat64 = (C2<ff>*)P->bhat64;
  auto eps32 = [&](int j) { return P->r32 + (size_t)j * 12 * n + 3 * n; };
  auto u32 = [&](int j) { return P->r32 + (size_t)j * 12 * n + 9 * n; };
  std::vector<double*> u64(B);
  for (int m = 0; m < B; ++m)
    u64[m] = in[m].u_out != nullptr ? (double*)in[m].u_out : P->u64 + (size_t)m * 3 * n;
  const PhaseTab<float> tab32 = make_tab<float>(nph, phases, C0);
  const PhaseTab<double> tab64 = make_tab<double>(nph, phases, C0);
  const PhaseTab<ff> tabff = make_tab<ff>(nph, phases, C0);
  const double zeroE[6] = {0, 0, 0, 0, 0, 0};
  // Above kIncStrainTol the rounds after the first carry eps64 forward by adding
  // each correction's FP32 strain (rounding ~6e-8 of an increment ~1e-3 of the
  // strain, so eps64 stays compatible to ~1e-10) and evaluate the defect from it;
  // below it every round re-forms eps64 = E + sym grad u64 exactly.
  const bool inc_eps = tol >= kIncStrainTol;
  std::vector<int> sweeps(B, 0), stalled(B, 0), status(B, BFCS_OK);
  std::vector<double> r_last(B, INFINITY), r64(B, INFINITY);
  std::vector<char> fin(B, 0);
  std::vector<Member> mem;
  std::vector<bfcs_info> inf(P->max_batch);
  auto shift_of = [&](int m) { return std::array<int, 3>{in[m].sx, in[m].sy, in[m].sz}; };

  // float-float load spectra of all members (slot = member), their complex64
  // copies for the FP32 phases, and their norms (the norm is a normaliser:
  // the complex64 copy carries all the digits it needs)
  CK(cudaMemsetAsync(P->ist64, 0, B * sizeof(IterState), st));
  {
    XArgs<ff> xa{};
    xa.g = g;
    xa.spec_out = bhat64;
    xa.spec_ms = 3 * cs;
    fill_xm(xa, in, B, XIN_B, 0);
    xa.ncomp = 3;
    xa.mode = XM_R2C;
    xa.tw = (const C2<ff>*)P->twff[0];
    CK(launch_xpass_b<ff>(xa, B, st));
    CArgs<ff> ca{};
    ca.data = bhat64;
    ca.ms = 3 * cs;
    ca.g = g;
    ca.ncomp = 3;
    ca.axis = 1; ca.tw = (const C2<ff>*)P->twff[1];
    CK(launch_colpass_b<ff>(ca, -1, B, st));
    ca.axis = 2; ca.tw = (const C2<ff>*)P->twff[2];
    CK(launch_colpass_b<ff>(ca, -1, B, st));
    CK(launch_cast_spec_ff(bhat32, bhat64, g, 3 * B, st));
    CK(launch_bden<float>(bhat32, g, P->part, P->ist64, st, B, 3 * cs));
  }

  // phase 1: all members, FP32
  bool any_warm = false;
  mem.clear();
  for (int m = 0; m < B; ++m) {
    const void* init = nullptr;
    if (in[m].eps_init != nullptr) {
      CK(launch_cast_d2f(eps32(m), (const double*)in[m].eps_init, 6 * n, st));
      init = eps32(m);
      any_warm = true;
    }
    const auto sh = shift_of(m);
    // the ladder carries the FP32 phases' displacement only: their strain is not written
    mem.push_back(make_member(in[m].phase, sh.data(), in[m].E, nullptr, init, SolveOut{nullptr, nullptr, u32(m)}));
  }
  CK(launch_bden<float>(bhat32, g, P->part, P->ist, st, B, 3 * cs));
  e = upload_members(P, B, mem.data());
  if (e != BFCS_OK) return e;
  // (the ladder's FP32 solves need the displacement and strain only: no final pass)
  const int s1 = run_batch<float>(P, B, tab32, C0, in[0].E, std::max(tol, P->switch_tol), maxit, inf.data(),
                                  any_warm, true);
  if (s1 < 0) return s1;
  for (int m = 0; m < B; ++m) {
    sweeps[m] += inf[m].iters;
    r_last[m] = inf[m].resid;
    CK(launch_cast_f2d(u64[m], u32(m), 3 * n, st));
  }

  for (int round = 0;; ++round) {
    std::vector<int> act;
    for (int m = 0; m < B; ++m)
      if (!fin[m]) act.push_back(m);
    if (act.empty()) break;
    mem.clear();
    // defect inputs: u64 as the real input, eps64 out; after a correction with
    // strain increments, eps64 (already updated) as the input
    const bool from_eps = inc_eps && round > 0;
    for (int m : act) {
      const auto sh = shift_of(m);
      mem.push_back(from_eps ? make_member(in[m].phase, sh.data(), in[m].E, nullptr, in[m].eps_out, SolveOut{})
                             : make_member(in[m].phase, sh.data(), in[m].E, u64[m], nullptr,
                                           SolveOut{in[m].eps_out, nullptr, nullptr}));
    }
    e = defect64(P, (int)act.size(), mem.data(), act.data(), tabff, from_eps);
    if (e != BFCS_OK) return e;
    IterState* h64 = P->ist_host + 2 * P->max_batch;
    CK(read_small(h64, P->ist64, B * sizeof(IterState), st));
    const int w = sync_stream(P);
    if (w != BFCS_OK) return w;
    std::vector<int> next;
    for (int m : act) {
      r64[m] = h64[m].resid_final;
      if (!std::isfinite(r64[m])) { status[m] = BFCS_ERR_DIVERGED; fin[m] = 1; continue; }
      if (r64[m] <= tol || round >= P->max_rounds || sweeps[m] >= maxit) { fin[m] = 1; continue; }
      next.push_back(m);
    }
    if (next.empty()) break;
    // correction problems of the unfinished members, packed into slots 0..k-1
    const int k = (int)next.size();
    int left = maxit;
    mem.clear();
    for (int j = 0; j < k; ++j) {
      const int m = next[j];
      if (j != m)   // j < m: slot j's own spectrum is no longer needed
        CK(cudaMemcpyAsync(bhat32 + (size_t)j * 3 * cs, bhat32 + (size_t)m * 3 * cs, 3 * cs * sizeof(C2<float>),
                           cudaMemcpyDeviceToDevice, st));
      const auto sh = shift_of(m);
      Member c = make_member(in[m].phase, sh.data(), zeroE, nullptr, nullptr,
                             SolveOut{inc_eps ? eps32(j) : nullptr, nullptr, u32(j)});
      c.tol = std::min(0.5, std::max(0.5 * tol / r64[m], P->switch_tol));   // well above the FP32 floor
      mem.push_back(c);
      left = std::min(left, maxit - sweeps[m]);
    }
    CK(launch_bden<float>(bhat32, g, P->part, P->ist, st, k, 3 * cs));
    e = upload_members(P, k, mem.data());
    if (e != BFCS_OK) return e;
    const int s2 = run_batch<float>(P, k, tab32, C0, zeroE, 0.5, std::max(left, 1), inf.data(), false, true);
    if (s2 < 0) return s2;
    for (int j = 0; j < k; ++j) {
      const int m = next[j];
      sweeps[m] += inf[j].iters;
      stalled[m] = inf[j].stalled;
      CK(launch_add_f2d(u64[m], u32(j), 3 * n, st));
      if (inc_eps) CK(launch_add_f2d((double*)in[m].eps_out, eps32(j), 6 * n, st));
    }
  }
  for (int m = 0; m < B; ++m)
    if (in[m].sig_out != nullptr)
      CK(launch_stress((double*)in[m].sig_out, (const double*)in[m].eps_out, in[m].phase, tab64, in[m].sx,
                       in[m].sy, in[m].sz, g.nx, g.ny, g.nz, st));
  const int w = sync_stream(P);
  if (w != BFCS_OK) return w;
  P->last_iters = 0;     // history of the FP32 phases is not kept across rounds
  int worst = BFCS_OK;
  for (int m = 0; m < B; ++m) {
    if (status[m] == BFCS_OK && !(r64[m] <= tol)) status[m] = BFCS_NOT_CONVERGED;
    if (infos != nullptr) {
      infos[m].iters = sweeps[m];
      infos[m].status = status[m];
      infos[m].resid = r64[m];
      infos[m].resid_prev = r_last[m];
      infos[m].precision_path = 2;
      infos[m].stalled = stalled[m];
    }
    if (severity(status[m]) > severity(worst)) worst = status[m];
  }
  return worst;
}

// One member through the batched ladder.
int solve_mixed(bfcs_plan P, const int8_t* phase, int nph, const bfcs_lame* phases, bfcs_lame C0,
                const void* b, const double* E, double tol, int maxit, const void* eps_init, SolveOut out,
                const int shift[3], bfcs_info* info) {
  if (E == nullptr || out.eps == nullptr || phase == nullptr || b == nullptr) return BFCS_ERR_INVALID_ARG;
  const Member m = make_member(phase, shift, E, b, eps_init, out);
  return solve_mixed_batch(P, 1, &m, nph, phases, C0, tol, maxit, info);
}

int ensure_tmp(bfcs_plan P) {
  if (P->tmp == nullptr) {
    const size_t members = (size_t)P->max_batch;
    if (cudaMalloc(&P->tmp, members * 15 * (size_t)P->g.n * P->rsz) != cudaSuccess) return BFCS_ERR_OOM;
  }
  if (P->tmp_hits == nullptr) {
    if (cudaMalloc(&P->tmp_hits, (size_t)P->g.n * sizeof(int)) != cudaSuccess) return BFCS_ERR_OOM;
  }
  return BFCS_OK;
}

// Member m of an averaging run: its phase map (the shared one translated by
// shift m, Eqs. 3.3-3.6, or configuration m of an ensemble, Eq. 3.8).
struct AvgMembers {
  const int8_t* phase;                // shared phase map (translations) or nullptr
  const int8_t* const* configs;       // host array of configuration phase maps or nullptr
  const int32_t* shifts;              // host, 3 per member, or nullptr (no translation)
  const int8_t* phase_of(int m) const { return configs != nullptr ? configs[m] : phase; }
  void shift_of(int m, int out[3]) const {
    for (int a = 0; a < 3; ++a) out[a] = shifts != nullptr ? shifts[3 * m + a] : 0;
  }
};

// Averages over `count` members with the load b fixed: u, V u, eps, V eps,
// sigma, V sigma summed in FP64 and divided by count (V = phase != 0 of the
// member's own phase map), max_batch members per batched solve.
template <typename R>
int average_impl(bfcs_plan P, int count, const AvgMembers& am, int nph, const bfcs_lame* phases, bfcs_lame C0,
                 const void* b, const double* E, double tol, int maxit, double* avg, int32_t* hits,
                 bfcs_info* infos) {
  int e = check_material(nph, phases, C0);
  if (e != BFCS_OK) return e;
  if (b == nullptr || E == nullptr || avg == nullptr || count < 1 || !(tol >= 0) || maxit < 0)
    return BFCS_ERR_INVALID_ARG;
  for (int m = 0; m < count; ++m)
    if (am.phase_of(m) == nullptr) return BFCS_ERR_INVALID_ARG;
  e = ensure_tmp(P);
  if (e != BFCS_OK) return e;
  if (am.configs == nullptr) {
    e = validate_inputs<R>(P, am.phase, b, nph);
    if (e != BFCS_OK) return e;
  }
  const long long n = P->g.n;
  int* h = hits != nullptr ? (int*)hits : P->tmp_hits;
  CK(cudaMemsetAsync(avg, 0, 30 * n * sizeof(double), P->st));
  CK(cudaMemsetAsync(h, 0, n * sizeof(int), P->st));
  const PhaseTab<R> tab = make_tab<R>(nph, phases, C0);
  int worst = BFCS_OK;
  std::vector<Member> mem;
  for (int start = 0; start < count; start += P->max_batch) {
    const int B = std::min(P->max_batch, count - start);
    if (am.configs != nullptr) {
      const std::vector<const void*> bs(B, b);
      e = validate_members<R>(P, B, am.configs + start, bs.data(), nph);
      if (e != BFCS_OK) return e;
    }
    mem.clear();
    for (int m = 0; m < B; ++m) {
      R* eps = (R*)P->tmp + (size_t)m * 15 * n;
      int shv[3];
      am.shift_of(start + m, shv);
      mem.push_back(make_member(am.phase_of(start + m), shv, E, b, nullptr,
                                SolveOut{eps, eps + 6 * n, eps + 12 * n}));
    }
    e = upload_members(P, B, mem.data());
    if (e != BFCS_OK) return e;
    e = transform_members<R>(P, B);            // b is fixed (Eq. 3.4)
    if (e != BFCS_OK) return e;
    const int s = run_batch<R>(P, B, tab, C0, E, tol, maxit, infos != nullptr ? infos + start : nullptr, false);
    if (s < 0) return s;
    if (severity(s) > severity(worst)) worst = s;
    for (int m = 0; m < B; ++m) {
      const R* eps = (const R*)P->tmp + (size_t)m * 15 * n;
      CK(launch_accumulate<R>(avg, h, eps, eps + 6 * n, eps + 12 * n, mem[m].phase, mem[m].sx, mem[m].sy,
                              mem[m].sz, P->g.nx, P->g.ny, P->g.nz, P->st));
    }
  }
  CK(launch_scale(avg, 30 * n, 1.0 / count, P->st));
  const int w = sync_stream(P);
  return w != BFCS_OK ? w : worst;
}

// The same through the batched precision ladder (fields in FP64).
int average_mixed(bfcs_plan P, int count, const AvgMembers& am, int nph, const bfcs_lame* phases,
                  bfcs_lame C0, const void* b, const double* E, double tol, int maxit, double* avg,
                  int32_t* hits, bfcs_info* infos) {
  if (avg == nullptr || count < 1 || E == nullptr || b == nullptr) return BFCS_ERR_INVALID_ARG;
  for (int m = 0; m < count; ++m)
    if (am.phase_of(m) == nullptr) return BFCS_ERR_INVALID_ARG;
  int e = ensure_tmp(P);
  if (e != BFCS_OK) return e;
  const long long n = P->g.n;
  int* h = hits != nullptr ? (int*)hits : P->tmp_hits;
  CK(cudaMemsetAsync(avg, 0, 30 * n * sizeof(double), P->st));
  CK(cudaMemsetAsync(h, 0, n * sizeof(int), P->st));
  int worst = BFCS_OK;
  std::vector<Member> mem;
  for (int start = 0; start < count; start += P->max_batch) {   // the batched ladder, max_batch members at a time
    const int B = std::min(P->max_batch, count - start);
    mem.clear();
    for (int m = 0; m < B; ++m) {
      double* eps = (double*)P->tmp + (size_t)m * 15 * n;
      int shv[3];
      am.shift_of(start + m, shv);
      mem.push_back(make_member(am.phase_of(start + m), shv, E, b, nullptr,
                                SolveOut{eps, eps + 6 * n, eps + 12 * n}));
    }
    const int s = solve_mixed_batch(P, B, mem.data(), nph, phases, C0, tol, maxit,
                                    infos != nullptr ? infos + start : nullptr);
    if (s < 0) return s;
    if (severity(s) > severity(worst)) worst = s;
    for (int m = 0; m < B; ++m) {
      const double* eps = (const double*)mem[m].eps_out;
      CK(launch_accumulate<double>(avg, h, eps, eps + 6 * n, eps + 12 * n, mem[m].phase, mem[m].sx, mem[m].sy,
                                   mem[m].sz, P->g.nx, P->g.ny, P->g.nz, P->st));
    }
  }
  CK(launch_scale(avg, 30 * n, 1.0 / count, P->st));
  const int w = sync_stream(P);
  return w != BFCS_OK ? w : worst;
}

int average_dispatch(bfcs_plan P, int count, const AvgMembers& am, int nph, const bfcs_lame* phases,
                     bfcs_lame C0, const void* b, const double* E, double tol, int maxit, double* avg,
                     int32_t* hits, bfcs_info* infos) {
  if (P == nullptr) return BFCS_ERR_INVALID_ARG;
  if (P->mixed) return average_mixed(P, count, am, nph, phases, C0, b, E, tol, maxit, avg, hits, infos);
  return P->fp64 ? average_impl<double>(P, count, am, nph, phases, C0, b, E, tol, maxit, avg, hits, infos)
                 : average_impl<float>(P, count, am, nph, phases, C0, b, E, tol, maxit, avg, hits, infos);
}

// Effective stiffness L* (<sigma> = L* <eps>, Eqs. 6.1-6.3) and inclusion strain
// concentration A* (<eps>_i = A* <eps>, Eq. 3.2): the classical problem (b = 0)
// under the six unit mean strains, min(max_batch, 6) members at a time; column
// J of both matrices is the response to unit tensorial strain J.  The members'
// fields sit in the plan's scratch: eps, sigma, and in the displacement slot
// the zero load (no displacement is formed).
template <typename R>
int moduli_impl(bfcs_plan P, const int8_t* phase, int nph, const bfcs_lame* phases, bfcs_lame C0, double tol,
                int maxit, double* Lstar, double* Astar, bfcs_info* infos) {
  if (phase == nullptr || Lstar == nullptr) return BFCS_ERR_INVALID_ARG;
  int e = ensure_tmp(P);
  if (e != BFCS_OK) return e;
  if (P->mod_buf == nullptr &&
      cudaMalloc(&P->mod_buf, (size_t)kModMembers * (kModParts + 1) * kModSums * sizeof(double)) != cudaSuccess)
    return BFCS_ERR_OOM;
  const long long n = P->g.n;
  double* part = P->mod_buf;
  double* sums = P->mod_buf + (size_t)kModMembers * kModParts * kModSums;
  const int chunk = std::min(P->max_batch, kModMembers);
  int worst = BFCS_OK;
  for (int start = 0; start < kModMembers; start += chunk) {
    const int B = std::min(chunk, kModMembers - start);
    bfcs_problem pr[kModMembers];
    ModArgs<R> ma{};
    for (int m = 0; m < B; ++m) {
      R* eps = (R*)P->tmp + (size_t)m * 15 * n;
      R* b = eps + 12 * n;
      CK(cudaMemsetAsync(b, 0, 3 * n * sizeof(R), P->st));
      bfcs_problem& q = pr[m];
      std::memset(&q, 0, sizeof(q));
      q.phase = phase;
      q.b = b;
      q.E[start + m] = 1.0;
      q.eps_out = eps;
      q.sig_out = eps + 6 * n;
      ma.eps[m] = eps;
      ma.sig[m] = eps + 6 * n;
    }
    ma.phase = phase;
    ma.n = n;
    const int s = bfcs_solve_batched(P, B, pr, nph, phases, C0, tol, maxit, infos != nullptr ? infos + start : nullptr);
    if (s < 0) return s;
    if (severity(s) > severity(worst)) worst = s;
    CK(launch_moduli<R>(ma, B, part, sums + (size_t)start * kModSums, P->st));
  }
  double host[kModMembers * kModSums];
  CK(cudaMemcpyAsync(host, sums, sizeof(host), cudaMemcpyDeviceToHost, P->st));
  const int w = sync_stream(P);
  if (w != BFCS_OK) return w;
  for (int J = 0; J < 6; ++J) {
    const double* h = host + J * kModSums;
    for (int I = 0; I < 6; ++I) {
      Lstar[I * 6 + J] = h[I] / (double)n;
      if (Astar != nullptr) Astar[I * 6 + J] = h[12] > 0.0 ? h[6 + I] / h[12] : std::nan("");
    }
  }
  return worst;
}

}  // namespace

extern "C" {

const char* bfcs_status_string(int s) {
  switch (s) {
    case BFCS_OK: return "ok";
    case BFCS_NOT_CONVERGED: return "not converged within maxit";
    case BFCS_ERR_INVALID_ARG: return "invalid argument";
    case BFCS_ERR_NONZERO_MEAN: return "body force is not mean-free (Eq. 2.5)";
    case BFCS_ERR_OOM: return "out of device memory";
    case BFCS_ERR_CUDA: return "CUDA runtime error";
    case BFCS_ERR_TIMEOUT: return "bounded wait expired";
    case BFCS_ERR_DIVERGED: return "residual is NaN or Inf";
    case BFCS_ERR_UNSUPPORTED: return "not supported by this build";
    default: return "unknown status";
  }
}

int bfcs_plan_create(bfcs_plan* out, int nx, int ny, int nz, int max_batch, int flags, void* stream) {
  if (out == nullptr) return BFCS_ERR_INVALID_ARG;
  *out = nullptr;
  const int prec = flags & 3;
  if (!supported_len(nx) || !supported_len(ny) || !supported_len(nz) || max_batch < 1 || max_batch > kMaxBatch ||
      (prec != BFCS_FP32 && prec != BFCS_FP64 && prec != BFCS_MIXED) ||
      (flags & ~(3 | BFCS_AUTOTUNE | BFCS_CG | BFCS_SPARSE_RESID | BFCS_CD | BFCS_CD_PRECOND)) != 0 ||
      ((flags & BFCS_CG) && (flags & (BFCS_CD | BFCS_CD_PRECOND))))
    return BFCS_ERR_INVALID_ARG;
  bfcs_plan P = new bfcs_plan_s();
  P->nx = nx; P->ny = ny; P->nz = nz;
  P->max_batch = max_batch;
  P->flags = flags;
  P->fp64 = prec == BFCS_FP64;
  P->mixed = prec == BFCS_MIXED;
  P->st = (cudaStream_t)stream;
  P->g.nx = nx; P->g.ny = ny; P->g.nz = nz;
  P->g.mx = nx / 2 + 1;
  P->g.p = (nx / 2 + 1 + 3) / 4 * 4;
  P->g.cs = (long long)nz * ny * P->g.p;
  P->g.n = (long long)nx * ny * nz;
  P->csz = P->fp64 ? sizeof(C2<double>) : sizeof(C2<float>);
  P->rsz = (P->fp64 || P->mixed) ? sizeof(double) : sizeof(float);
  P->ev[0] = P->ev[1] = nullptr;
  P->order_ev[0] = P->order_ev[1] = nullptr;
  bool ok = cudaEventCreateWithFlags(&P->ev[0], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&P->ev[1], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&P->order_ev[0], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&P->order_ev[1], cudaEventDisableTiming) == cudaSuccess &&
            cudaStreamCreateWithFlags(&P->loop_st, cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) { free_plan(P); return BFCS_ERR_CUDA; }
  const size_t cs = (size_t)P->g.cs;
  P->ngreen = P->fp64 ? green_nparts<double>(P->g) : green_nparts<float>(P->g);
  P->npart = std::max(P->ngreen, 512);
  const size_t MB = (size_t)max_batch;
  ok = cudaMalloc(&P->spec, MB * 6 * cs * P->csz) == cudaSuccess &&
       cudaMalloc(&P->bhat, MB * 3 * cs * P->csz) == cudaSuccess &&
       cudaMalloc(&P->dprev, MB * 3 * cs * P->csz) == cudaSuccess &&
       cudaMalloc(&P->part, MB * P->npart * sizeof(ResidSlot)) == cudaSuccess &&
       cudaMalloc(&P->ist, MB * sizeof(IterState)) == cudaSuccess &&
       cudaMalloc(&P->io_dev, 2 * sizeof(unsigned long long)) == cudaSuccess &&
       cudaMalloc(&P->hist, MB * kHistCap * sizeof(double)) == cudaSuccess &&
       cudaMalloc(&P->mem_dev, MB * sizeof(Member)) == cudaSuccess &&
       cudaMallocHost(&P->mem_host, MB * sizeof(Member)) == cudaSuccess &&
       cudaMalloc(&P->ival, MB * 2 * sizeof(int)) == cudaSuccess &&
       cudaMalloc(&P->dval, MB * 6 * sizeof(double)) == cudaSuccess &&
       cudaMalloc(&P->dscratch, std::max(validate_scratch(P->g.n), body_force_scratch(P->g.n)) *
                                    sizeof(double)) == cudaSuccess &&
       cudaMallocHost(&P->ist_host, 3 * MB * sizeof(IterState)) == cudaSuccess &&
       cudaMallocHost(&P->ival_host, MB * 2 * sizeof(int)) == cudaSuccess &&
       cudaMallocHost(&P->dval_host, MB * 6 * sizeof(double)) == cudaSuccess;
  if (!ok) { cudaGetLastError(); free_plan(P); return BFCS_ERR_OOM; }
  P->hist_cap = kHistCap;
  const int dims[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a) {
    P->tw[a] = P->fp64 ? make_twiddles<double>(dims[a]) : make_twiddles<float>(dims[a]);
    if (P->tw[a] == nullptr) { free_plan(P); return BFCS_ERR_OOM; }
  }
  if (P->mixed) {
    ok = cudaMalloc(&P->spec64, MB * 6 * cs * sizeof(C2<double>)) == cudaSuccess &&
         cudaMalloc(&P->bhat64, MB * 3 * cs * sizeof(C2<double>)) == cudaSuccess &&
         cudaMalloc(&P->ist64, MB * sizeof(IterState)) == cudaSuccess &&
         cudaMalloc(&P->r32, MB * 12 * (size_t)P->g.n * sizeof(float)) == cudaSuccess &&
         cudaMalloc(&P->u64, MB * 3 * (size_t)P->g.n * sizeof(double)) == cudaSuccess;
    if (!ok) { cudaGetLastError(); free_plan(P); return BFCS_ERR_OOM; }
    for (int a = 0; a < 3; ++a) {
      P->tw64[a] = make_twiddles<double>(dims[a]);
      P->twff[a] = make_twiddles<ff>(dims[a]);
      if (P->tw64[a] == nullptr || P->twff[a] == nullptr) { free_plan(P); return BFCS_ERR_OOM; }
    }
  }
  if (flags & (BFCS_CD | BFCS_CD_PRECOND)) {   // u1, r, p, q (and z) vectors of 3 components in cg_vec
    P->use_cd = true;
    P->cd_precond = (flags & BFCS_CD_PRECOND) ? 1 : 0;
    ok = cudaMalloc(&P->cd_part, MB * 2 * (size_t)cd_parts(P->g) * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&P->cd_state, MB * sizeof(CdState)) == cudaSuccess &&
         cudaMallocHost(&P->cd_host, MB * sizeof(CdState)) == cudaSuccess;
    if (!ok) { cudaGetLastError(); free_plan(P); return BFCS_ERR_OOM; }
  }
  if (flags & (BFCS_CG | BFCS_CD | BFCS_CD_PRECOND)) {
    P->use_cg = (flags & BFCS_CG) != 0;
    ok = cudaMalloc(&P->cg_vec, 4 * MB * 6 * cs * P->csz) == cudaSuccess &&
         cudaMalloc(&P->cg_part, MB * kCgParts * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&P->cg_state, MB * sizeof(CgState)) == cudaSuccess &&
         cudaMalloc(&P->cg_skip, MB * sizeof(IterState)) == cudaSuccess &&
         cudaMallocHost(&P->cg_host, MB * sizeof(CgState)) == cudaSuccess;
    if (!ok) { cudaGetLastError(); free_plan(P); return BFCS_ERR_OOM; }
  }
  if (cudaMemset(P->ist, 0, MB * sizeof(IterState)) != cudaSuccess ||
      cudaMemset(P->io_dev, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) {
    free_plan(P);
    return BFCS_ERR_CUDA;
  }
  if (const char* gs = std::getenv("BFCS_GRAPH_SWEEPS")) P->graph_sweeps = std::max(0, std::atoi(gs));
  if (flags & BFCS_SPARSE_RESID) {
    P->resid_max = kSparseResidMax;
    if (const char* ri = std::getenv("BFCS_RESID_INTERVAL")) P->resid_max = std::max(1, std::min(64, std::atoi(ri)));
  }
  if (!P->fp64) P->tmap_ok = encode_spectrum_map(P);
  if (!P->fp64) {
    const char* cv = std::getenv("BFCS_COL_VARIANT");
    if (cv != nullptr) {
      const int v = std::atoi(cv);
      P->col_variant = col_variant_valid(v, ny) && (!col_variant_tma(v) || P->tmap_ok) ? v : 0;
    } else if (flags & BFCS_AUTOTUNE) {
      const int e = autotune(P);
      if (e != BFCS_OK) { free_plan(P); return e; }
    }
  }
  *out = P;
  return BFCS_OK;
}

int bfcs_plan_destroy(bfcs_plan P) {
  if (P == nullptr) return BFCS_ERR_INVALID_ARG;
  cudaStreamSynchronize(P->st);
  free_plan(P);
  return BFCS_OK;
}

int bfcs_voxelize(int nx, int ny, int nz, int cx, int cy, int cz, int nsph, const int32_t* spheres,
                  int8_t* phase_out, void* stream) {
  if (nx < 1 || ny < 1 || nz < 1 || cx < 1 || cy < 1 || cz < 1 || nx % cx || ny % cy || nz % cz ||
      nsph < 0 || (nsph > 0 && spheres == nullptr) || phase_out == nullptr)
    return BFCS_ERR_INVALID_ARG;
  for (int k = 0; k < nsph; ++k) {
    const int32_t* S = spheres + 5 * k;
    if (S[3] < 0 || S[4] < -128 || S[4] > 127) return BFCS_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int* d = nullptr;
  cudaError_t e = cudaSuccess;
  if (nsph > 0) {
    if (cudaMallocAsync((void**)&d, sizeof(int) * 5 * nsph, st) != cudaSuccess) return BFCS_ERR_OOM;
    e = cudaMemcpyAsync(d, spheres, sizeof(int) * 5 * nsph, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) e = launch_voxelize(phase_out, nx, ny, nz, cx, cy, cz, d, nsph, st);
  // the sphere table is released on every path, failed launches included
  if (d != nullptr && cudaFreeAsync(d, st) != cudaSuccess) return BFCS_ERR_CUDA;
  return e == cudaSuccess ? BFCS_OK : BFCS_ERR_CUDA;
}

int bfcs_body_force(int nx, int ny, int nz, double cx, double cy, double cz, double a, int precision,
                    void* b_out, void* stream) {
  if (nx < 1 || ny < 1 || nz < 1 || !(a > 0) || b_out == nullptr ||
      (precision != BFCS_FP32 && precision != BFCS_FP64) || !std::isfinite(cx) || !std::isfinite(cy) ||
      !std::isfinite(cz))
    return BFCS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const long long n = (long long)nx * ny * nz;
  double* scratch = nullptr;
  if (cudaMallocAsync((void**)&scratch, sizeof(double) * body_force_scratch(n), st) != cudaSuccess)
    return BFCS_ERR_OOM;
  cudaError_t e = precision == BFCS_FP64
                      ? launch_body_force<double>((double*)b_out, nx, ny, nz, cx, cy, cz, a, scratch, st)
                      : launch_body_force<float>((float*)b_out, nx, ny, nz, cx, cy, cz, a, scratch, st);
  // the scratch is released on every path, a failed launch included
  if (cudaFreeAsync(scratch, st) != cudaSuccess) return BFCS_ERR_CUDA;
  return e == cudaSuccess ? BFCS_OK : BFCS_ERR_CUDA;
}

int bfcs_solve(bfcs_plan P, const int8_t* phase, int nph, const bfcs_lame* phases, bfcs_lame C0,
               const void* b, const double E[6], double tol, int maxit, const void* eps_init,
               void* eps_out, void* sig_out, void* u_out, bfcs_info* info) {
  if (P == nullptr) return BFCS_ERR_INVALID_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  const int shift[3] = {0, 0, 0};
  const SolveOut out{eps_out, sig_out, u_out};
  const int s = P->mixed ? solve_mixed(P, phase, nph, phases, C0, b, E, tol, maxit, eps_init, out, shift,
                                       info)
                : P->fp64 ? solve_impl<double>(P, phase, nph, phases, C0, b, E, tol, maxit, eps_init, out,
                                               shift, info)
                          : solve_impl<float>(P, phase, nph, phases, C0, b, E, tol, maxit, eps_init, out,
                                              shift, info);
  if (info != nullptr) {
    info->status = s;
    info->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return s;
}

int bfcs_solve_batched(bfcs_plan P, int batch, const bfcs_problem* pr, int nph, const bfcs_lame* phases,
                       bfcs_lame C0, double tol, int maxit, bfcs_info* infos) {
  if (P == nullptr || batch < 0 || (batch > 0 && pr == nullptr)) return BFCS_ERR_INVALID_ARG;
  if (batch == 0) return BFCS_OK;
  const auto t0 = std::chrono::steady_clock::now();
  if (!P->mixed) {
    const int s = P->fp64 ? solve_batch_impl<double>(P, batch, pr, nph, phases, C0, tol, maxit, infos)
                          : solve_batch_impl<float>(P, batch, pr, nph, phases, C0, tol, maxit, infos);
    if (infos != nullptr) {
      const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      for (int m = 0; m < batch; ++m) infos[m].ms = ms;
    }
    return s;
  }
  int worst = BFCS_OK;
  std::vector<Member> mem;
  for (int start = 0; start < batch; start += P->max_batch) {   // the ladder, max_batch members at a time
    const int B = std::min(P->max_batch, batch - start);
    mem.clear();
    for (int m = start; m < start + B; ++m)
      mem.push_back(make_member(pr[m].phase, pr[m].shift, pr[m].E, pr[m].b, pr[m].eps_init,
                                SolveOut{pr[m].eps_out, pr[m].sig_out, pr[m].u_out}));
    const int s = solve_mixed_batch(P, B, mem.data(), nph, phases, C0, tol, maxit,
                                    infos != nullptr ? infos + start : nullptr);
    if (s < 0) return s;
    if (severity(s) > severity(worst)) worst = s;
  }
  if (infos != nullptr) {
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (int m = 0; m < batch; ++m) infos[m].ms = ms;
  }
  return worst;
}

int bfcs_solve_group(int nitems, const bfcs_group_item* items, int nph, const bfcs_lame* phases, bfcs_lame C0,
                     double tol, int maxit) {
  if (nitems < 1 || nitems > BFCS_MAX_GROUP || items == nullptr) return BFCS_ERR_INVALID_ARG;
  for (int i = 0; i < nitems; ++i) {
    const bfcs_plan P = items[i].plan;
    if (P == nullptr || items[i].batch < 1 || items[i].batch > P->max_batch || items[i].problems == nullptr)
      return BFCS_ERR_INVALID_ARG;
    if (P->mixed) return BFCS_ERR_UNSUPPORTED;
    if (P->fp64 != items[0].plan->fp64) return BFCS_ERR_INVALID_ARG;
    for (int k = 0; k < i; ++k)
      if (items[k].plan == P) return BFCS_ERR_INVALID_ARG;
  }
  const auto t0 = std::chrono::steady_clock::now();
  const int s = items[0].plan->fp64 ? solve_group_impl<double>(nitems, items, nph, phases, C0, tol, maxit)
                                    : solve_group_impl<float>(nitems, items, nph, phases, C0, tol, maxit);
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < nitems; ++i)
    if (items[i].infos != nullptr)
      for (int m = 0; m < items[i].batch; ++m) items[i].infos[m].ms = ms;
  return s;
}

int bfcs_translate_average(bfcs_plan P, const int8_t* phase, int nph, const bfcs_lame* phases,
                           bfcs_lame C0, const void* b, const double E[6], int nshift,
                           const int32_t* shifts, double tol, int maxit, double* avg_out,
                           int32_t* hits_out, bfcs_info* infos) {
  if (phase == nullptr || shifts == nullptr) return BFCS_ERR_INVALID_ARG;
  const AvgMembers am{phase, nullptr, shifts};
  return average_dispatch(P, nshift, am, nph, phases, C0, b, E, tol, maxit, avg_out, hits_out, infos);
}

int bfcs_ensemble_average(bfcs_plan P, int nconf, const int8_t* const* configs, int nph, const bfcs_lame* phases,
                          bfcs_lame C0, const void* b, const double E[6], double tol, int maxit, double* avg_out,
                          int32_t* hits_out, bfcs_info* infos) {
  if (configs == nullptr) return BFCS_ERR_INVALID_ARG;
  const AvgMembers am{nullptr, configs, nullptr};
  return average_dispatch(P, nconf, am, nph, phases, C0, b, E, tol, maxit, avg_out, hits_out, infos);
}

int bfcs_effective_stiffness(bfcs_plan P, const int8_t* phase, int nph, const bfcs_lame* phases, bfcs_lame C0,
                             double tol, int maxit, double* Lstar, double* Astar, bfcs_info* infos) {
  if (P == nullptr) return BFCS_ERR_INVALID_ARG;
  return P->fp64 || P->mixed ? moduli_impl<double>(P, phase, nph, phases, C0, tol, maxit, Lstar, Astar, infos)
                             : moduli_impl<float>(P, phase, nph, phases, C0, tol, maxit, Lstar, Astar, infos);
}

int bfcs_radial_profile(bfcs_plan P, const void* field, int ncomp, const double centre[3], int nbins,
                        double* prof_out, int64_t* counts_out) {
  if (P == nullptr || field == nullptr || centre == nullptr || prof_out == nullptr || (ncomp != 3 && ncomp != 6) ||
      nbins < 1 || nbins > kMaxShells)
    return BFCS_ERR_INVALID_ARG;
  const int dims[3] = {P->g.nx, P->g.ny, P->g.nz};
  int c2[3];
  for (int a = 0; a < 3; ++a) {
    const double t = 2.0 * centre[a];
    if (!std::isfinite(t) || std::fabs(t - std::nearbyint(t)) > 1e-9 || std::fabs(t) > 1e9) return BFCS_ERR_INVALID_ARG;
    const long long m = 2LL * dims[a];
    c2[a] = (int)((((long long)std::nearbyint(t)) % m + m) % m);
  }
  if (P->prof_buf == nullptr &&
      cudaMalloc(&P->prof_buf, 2 * (size_t)kMaxShells * sizeof(unsigned long long)) != cudaSuccess)
    return BFCS_ERR_OOM;
  CK(cudaMemsetAsync(P->prof_buf, 0, 2 * (size_t)nbins * sizeof(unsigned long long), P->st));
  if (P->fp64 || P->mixed)
    CK(launch_radial_max<double>((const double*)field, ncomp, dims[0], dims[1], dims[2], c2, nbins, P->prof_buf,
                                 P->prof_buf + nbins, P->st));
  else
    CK(launch_radial_max<float>((const float*)field, ncomp, dims[0], dims[1], dims[2], c2, nbins, P->prof_buf,
                                P->prof_buf + nbins, P->st));
  std::vector<unsigned long long> h(2 * (size_t)nbins);
  CK(cudaMemcpyAsync(h.data(), P->prof_buf, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, P->st));
  const int w = sync_stream(P);
  if (w != BFCS_OK) return w;
  for (int k = 0; k < nbins; ++k) {
    double v;
    std::memcpy(&v, &h[k], sizeof(v));
    prof_out[k] = v;
    if (counts_out != nullptr) counts_out[k] = (int64_t)h[nbins + k];
  }
  return BFCS_OK;
}

int bfcs_plan_tuning(bfcs_plan P, int* col_variant, int* col_tile, int* col_swap, double* variant_ms) {
  if (P == nullptr) return BFCS_ERR_INVALID_ARG;
  if (col_variant) *col_variant = P->col_variant;
  if (col_tile) *col_tile = col_variant_tile(P->col_variant);
  if (col_swap) *col_swap = col_variant_swap(P->col_variant) ? 1 : 0;
  if (variant_ms)
    for (int v = 0; v < kColVariants; ++v) variant_ms[v] = P->col_variant_ms[v];
  return BFCS_OK;
}

int bfcs_surrogate_infer(bfcs_plan P, const void* weights, const void* b, const int8_t* phase, int nph,
                         const bfcs_lame* phases, void* eps_pred) {
  if (P == nullptr || weights == nullptr || b == nullptr || phase == nullptr || eps_pred == nullptr)
    return BFCS_ERR_INVALID_ARG;
  if (P->net == nullptr) {
    const int s = bfcs_net_create(&P->net, P->nx, P->ny, P->nz, 1, 0, P->st);
    if (s != BFCS_OK) return s;
  }
  const void* bs[1] = {b};
  const int8_t* ps[1] = {phase};
  void* es[1] = {eps_pred};
  const int prec = (P->fp64 || P->mixed) ? BFCS_FP64 : BFCS_FP32;
  return bfcs_net_predict(P->net, (const float*)weights, prec, 1, bs, ps, nph, phases, es);
}

}  // extern "C"

template <typename R>
static int fft3d_impl(bfcs_plan P, int dir, int ncomp, const void* in, void* out, void* specbuf,
                      void* const* twb) {
  const Geo g = P->g;
  const size_t csz = sizeof(C2<R>);
  C2<R>* spec = (C2<R>*)specbuf;
  CArgs<R> ca{};
  ca.data = spec;
  ca.g = g;
  ca.ncomp = ncomp;
  XArgs<R> xa{};
  xa.g = g;
  xa.ncomp = ncomp;
  xa.tw = (const C2<R>*)twb[0];
  const size_t rows = (size_t)ncomp * g.nz * g.ny;
  if (dir < 0) {
    xa.mode = XM_R2C;
    xa.real_in = (const R*)in;
    xa.spec_out = spec;
    CK(launch_xpass<R>(xa, P->st));
    ca.axis = 1; ca.tw = (const C2<R>*)twb[1];
    CK(launch_colpass<R>(ca, -1, P->st));
    ca.axis = 2; ca.tw = (const C2<R>*)twb[2];
    CK(launch_colpass<R>(ca, -1, P->st));
    CK(cudaMemcpy2DAsync(out, g.mx * csz, spec, g.p * csz, g.mx * csz, rows, cudaMemcpyDeviceToDevice,
                         P->st));
  } else {
    CK(cudaMemcpy2DAsync(spec, g.p * csz, in, g.mx * csz, g.mx * csz, rows, cudaMemcpyDeviceToDevice,
                         P->st));
    ca.axis = 2; ca.tw = (const C2<R>*)twb[2];
    CK(launch_colpass<R>(ca, +1, P->st));
    ca.axis = 1; ca.tw = (const C2<R>*)twb[1];
    CK(launch_colpass<R>(ca, +1, P->st));
    xa.mode = XM_C2R;
    xa.spec_in = spec;
    xa.real_out = (R*)out;
    CK(launch_xpass<R>(xa, P->st));
  }
  return sync_stream(P);
}

// FP64 forward transform of ncomp (<= 6) real fields into spec ([c][z][y][p]),
// or the inverse of spec into real fields (unnormalised), with the given twiddles
static int fp64_forward(bfcs_plan P, const double* in, int ncomp, C2<double>* spec, void* const* tw) {
  XArgs<double> xa{};
  xa.g = P->g;
  xa.ncomp = ncomp;
  xa.tw = (const C2<double>*)tw[0];
  xa.mode = XM_R2C;
  xa.real_in = in;
  xa.spec_out = spec;
  CK(launch_xpass<double>(xa, P->st));
  CArgs<double> ca{};
  ca.data = spec;
  ca.g = P->g;
  ca.ncomp = ncomp;
  ca.axis = 1; ca.tw = (const C2<double>*)tw[1];
  CK(launch_colpass<double>(ca, -1, P->st));
  ca.axis = 2; ca.tw = (const C2<double>*)tw[2];
  CK(launch_colpass<double>(ca, -1, P->st));
  return BFCS_OK;
}
static int fp64_inverse(bfcs_plan P, C2<double>* spec, int ncomp, double* out, void* const* tw) {
  CArgs<double> ca{};
  ca.data = spec;
  ca.g = P->g;
  ca.ncomp = ncomp;
  ca.axis = 2; ca.tw = (const C2<double>*)tw[2];
  CK(launch_colpass<double>(ca, +1, P->st));
  ca.axis = 1; ca.tw = (const C2<double>*)tw[1];
  CK(launch_colpass<double>(ca, +1, P->st));
  XArgs<double> xa{};
  xa.g = P->g;
  xa.ncomp = ncomp;
  xa.tw = (const C2<double>*)tw[0];
  xa.mode = XM_C2R;
  xa.spec_in = spec;
  xa.real_out = out;
  CK(launch_xpass<double>(xa, P->st));
  return BFCS_OK;
}

// device buffers of one nonlocal-kernel call, freed on exit
struct NlBufs {
  void* p[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  ~NlBufs() {
    for (void* q : p) cudaFree(q);
  }
  bool alloc(int i, size_t bytes) { return cudaMalloc(&p[i], bytes) == cudaSuccess; }
};

static int nl_check(bfcs_plan P, int degree, double delta) {
  if (P == nullptr || degree < 0 || degree >= kNlMaxBasis || !(delta > 0) || !std::isfinite(delta))
    return BFCS_ERR_INVALID_ARG;
  if (!P->fp64 && !P->mixed) return BFCS_ERR_UNSUPPORTED;
  if (2.0 * delta >= (double)std::min(P->g.nx, std::min(P->g.ny, P->g.nz))) return BFCS_ERR_INVALID_ARG;
  return BFCS_OK;
}

extern "C" {

int bfcs_kernel_fit(bfcs_plan P, int nload, const void* const* u, const void* const* gamma, double delta,
                    int degree, double lam, int iters, double lr, double* coef_out, double* exact_out,
                    double* loss_out, double* gram_out, double* rhs_out) {
  int e = nl_check(P, degree, delta);
  if (e != BFCS_OK) return e;
  if (nload < 1 || u == nullptr || gamma == nullptr || coef_out == nullptr || !(lam >= 0) || !std::isfinite(lam) ||
      iters < 0 || !(lr > 0) || !std::isfinite(lr))
    return BFCS_ERR_INVALID_ARG;
  for (int k = 0; k < nload; ++k)
    if (u[k] == nullptr || gamma[k] == nullptr) return BFCS_ERR_INVALID_ARG;
  const Geo g = P->g;
  const int nb = degree + 1;
  const int nacc = nb * (nb + 1) / 2 + nb + 1;
  const int nout = 2 * nb + 2 + nb * nb + nb;
  const size_t modes = (size_t)g.nz * g.ny * g.mx;
  C2<double>* spec = (C2<double>*)(P->mixed ? P->spec64 : P->spec);
  void* const* tw = P->mixed ? P->tw64 : P->tw;
  NlBufs B;
  if (!B.alloc(0, nb * modes * sizeof(double)) || !B.alloc(1, std::min(nb, 6) * (size_t)g.n * sizeof(double)) ||
      !B.alloc(2, (size_t)kNlParts * nacc * sizeof(double)) || !B.alloc(3, nacc * sizeof(double)) ||
      !B.alloc(4, nout * sizeof(double))) {
    cudaGetLastError();
    return BFCS_ERR_OOM;
  }
  double* W = (double*)B.p[0];
  double* wf = (double*)B.p[1];
  CK(cudaMemsetAsync(B.p[3], 0, nacc * sizeof(double), P->st));
  const NlCoef none{};
  for (int m0 = 0; m0 < nb; m0 += 6) {            // spectra of the basis kernels, six at a time
    const int k = std::min(6, nb - m0);
    CK(launch_basis_fields(wf, k, degree, m0, none, delta, g, P->st));
    e = fp64_forward(P, wf, k, spec, tw);
    if (e != BFCS_OK) return e;
    CK(launch_extract_real(spec, k, g, W, m0, P->st));
  }
  for (int k = 0; k < nload; ++k) {                // Gram matrix, right-hand side and |Gamma|^2 of every load
    e = fp64_forward(P, (const double*)u[k], 3, spec, tw);
    if (e == BFCS_OK) e = fp64_forward(P, (const double*)gamma[k], 3, spec + 3 * g.cs, tw);
    if (e != BFCS_OK) return e;
    CK(launch_kernel_gram(nb, W, spec, g, (double*)B.p[2], (double*)B.p[3], P->st));
  }
  CK(launch_kernel_adam((const double*)B.p[3], nb, lam, iters, lr, (double*)B.p[4], P->st));
  std::vector<double> h(nout);
  CK(cudaMemcpyAsync(h.data(), B.p[4], nout * sizeof(double), cudaMemcpyDeviceToHost, P->st));
  const int w = sync_stream(P);
  if (w != BFCS_OK) return w;
  for (int a = 0; a < nb; ++a) {
    coef_out[a] = h[a];
    if (exact_out != nullptr) exact_out[a] = h[nb + a];
    if (rhs_out != nullptr) rhs_out[a] = h[2 * nb + 2 + nb * nb + a];
  }
  if (loss_out != nullptr) { loss_out[0] = h[2 * nb]; loss_out[1] = h[2 * nb + 1]; }
  if (gram_out != nullptr)
    for (int a = 0; a < nb * nb; ++a) gram_out[a] = h[2 * nb + 2 + a];
  return BFCS_OK;
}

int bfcs_kernel_apply(bfcs_plan P, int degree, const double* coef, double delta, const void* u, void* out) {
  int e = nl_check(P, degree, delta);
  if (e != BFCS_OK) return e;
  if (coef == nullptr || u == nullptr || out == nullptr) return BFCS_ERR_INVALID_ARG;
  const Geo g = P->g;
  NlCoef kc{};
  kc.use = 1;
  for (int m = 0; m <= degree; ++m) {
    if (!std::isfinite(coef[m])) return BFCS_ERR_INVALID_ARG;
    kc.c[m] = coef[m];
  }
  C2<double>* spec = (C2<double>*)(P->mixed ? P->spec64 : P->spec);
  void* const* tw = P->mixed ? P->tw64 : P->tw;
  NlBufs B;
  if (!B.alloc(0, (size_t)g.n * sizeof(double)) ||
      !B.alloc(1, (size_t)g.nz * g.ny * g.mx * sizeof(double))) {
    cudaGetLastError();
    return BFCS_ERR_OOM;
  }
  CK(launch_basis_fields((double*)B.p[0], 1, degree, 0, kc, delta, g, P->st));    // K on the grid
  e = fp64_forward(P, (const double*)B.p[0], 1, spec, tw);
  if (e != BFCS_OK) return e;
  CK(launch_extract_real(spec, 1, g, (double*)B.p[1], 0, P->st));                 // K_hat (real)
  e = fp64_forward(P, (const double*)u, 3, spec, tw);
  if (e != BFCS_OK) return e;
  CK(launch_kernel_mult(spec, 3, g, (const double*)B.p[1], 1.0 / (double)g.n, P->st));
  e = fp64_inverse(P, spec, 3, (double*)out, tw);
  if (e != BFCS_OK) return e;
  return sync_stream(P);
}

int bfcs_polarize(bfcs_plan P, const int8_t* phase, int nph, const bfcs_lame* phases, bfcs_lame C0,
                  const void* eps, void* tau) {
  if (P == nullptr || phase == nullptr || eps == nullptr || tau == nullptr) return BFCS_ERR_INVALID_ARG;
  const int cm = check_material(nph, phases, C0);
  if (cm != BFCS_OK) return cm;
  if (P->fp64 || P->mixed)
    CK(launch_polarize<double>((double*)tau, (const double*)eps, phase, make_tab<double>(nph, phases, C0), P->g.n,
                               P->st));
  else
    CK(launch_polarize<float>((float*)tau, (const float*)eps, phase, make_tab<float>(nph, phases, C0), P->g.n,
                              P->st));
  return BFCS_OK;
}

int bfcs_green_apply(bfcs_plan P, bfcs_lame C0, const double E[6], const void* b_hat, void* spec, void* d_prev,
                     double* num_out) {
  if (P == nullptr || E == nullptr || b_hat == nullptr || spec == nullptr || (d_prev == nullptr) != (num_out == nullptr))
    return BFCS_ERR_INVALID_ARG;
  if (!(std::isfinite(C0.lambda) && std::isfinite(C0.mu) && C0.mu > 0 && C0.lambda + 2 * C0.mu > 0))
    return BFCS_ERR_INVALID_ARG;
  Geo g = P->g;                       // dense rows: nx/2 + 1 modes each
  g.p = g.mx;
  g.cs = (long long)g.nz * g.ny * g.mx;
  const int blocks = std::max(1, std::min(P->npart, 4 * 152));
  if (P->fp64 || P->mixed)
    CK(launch_green_dense<double>((C2<double>*)spec, (const C2<double>*)b_hat, (C2<double>*)d_prev, g, C0.lambda,
                                  C0.mu, E, P->part, blocks, num_out, P->st));
  else
    CK(launch_green_dense<float>((C2<float>*)spec, (const C2<float>*)b_hat, (C2<float>*)d_prev, g, C0.lambda,
                                 C0.mu, E, P->part, blocks, num_out, P->st));
  return BFCS_OK;
}

int bfcs_fft3d(bfcs_plan P, int direction, int ncomp, const void* in, void* out) {
  if (P == nullptr || in == nullptr || out == nullptr || ncomp < 1 || ncomp > 6 ||
      (direction != -1 && direction != 1))
    return BFCS_ERR_INVALID_ARG;
  if (P->mixed) return fft3d_impl<double>(P, direction, ncomp, in, out, P->spec64, P->tw64);
  return P->fp64 ? fft3d_impl<double>(P, direction, ncomp, in, out, P->spec, P->tw)
                 : fft3d_impl<float>(P, direction, ncomp, in, out, P->spec, P->tw);
}

long long bfcs_kernel_launches(void) { return launches_so_far(); }

int bfcs_profile_kernel(bfcs_plan P, int kind) {
  if (P == nullptr || kind < 0 || kind > 3) return BFCS_ERR_INVALID_ARG;
  if (kind != 0 && P->prof_ev.empty()) {
    const int pairs = 4096;
    P->prof_ev.resize(2 * pairs, nullptr);
    for (auto& e : P->prof_ev)
      if (cudaEventCreate(&e) != cudaSuccess) return BFCS_ERR_CUDA;
    P->prof_sweep.assign(pairs, 0);
  }
  P->prof_kind = kind;
  P->prof_launches = 0;
  P->prof_ms = 0.0;
  CK(cudaMemsetAsync(P->io_dev, 0, 2 * sizeof(unsigned long long), P->st));
  return BFCS_OK;
}

int bfcs_profile_green_io(bfcs_plan P, long long* d_reads, long long* d_writes) {
  if (P == nullptr || d_reads == nullptr || d_writes == nullptr) return BFCS_ERR_INVALID_ARG;
  unsigned long long h[2] = {0, 0};
  CK(cudaMemcpyAsync(h, P->io_dev, sizeof(h), cudaMemcpyDeviceToHost, P->st));
  const int w = sync_stream(P);
  if (w != BFCS_OK) return w;
  *d_reads = (long long)h[0];
  *d_writes = (long long)h[1];
  CK(cudaMemsetAsync(P->io_dev, 0, sizeof(h), P->st));
  return BFCS_OK;
}

int bfcs_profile_read(bfcs_plan P, long long* launches, double* total_ms) {
  if (P == nullptr || launches == nullptr || total_ms == nullptr) return BFCS_ERR_INVALID_ARG;
  *launches = P->prof_launches;
  *total_ms = P->prof_ms;
  P->prof_launches = 0;
  P->prof_ms = 0.0;
  return BFCS_OK;
}

int bfcs_twiddles(int n, int precision, void* out, int cap) {
  int r1 = 0, r2 = 0;
  line_radices(n, r1, r2);
  if (r1 == 0 || (precision != BFCS_FP32 && precision != BFCS_FP64 && precision != BFCS_MIXED) || cap < 0)
    return BFCS_ERR_INVALID_ARG;
  if (precision == BFCS_MIXED) {
    const std::vector<C2<ff>> h = twiddle_table<ff>(n);
    if (out != nullptr && (int)h.size() <= cap) std::memcpy(out, h.data(), h.size() * sizeof(C2<ff>));
    return (int)h.size();
  }
  if (precision == BFCS_FP32) {
    const std::vector<C2<float>> h = twiddle_table<float>(n);
    if (out != nullptr && (int)h.size() <= cap) std::memcpy(out, h.data(), h.size() * sizeof(C2<float>));
    return (int)h.size();
  }
  const std::vector<C2<double>> h = twiddle_table<double>(n);
  if (out != nullptr && (int)h.size() <= cap) std::memcpy(out, h.data(), h.size() * sizeof(C2<double>));
  return (int)h.size();
}

int bfcs_last_history(bfcs_plan P, double* hist, int cap) {
  if (P == nullptr || hist == nullptr || cap < 0) return BFCS_ERR_INVALID_ARG;
  const int n = std::min(cap, std::min(P->last_iters, P->hist_cap));
  if (n > 0) {
    if (cudaMemcpyAsync(hist, P->hist, n * sizeof(double), cudaMemcpyDeviceToHost, P->st) != cudaSuccess)
      return BFCS_ERR_CUDA;
    const int w = sync_stream(P);
    if (w != BFCS_OK) return w;
  }
  return n;
}

}  // extern "C"
