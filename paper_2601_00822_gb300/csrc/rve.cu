// RVE-size loop of Def. 2.2 and Sec. 5, written as a client of the library's
// public entry points: for each candidate body-force unit cell (a cubic grid of
// whole microstructure cells, the load centred at the cell corner nearest the
// grid centre) the BFCS problem is solved, the shell maxima of |eps| and
// |sigma| about the centre give the RVE radius (the fields stay below tol_f
// times their maximum beyond it), and the loop stops at the first grid that
// holds the RVE together with an annulus of half the support radius.
#include "bfcs.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace {

// smallest r with every shell r <= k < rmax of every profile at most tol_f
// times the profile's largest value; -1 when the outermost shell is above
int rve_radius(const std::vector<const double*>& profs, double tol_f, int rmax) {
  int r = 0;
  for (const double* p : profs) {
    double mx = 0.0;
    for (int k = 0; k < rmax; ++k) mx = std::max(mx, p[k]);
    const double lim = tol_f * mx;
    int rp = 0;
    for (int k = 0; k < rmax; ++k)
      if (p[k] > lim) rp = k + 1;
    if (rp >= rmax) return -1;
    r = std::max(r, rp);
  }
  return r;
}

int severity(int s) { return s < 0 ? 1000 - s : s; }

struct Buffers {
  void* p[4] = {nullptr, nullptr, nullptr, nullptr};
  ~Buffers() {
    for (void* q : p) cudaFree(q);
  }
};

}  // namespace

extern "C" int bfcs_rve_size(int cx, int cy, int cz, int nsph, const int32_t* spheres, int nph,
                             const bfcs_lame* phases, bfcs_lame C0, double a, int nsizes, const int* sizes, int flags,
                             double tol, int maxit, double tol_f, bfcs_rve_record* records, double* profiles,
                             int* accepted, void* stream) {
  if (cx < 1 || cy < 1 || cz < 1 || nsph < 0 || (nsph > 0 && spheres == nullptr) || nsizes < 1 ||
      sizes == nullptr || records == nullptr || !(a > 0) || !(tol_f > 0) || !(tol >= 0))
    return BFCS_ERR_INVALID_ARG;
  int maxbins = 0;
  for (int i = 0; i < nsizes; ++i) {
    const int n = sizes[i];
    if (n < 4 || n % cx || n % cy || n % cz) return BFCS_ERR_INVALID_ARG;
    maxbins = std::max(maxbins, n / 2);
  }
  if (accepted != nullptr) *accepted = -1;
  if (profiles != nullptr) std::memset(profiles, 0, sizeof(double) * (size_t)nsizes * 2 * maxbins);
  const int prec = flags & 3;
  const size_t rsz = prec == BFCS_FP32 ? sizeof(float) : sizeof(double);
  int worst = BFCS_OK;
  for (int i = 0; i < nsizes; ++i) {
    const int n = sizes[i];
    const size_t N = (size_t)n * n * n;
    bfcs_rve_record& rec = records[i];
    std::memset(&rec, 0, sizeof(rec));
    rec.n = n;
    rec.r_rve = -1;
    const int cell[3] = {cx, cy, cz};
    for (int d = 0; d < 3; ++d) rec.centre[d] = cell[d] * std::floor(n / (2.0 * cell[d]) + 0.5);
    bfcs_plan plan = nullptr;
    int e = bfcs_plan_create(&plan, n, n, n, 1, flags, stream);
    if (e != BFCS_OK) return e;
    Buffers buf;
    if (cudaMalloc(&buf.p[0], N) != cudaSuccess || cudaMalloc(&buf.p[1], 3 * N * rsz) != cudaSuccess ||
        cudaMalloc(&buf.p[2], 6 * N * rsz) != cudaSuccess || cudaMalloc(&buf.p[3], 6 * N * rsz) != cudaSuccess) {
      cudaGetLastError();
      bfcs_plan_destroy(plan);
      return BFCS_ERR_OOM;
    }
    const double E[6] = {0, 0, 0, 0, 0, 0};
    bfcs_info info{};
    std::vector<double> pe(n / 2), ps(n / 2);
    e = bfcs_voxelize(n, n, n, cx, cy, cz, nsph, spheres, (int8_t*)buf.p[0], stream);
    if (e == BFCS_OK)
      e = bfcs_body_force(n, n, n, rec.centre[0], rec.centre[1], rec.centre[2], a,
                          prec == BFCS_FP32 ? BFCS_FP32 : BFCS_FP64, buf.p[1], stream);
    if (e == BFCS_OK)
      e = bfcs_solve(plan, (const int8_t*)buf.p[0], nph, phases, C0, buf.p[1], E, tol, maxit, nullptr, buf.p[2],
                     buf.p[3], nullptr, &info);
    if (e >= 0) {
      rec.iters = info.iters;
      rec.status = e;
      rec.resid = info.resid;
      if (severity(e) > severity(worst)) worst = e;
      int e2 = bfcs_radial_profile(plan, buf.p[2], 6, rec.centre, n / 2, pe.data(), nullptr);
      if (e2 == BFCS_OK) e2 = bfcs_radial_profile(plan, buf.p[3], 6, rec.centre, n / 2, ps.data(), nullptr);
      e = e2 == BFCS_OK ? e : e2;
    }
    bfcs_plan_destroy(plan);
    if (e < 0) return e;
    for (int k = 0; k < n / 2; ++k) {
      rec.eps_max = std::max(rec.eps_max, pe[k]);
      rec.sig_max = std::max(rec.sig_max, ps[k]);
    }
    if (profiles != nullptr) {
      std::memcpy(profiles + (size_t)(2 * i) * maxbins, pe.data(), sizeof(double) * (n / 2));
      std::memcpy(profiles + (size_t)(2 * i + 1) * maxbins, ps.data(), sizeof(double) * (n / 2));
    }
    rec.r_rve = rve_radius({pe.data(), ps.data()}, tol_f, n / 2);
    rec.contained = rec.r_rve >= 0 && rec.r_rve + 0.5 * a <= 0.5 * n;
    if (rec.contained) {
      if (accepted != nullptr) *accepted = i;
      break;
    }
  }
  return worst;
}
