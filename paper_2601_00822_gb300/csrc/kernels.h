// Host-side launch interfaces of the BFCS kernels (internal; the public C-ABI
// is include/bfcs.h).  Every launcher returns a cudaError_t and enqueues on
// the given stream.
#pragma once
#include "common.cuh"

namespace bfcs {

// ---- x pass: along x (contiguous) with the real<->half-spectrum transform.
enum XMode : int {
  XM_SWEEP = 0,    // spectrum -> C2R -> eps -> tau = L1 eps -> R2C -> spectrum (Eqs. 5.7, 5.8, 5.10)
  XM_REALTAU = 1,  // real eps (warm start) -> tau -> R2C -> spectrum
  XM_R2C = 2,      // plain forward real -> half spectrum along x
  XM_C2R = 3,      // plain inverse half spectrum -> real along x
  XM_REALSIG = 4,  // real eps -> sigma = L eps -> R2C -> spectrum (defect evaluation)
  XM_SWEEPSIG = 5, // spectrum -> C2R -> eps (written) -> sigma = L eps -> R2C -> spectrum
};

// Which member fields a batched x pass reads and writes (host-side selection).
enum XMemIO : int {
  XIN_NONE = 0, XIN_EPS_INIT = 1, XIN_B = 2,
  XOUT_EPS = 1, XOUT_SIG = 2, XOUT_U = 4,
};

// Members per batched launch (their x-pass fields travel in the launch arguments).
constexpr int kMaxBatch = 64;

// Per-member fields of the x pass, passed by value in the launch arguments so
// that every block reads them from the constant bank.
struct XMember {
  const int8_t* phase;
  const void* real_in;    // selected input (b or eps_init) or null
  void* eps_out;
  void* sig_out;
  void* real_out;         // u output or null
  int sx, sy, sz, warm;
};

template <typename R> struct XArgs {
  Geo g;
  const C2<R>* spec_in;   // [ncomp][nz][ny][p]
  C2<R>* spec_out;        // may alias spec_in (each block owns its lines)
  const R* real_in;       // [ncomp][nz][ny][nx]
  R* real_out;            // [ncomp][nz][ny][nx]
  R* eps_out;             // optional, sweep modes: 6 x N
  R* sig_out;             // optional, sweep modes: 6 x N
  const int8_t* phase;    // [nz][ny][nx] phase ids of the untranslated microstructure
  int sx, sy, sz;         // translation chi: phase(x) = phase0(x - chi) (Eq. 3.3)
  PhaseTab<R> tab;
  const C2<R>* tw;        // exp(-2 pi i j / nx), j < nx
  const IterState* st;    // nullable: per-member state; a member with st[m].done skips
  long long spec_ms;      // spectrum stride between members (complex elements)
  int use_xm;             // 1: member m = blockIdx.z takes phase, shift, I/O from xm[m]
  R out_scale;            // XM_R2C: factor applied to the stored half spectrum (0 means 1)
  int ncomp;
  int mode;
  XMember xm[kMaxBatch];
};

// ---- column passes along y (axis 1) or z (axis 2) on the half spectrum, in place.
template <typename R> struct CArgs {
  C2<R>* data;
  Geo g;
  int axis;
  int ncomp;
  const C2<R>* tw;        // exp(-2 pi i j / n_axis)
  const IterState* st;    // nullable: member m = blockIdx.z skips once st[m].done
  long long ms;           // data stride between members (complex elements)
  int variant;            // FP32 only: column tile and factor order (kColVariants; 0 = default)
  const void* tmap;       // host array of the two tensor maps (8, 16 columns) of a y pass over 6-component spectra, or null
  const void* tmap_data;  // the buffer the maps address: the tensor-copy tiles run only when data is this buffer
};

// Column-pass variants an autotuner can pick from (FP32): tile width in kx
// columns, the order of the two radices of the line length, and (6, 7) tiles
// loaded by one tensor-memory-access copy per block (y passes of the sweep).
constexpr int kColVariants = 8;
constexpr int col_variant_tile(int v) {
  return v == 6 ? 8 : v == 7 ? 16 : v % 3 == 0 ? 16 : v % 3 == 1 ? 8 : 32;
}
constexpr bool col_variant_swap(int v) { return v >= 3 && v < 6; }
constexpr bool col_variant_tma(int v) { return v >= 6; }
// whether variant v exists for line length n (only lengths with two different
// radices have a swapped order; the tunable lengths are 32..256)
bool col_variant_valid(int v, int n);

// ---- conjugate gradients on the operator of Eq. 5.13 (k_cg.cu)
struct CgState {
  double rr, rr0;        // <r, r>_C0 now and at the start
  double alpha, beta;
  double tol2;           // stop once <r, r> <= tol2 * rr0
  double best;           // smallest <r, r> so far
  int done, iters, maxit;
  int best_it;           // iteration of `best`; no new best for kCgStagnation iterations ends the member
};
constexpr int kCgStagnation = 50;
constexpr int kCgParts = 512;       // partial sums per member
template <typename R> struct CgArgs {
  C2<R>* c;              // iterate (state layout, members at ms)
  C2<R>* r;              // residual
  C2<R>* p;              // search direction
  C2<R>* q;              // A p (holds U0 * L1 p on entry of the PQ step)
  const C2<R>* s;        // INIT: one sweep applied to c
  long long ms;
  Geo g;
  double lam0, mu0;
  double* part;          // kCgParts doubles per member
  CgState* cg;
  IterState* skip;       // done flags read by the FFT passes of A p
};
// mode 0 INIT (r = s - c, p = r), 1 PQ (q = p - q, alpha), 2 UPDATE (c, r, beta,
// convergence), 3 DIR (p = r + beta p); the scalar step follows modes 0-2.
template <typename R> cudaError_t launch_cg_vec(const CgArgs<R>& a, int mode, int batch, cudaStream_t st);

// ---- displacement-based conjugate gradients, Algorithm 3 (k_cd.cu)
struct CdMode { enum : int { INIT = 0, PQ = 1, UPDATE = 2, FINAL = 4, FINAL_U = 5, RESID = 6 }; };
struct CdState {
  double rz;             // <r, z> (<r, r> without preconditioner)
  double alpha, beta;
  double s0b[6];         // sigma_hat(0) of L eps^{b(0)} (DFT scale)
  double s0u[6];         // sigma_hat(0) of L grad^s u1 (after RESID: of the returned strain)
  double s0p[6];         // sigma_hat(0) of L grad^s p (this iteration)
  double tol;            // stop at residual <= tol (Eq. 5.11)
  double resid;          // residual of the current iterate
  int done, iters, maxit;
  int status;            // 0 running, 1 converged, 2 iteration limit, 3 breakdown or NaN
  int pend;              // 1: an update step ended the member before its direction step
                         // added alpha p to u1 (the final steps add it)
};
constexpr int kCdParts = 512;       // partial sums (pairs) per member
template <typename R> struct CdArgs {
  C2<R>* u;              // u1_hat (3 components, fully transformed half spectrum)
  C2<R>* r;              // residual b^A - A(u1) (z = M r is formed where used)
  C2<R>* p;              // search direction
  C2<R>* q;              // A p
  C2<R>* s;              // 6-component work spectrum (operator input and output)
  const C2<R>* bhat;     // body force spectrum (3 components)
  long long ms, sms, b_ms;   // member strides of the vectors, of s and of bhat
  Geo g;
  double lam0, mu0;
  double* part;          // 2 x kCdParts doubles per member
  CdState* cd;
  IterState* skip;       // done flags read by the FFT passes of A p
  const Member* mem;     // per-member mean strain (FINAL)
  int precond;           // 1: z = G0 r
  const C2<R>* tw;       // z twiddles exp(-2 pi i j / nz) (fused z passes)
};
// the vector step `mode` for members 0..batch-1, then (INIT, PQ, UPDATE, RESID)
// the scalar step; ist: the members' IterState (bden read; iterations, residuals,
// status written)
template <typename R>
cudaError_t launch_cd_vec(const CdArgs<R>& a, int mode, int batch, IterState* ist, const Member* mem, int maxdim,
                          cudaStream_t st);
// the operator's z transforms fused with the CG steps beside them: fwd = the forward z
// transform of the stress spectrum in a.s, then q = -i xi . sigma_hat, <p, q> and
// alpha (replaces the forward z column pass and PQ); !fwd = p = M r + beta p, the
// strain spectrum sym(i xi (x) p) / N and its inverse z transform into a.s
// (replaces DIR and the inverse z column pass).  a.tw: the z twiddles.  The <p, q>
// partials take one pair per tile: a.part holds at least tiles x batch pairs.
template <typename R>
cudaError_t launch_zcd(const CdArgs<R>& a, bool fwd, int batch, IterState* ist, const Member* mem, int maxdim,
                       cudaStream_t st);
// partial pairs per member the Algorithm 3 kernels need (vector steps: kCdParts; fused
// forward z pass: one per tile)
inline int cd_parts(const Geo& g) {
  const int tiles = (g.mx + 3) / 4 * g.ny;
  return tiles > kCdParts ? tiles : kCdParts;
}

// ---- fused z pass: forward z FFT -> Green operators -> residual -> inverse z FFT.
enum GMode : int {
  GM_SWEEP = 0,   // eps_hat^{s+1} = -Gamma0 tau_hat^s + eps_hat^{b(0)}, k=0 <- E; residual of eps^s
  GM_INIT = 1,    // tau_hat = 0: eps_hat^0 = eps_hat^{b(0)} (+E); d_prev <- 0
  GM_FINAL = 2,   // residual of eps^S; u_hat^S = i G0 (d_prev - i b_hat) into components 0..2
  GM_APPLY = 3,   // the operator alone (Eq. 5.13): eps_hat = U0 tau_hat, no load, k=0 <- 0, no d, no residual
};

template <typename R> struct GArgs {
  C2<R>* spec;            // 6 components, x- and y-transformed
  const C2<R>* bhat;      // 3 components, fully transformed body force
  C2<R>* dprev;           // 3 components: d = tau_hat . xi of the previous sweep
  Geo g;
  R lam0, mu0;
  R E[6];
  R inv_n;                // 1 / |N| of Eq. 4.4
  const C2<R>* tw;        // exp(-2 pi i j / nz)
  ResidSlot* part;        // one slot per block (per member: part_ms slots)
  IterState* st;          // per member
  long long spec_ms, b_ms, d_ms;   // member strides (complex elements)
  int part_ms;
  int skip_done;          // 1: members with st[m].done skip the launch
  int use_me;             // 1: member m takes its mean strain from mE[m]
  int mode;
  // GM_SWEEP with sparse residual evaluation: sweep s = st[m].iters reads d_prev
  // and forms the residual only when s == st[m].next_check, and writes d only on
  // that sweep, the one before it and the last sweep (s + 1 == maxit)
  int sparse;
  int maxit;
  R mE[kMaxBatch][6];
};

// ---- defect of an approximate strain on the fully transformed stress spectrum:
// R_hat = i xi . sigma_hat + b_hat on modes with xi != 0 (0 elsewhere), written
// as complex64 to out32; per-block partial sums of w |R_hat|^2; sigma_hat(0)
// (6 values) into st->tau0.
// Batched over slots (blockIdx.y): slot j works on member idx[j]; spec and part
// are slot-major, bhat, out32 and st member-major.
template <typename R> struct DArgs {
  const C2<R>* spec;      // 6 components: sigma_hat
  const C2<R>* bhat;      // 3 components
  C2<float>* out32;       // 3 components: R_hat rounded to complex64 (the FP32 correction load)
  Geo g;
  ResidSlot* part;
  IterState* st;
  long long spec_ms, b_ms, o_ms;   // member strides (elements)
  int idx[kMaxBatch];
};

// eps_hat = sym(i xi (x) u_hat) / N on modes with xi != 0, E at k = 0, 0 on the
// other xi = 0 modes: components 0..2 of `spec` (u_hat, fully transformed) in,
// components 0..5 out, in place.
template <typename R> cudaError_t launch_symgrad(C2<R>* spec, long long ms, const Geo& g, const Member* mem, int batch,
                                                 cudaStream_t s);

// Green step on a dense half spectrum (row pitch g.p = g.mx, component stride
// g.cs): spec holds tau_hat on entry and eps_hat^{s+1} (unnormalised) on exit;
// with dprev and num_out, the residual numerator of Eq. 5.11 from |d - d_prev|
// goes to *num_out (block partials in part, nblocks slots) and d to dprev.
template <typename R>
cudaError_t launch_green_dense(C2<R>* spec, const C2<R>* bhat, C2<R>* dprev, const Geo& g, double lam0,
                               double mu0, const double* E, ResidSlot* part, int nblocks, double* num_out,
                               cudaStream_t st);
// tau = (L(x) - L0) : eps pointwise (table lam1 / mu1; phase ids outside the
// table read entry 0)
template <typename R>
cudaError_t launch_polarize(R* tau, const R* eps, const int8_t* phase, const PhaseTab<R>& tab, long long n,
                            cudaStream_t s);

template <typename R> cudaError_t launch_xpass(const XArgs<R>& a, cudaStream_t s);
template <typename R> cudaError_t launch_defect(const DArgs<R>& a, int blocks, int batch, cudaStream_t s);
// r(eps64) of slot j's member idx[j] from its defect partials (Eq. 5.11 reading):
// st[idx[j]].resid_final = sqrt(sum part) / (bden + 2 pi / maxdim |sigma_hat(0)|_F).
cudaError_t launch_defect_final(const ResidSlot* part, int nparts, IterState* st, const int* idx_host, int batch,
                                int maxdim, cudaStream_t s);
template <typename R> cudaError_t launch_colpass(const CArgs<R>& a, int dir, cudaStream_t s);
template <typename R> cudaError_t launch_zgreen(const GArgs<R>& a, cudaStream_t s);
template <typename R> int green_nparts(const Geo& g);
// residual partial slots per member written by a GM_SWEEP launch of the z pass
// (fewer than green_nparts when the persistent form runs)
template <typename R> int green_sweep_parts(const Geo& g);
template <typename R> cudaError_t launch_xpass_b(const XArgs<R>& a, int batch, cudaStream_t s);
template <typename R> cudaError_t launch_colpass_b(const CArgs<R>& a, int dir, int batch, cudaStream_t s);
template <typename R> cudaError_t launch_zgreen_b(const GArgs<R>& a, int batch, cudaStream_t s);
// u_hat^S = i G0(xi) (d_prev - i b_hat) / N into components 0..2 of a.spec for members
// 0..batch-1 (the displacement of the last iterate from the d_prev its sweep stored)
template <typename R> cudaError_t launch_uhat(const GArgs<R>& a, int batch, cudaStream_t s);

// ---- nonlocal kernel regression (k_nonlocal.cu, FP64)
constexpr int kNlMaxBasis = 8;      // Bernstein degree <= 7
constexpr int kNlParts = 2 * 152;   // partial sums of the Gram reduction
struct NlCoef { int use; double c[kNlMaxBasis]; };
// nb basis fields B_{m0..m0+nb-1}(|xi| / delta) (or, coef.use, one field sum_m c_m B_m) at minimum-image offsets
cudaError_t launch_basis_fields(double* w, int nb, int M, int m0, const NlCoef& coef, double delta, const Geo& g,
                                cudaStream_t s);
// W[(m0 + c) * modes + i] = Re of spectral component c at compact mode i
cudaError_t launch_extract_real(const C2<double>* spec, int ncomp, const Geo& g, double* W, int m0, cudaStream_t s);
// acc += (packed upper G, g, s) / N of one load: spec components 0..2 u_hat, 3..5 Gamma_hat
cudaError_t launch_kernel_gram(int nb, const double* W, const C2<double>* spec, const Geo& g, double* part,
                               double* acc, cudaStream_t s);
// Adam (iters steps from 0) and the exact minimiser; out: coef, exact, J(coef), J(exact), G, g
cudaError_t launch_kernel_adam(const double* acc, int nb, double lam, int iters, double lr, double* out,
                               cudaStream_t s);
// spec_c *= (K_hat - K_hat(0)) * scale, c < ncomp
cudaError_t launch_kernel_mult(C2<double>* spec, int ncomp, const Geo& g, const double* Kr, double scale,
                               cudaStream_t s);

// copy `bytes` (a multiple of 4) from device memory into pinned host memory with a kernel
cudaError_t launch_copy_words(void* dst, const void* src, size_t bytes, cudaStream_t s);

bool supported_len(int n);

// process-wide count of kernel launches made by this library
void count_launches(long long n);
long long launches_so_far();

// ---- misc kernels (k_misc.cu)
cudaError_t launch_voxelize(int8_t* out, int nx, int ny, int nz, int cx, int cy, int cz,
                            const int* sph_dev, int nsph, cudaStream_t s);
template <typename R>
cudaError_t launch_body_force(R* b, int nx, int ny, int nz, double cx, double cy, double cz,
                              double a, double* scratch /* >= body_force_scratch() doubles */,
                              cudaStream_t s);
int body_force_scratch(long long n);
template <typename R>
cudaError_t launch_body_force_blocks(R* b, int nx, int ny, int nz, double cx, double cy, double cz,
                                     double a, int blocks, double* scratch /* >= blocks + 1 doubles */,
                                     cudaStream_t s);

// validation: phase id range and body-force sums; out[0..1] = min/max phase,
// dout[0..2] = sum b_c, dout[3..5] = sum |b_c|
template <typename R>
cudaError_t launch_validate(const int8_t* phase, const R* b, long long n, int* iout, double* dout,
                            double* scratch, cudaStream_t s);
int validate_scratch(long long n);

// sum over modes with xi != 0 of w |b_hat|^2 -> st->bden = sqrt(sum); batched:
// member m uses bhat + m * b_ms, part + m * 512 and st + m
template <typename R>
cudaError_t launch_bden(const C2<R>* bhat, const Geo& g, ResidSlot* part, IterState* st, cudaStream_t s,
                        int batch = 1, long long b_ms = 0);

// residual reduction of the Green-pass partials; mode = GM_SWEEP, GM_FINAL or
// kReduceDefect.  One block per member: member m reduces part[m * nparts ...],
// updates st[m] and writes hist[m * hist_cap + sweep]; its E and warm flag
// come from mem[m] when mem is given, else from E / warm_all.  In GM_SWEEP the
// sweep index is the device counter st[m].iters.  check_max > 1: sparse
// evaluation, only sweeps s == st[m].next_check carry a residual (others
// record NaN in hist); after each evaluation the next one is placed at the
// sweep where the observed contraction rate predicts r <= tol, at most
// check_max sweeps ahead (every check_max sweeps when tol = 0).  io (nullable):
// two counters that GM_SWEEP adds to, per member, whether the sweep's Green
// pass read d_prev and whether it wrote d (maxit: the call's sweep limit).
cudaError_t launch_resid_reduce(const ResidSlot* part, int nparts, IterState* st, const Member* mem,
                                double* hist, int hist_cap, double tol, double c0_lam, double c0_mu,
                                const double* E, long long n, int maxdim, int mode, int warm_all,
                                int stall_window, int check_max, int maxit, unsigned long long* io, int batch,
                                cudaStream_t s);
// mode for launch_resid_reduce: tau0 already holds sigma_hat(0) (defect evaluation)
constexpr int kReduceDefect = 7;

// elementwise helpers (k_misc.cu)
cudaError_t launch_cast_d2f(float* dst, const double* src, long long count, cudaStream_t s);
cudaError_t launch_cast_f2d(double* dst, const float* src, long long count, cudaStream_t s);
cudaError_t launch_add_f2d(double* dst, const float* src, long long count, cudaStream_t s);
// complex128 -> complex64 copy of ncomp spectral components (same geometry)
cudaError_t launch_cast_spec(C2<float>* dst, const C2<double>* src, const Geo& g, int ncomp, cudaStream_t s);
cudaError_t launch_cast_spec_ff(C2<float>* dst, const C2<ff>* src, const Geo& g, int ncomp, cudaStream_t s);
// sigma = L(x) eps pointwise (FP64), phase translated by (sx, sy, sz)
cudaError_t launch_stress(double* sig, const double* eps, const int8_t* phase, const PhaseTab<double>& tab,
                          int sx, int sy, int sz, int nx, int ny, int nz, cudaStream_t s);

template <typename R>
cudaError_t launch_accumulate(double* acc, int* hits, const R* eps, const R* sig, const R* u,
                              const int8_t* phase, int sx, int sy, int sz, int nx, int ny, int nz,
                              cudaStream_t s);
cudaError_t launch_scale(double* acc, long long count, double f, cudaStream_t s);

// Effective moduli (Eqs. 6.1-6.3, 3.2): for each of up to kModMembers members the
// FP64 sums of sigma over the cell, of eps over the inclusion voxels and their
// count (kModSums values per member, written to out[m * kModSums + j]).
constexpr int kModMembers = 6;
constexpr int kModSums = 13;
constexpr int kModParts = 2 * 152;
template <typename R>
struct ModArgs {
  const R* eps[kModMembers];
  const R* sig[kModMembers];
  const int8_t* phase;
  long long n;
};
template <typename R>
cudaError_t launch_moduli(const ModArgs<R>& a, int batch, double* part, double* out, cudaStream_t s);

// RVE diagnostic (Def. 2.2): per shell k of the doubled-coordinate distance
// about c2 (2 x centre), the largest pointwise norm (merged into bits[k] as the
// bit pattern of a non-negative double) and the voxel count; ncomp 3 (vector)
// or 6 (symmetric tensor, shears counted twice); nbins <= kMaxShells.
constexpr int kMaxShells = 2048;
template <typename R>
cudaError_t launch_radial_max(const R* f, int ncomp, int nx, int ny, int nz, const int c2[3], int nbins,
                              unsigned long long* bits, unsigned long long* counts, cudaStream_t s);

}  // namespace bfcs
