/*
 * bfcs.h - C ABI of the GB300 (sm_103a) FFT solver for periodic linear-elastic
 * composites loaded by a body force with compact support (BFCS).
 *
 * Method: V. A. Buryachenko, "New RVE concept and FFT methods in micromechanics
 * of composites subjected to body force with compact support".  The solver runs
 * the modified basic scheme (Algorithm 1, Eqs. 5.7-5.10) for the modified
 * Lippmann-Schwinger equation (Eq. 2.14, Fourier form Eqs. 5.3-5.4) and the
 * translated averaging of Eqs. 3.3-3.7.
 *
 * Conventions shared by every call
 *  - Grid: nx, ny, nz even (Eq. 4.1); each in {4,6,8,12,16,24,32,48,64,96,128,
 *    192,256}.  Voxel (x, y, z) has linear index x + nx*(y + ny*z); h = 1.
 *  - Symmetric tensors: 6 components in the order xx, yy, zz, yz, xz, xy, with
 *    tensorial (not engineering) shears, stored component-major (SoA): component
 *    c of voxel v at [c*N + v], N = nx*ny*nz.  Vectors: 3 components, same way.
 *  - Phase maps: int8 per voxel, phase id 0 = matrix, ids >= 1 = inclusions
 *    (the indicator V of Eqs. 3.5-3.6 is phase != 0).
 *  - Memory: "dev" arguments are device pointers (for example torch tensor
 *    data_ptr()), "host" arguments host pointers.  The caller owns every buffer
 *    it passes; a plan owns its workspace.  Element types of real fields follow
 *    the plan precision: float for BFCS_FP32, double for BFCS_FP64.
 *  - Streams: all device work of a plan is ordered on the plan's stream.  The
 *    solve calls return when their results are written (they wait on the stream
 *    with a bounded host-side wait; an expired wait returns BFCS_ERR_TIMEOUT.
 *    The bound is 900 s, or the number of seconds in the environment variable
 *    BFCS_WAIT_TIMEOUT_S).
 *  - Status: 0 = OK, > 0 = completed with a warning, < 0 = error (see below).
 *    On error the output buffers are unspecified.
 *  - Wavevector (where the paper writes F(grad f) = i k f_hat, Eq. 4.8):
 *    xi_a = 2 pi k_a / N_a with signed k_a, and xi_a = 0 on the Nyquist index
 *    k_a = N_a/2 (spectral differentiation for even N).  Modes with xi = 0 other
 *    than k = 0 carry neither strain fluctuation nor load.
 */
#ifndef BFCS_H
#define BFCS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes */
#define BFCS_OK 0
#define BFCS_NOT_CONVERGED 1          /* maxit reached; result of the last sweep written */
#define BFCS_ERR_INVALID_ARG (-1)     /* bad size, pointer, phase id, tolerance, C0 ... */
#define BFCS_ERR_NONZERO_MEAN (-2)    /* body force not self-equilibrated (Eq. 2.5) */
#define BFCS_ERR_OOM (-3)             /* workspace allocation failed */
#define BFCS_ERR_CUDA (-4)            /* a CUDA runtime call failed */
#define BFCS_ERR_TIMEOUT (-5)         /* bounded wait on the stream expired */
#define BFCS_ERR_DIVERGED (-6)        /* NaN/Inf residual */
#define BFCS_ERR_UNSUPPORTED (-7)     /* feature not available in this build */

/* ---- plan flags */
#define BFCS_FP32 0                   /* FP32 fields and FFTs, FP64 residual sums */
#define BFCS_FP64 1                   /* FP64 throughout */
#define BFCS_MIXED 2                  /* FP32 sweeps with float-float defect correction; FP64 fields */
#define BFCS_AUTOTUNE 4               /* OR-ed with FP32 or MIXED: time the y-pass variants at plan creation */
#define BFCS_CG 8                     /* OR-ed with any precision: conjugate gradients (Algorithm 2) */
#define BFCS_SPARSE_RESID 16          /* OR-ed with any precision: residual (Eq. 5.11) on predicted sweeps only */
#define BFCS_CD 32                    /* OR-ed with any precision: displacement-based CG (Algorithm 3), as printed */
#define BFCS_CD_PRECOND 64            /* as BFCS_CD, with the reference medium's G0 as preconditioner */

#define BFCS_MAX_PHASES 16

typedef struct bfcs_plan_s* bfcs_plan;

/* Isotropic phase, L = 3k N1 + 2 mu N2 written with Lame constants (Sec. 2). */
typedef struct { double lambda, mu; } bfcs_lame;

typedef struct {
  int iters;            /* sweeps run (each sweep = Eqs. 5.7-5.10 once) */
  int status;           /* same value the call returned for this solve */
  double resid;         /* residual (Eq. 5.11 reading below) of the returned strain, FP64 */
  double resid_prev;    /* residual of the iterate that triggered the stop */
  int precision_path;   /* 0 = FP32 sweeps, 1 = FP64 sweeps, 2 = BFCS_MIXED ladder (resid: float-float defect of the FP64 strain) */
  int stalled;          /* 1 if the residual did not drop by 10% over 100 sweeps (stops the solve) */
  double ms;            /* host wall time of the call, milliseconds */
} bfcs_info;

/* One member of a batched solve (see bfcs_solve for field meanings). */
typedef struct {
  const int8_t* phase;          /* dev, N */
  const void* b;                /* dev, 3 x N */
  double E[6];                  /* prescribed mean strain */
  int shift[3];                 /* microstructure translation chi (Eq. 3.3) */
  const void* eps_init;         /* dev 6 x N or NULL */
  void* eps_out;                /* dev 6 x N */
  void* sig_out;                /* dev 6 x N or NULL */
  void* u_out;                  /* dev 3 x N or NULL */
} bfcs_problem;

/*
 * bfcs_plan_create - workspace and precision for solves on an nx*ny*nz grid.
 *  out:       receives the plan handle (host).
 *  nx,ny,nz:  grid (BFUC of Eq. 2.7 / Sec. 4 unit cell), even, supported sizes.
 *  max_batch: >= 1; members of bfcs_solve_batched are run in groups of at most
 *             this many.
 *  flags:     BFCS_FP32, BFCS_FP64 or BFCS_MIXED, optionally OR BFCS_AUTOTUNE
 *             (FP32 / MIXED: pick the y-pass variant by timing, see
 *             bfcs_plan_tuning) and BFCS_CG (the sweeps are driven by
 *             conjugate gradients on the operator of Eq. 5.13, Algorithm 2:
 *             rounds of CG to 0.1 tol, 0.01 tol, ... relative to their start
 *             in the C0-weighted norm, each verified by two sweeps of the
 *             residual of Eq. 5.11; info.iters counts operator applications;
 *             allocates four more strain spectra per member) and
 *             BFCS_CD or BFCS_CD_PRECOND (the displacement-based conjugate
 *             gradients of Algorithm 3, Eqs. 5.14-5.22, replace the sweeps:
 *             the unknown is the displacement fluctuation u1 of Eq. 2.10 in
 *             Fourier space, A(u1) = -div L grad^s u1 = div L1 eps^{b(0)}
 *             (Eq. 5.14 read with L1 = L - L0 on the right), u1 starts at 0,
 *             the CG residual is the equilibrium residual of Eq. 5.11, and
 *             BFCS_CD_PRECOND applies the reference medium's G0 to it; info.iters
 *             counts operator applications, info.resid is the residual of the
 *             returned strain; an eps_init is rejected with INVALID_ARG; not
 *             with BFCS_CG) and
 *             BFCS_SPARSE_RESID (the residual of Eq. 5.11 is evaluated on
 *             the first two sweeps and then on the sweep where the observed
 *             contraction rate predicts r <= tol, at most 8 sweeps apart;
 *             with tol = 0 on every 8th sweep from the first; the other sweeps neither read nor
 *             write the previous polarization's divergence, which saves 48 of
 *             the fused z pass's 168 bytes per mode; the fields of every
 *             sweep are the same as without the flag, the stopping sweep can
 *             only come later, and the history holds NaN on sweeps without a
 *             residual).  BFCS_MIXED runs the sweeps in FP32 and
 *             corrects them with defects evaluated in float-float
 *             arithmetic (below); its fields at the API (b, eps,
 *             sigma, u, eps_init, fft3d data) are double.
 *  stream:    cudaStream_t to order work on (NULL = legacy default stream).
 * Allocates about (6 + 3 + 3) * nz*ny*(nx/2+4) complex values of workspace.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
int bfcs_plan_create(bfcs_plan* out, int nx, int ny, int nz, int max_batch, int flags, void* stream);
int bfcs_plan_destroy(bfcs_plan plan);

/*
 * bfcs_voxelize - phase map of spheres in a periodic unit cell (Eqs. 2.21, 3.3).
 *  spheres: host, nsph rows of 5 int32 (X, Y, Z, T, phase): doubled centre in
 *           cell coordinates and T = floor((2R)^2).  A voxel with doubled centre
 *           (2i+1, 2j+1, 2k+1) (cell coordinates) is inside when its squared
 *           periodic minimum-image distance on the doubled grid is <= T; the
 *           last containing sphere wins; otherwise phase 0.
 *  cell:    cx, cy, cz dividing nx, ny, nz; the cell is tiled over the grid.
 *  phase_out: dev, N int8.  Integer arithmetic only (bit-exact).
 */
int bfcs_voxelize(int nx, int ny, int nz, int cx, int cy, int cz, int nsph, const int32_t* spheres,
                  int8_t* phase_out, void* stream);

/*
 * bfcs_body_force - BFCS field of Eq. 2.5 in the form b = (d phi/d x1, 0, 0),
 * phi = (1 - r^2/a^2)^3 for r < a, at voxel centres i + 0.5 with the periodic
 * minimum image about (cx, cy, cz), made mean-free in FP64.
 *  b_out: dev, 3 x N, float (precision = BFCS_FP32) or double (BFCS_FP64).
 */
int bfcs_body_force(int nx, int ny, int nz, double cx, double cy, double cz, double a, int precision,
                    void* b_out, void* stream);

/*
 * bfcs_body_force_noalloc - the same field as bfcs_body_force, for callers that
 * must not allocate device memory during the call (their device memory is
 * owned by their own pool or caching allocator, or an allocation could stall
 * a time-critical loop).  It makes no cudaMalloc/cudaMallocAsync/cudaFree call
 * and uses no allocating library routine.  The paper has no counterpart: this
 * is an allocation-free way to produce the load of Eq. 2.5.
 *  Scratch: a fixed 16 KiB FP64 array inside the library (up to 2048 partial
 *           sums + the mean), held on every GPU that loads the library until exit.
 *  Limit:   nx*ny*nz <= 134217728 voxels (a 512^3 grid), the stated maximum of
 *           this entry point; larger grids return BFCS_ERR_INVALID_ARG before
 *           any device work.
 *  Set-up:  the first call on each device (and the first in each new context
 *           of it, e.g. after cudaDeviceReset) looks up the array's device
 *           address (cudaGetSymbolAddress) with that device current; make that
 *           first call before any stream capture on the device.
 *  Sharing: every call uses the same array, which keeps the last call's
 *           contents; each call writes every slot it reads before reading it,
 *           so nothing needs clearing.  Calls whose work overlaps on the GPU
 *           (different streams, no ordering) race on the array: order them on
 *           one stream.  The mean is summed over a different number of blocks
 *           than bfcs_body_force uses, so results may differ in the last bits.
 * Arguments and layout as bfcs_body_force.
 */
int bfcs_body_force_noalloc(int nx, int ny, int nz, double cx, double cy, double cz, double a,
                            int precision, void* b_out, void* stream);

/*
 * bfcs_solve - modified basic scheme, Algorithm 1 (Eqs. 5.7-5.10).
 *  phase:   dev, N int8 phase ids in [0, nphases).
 *  phases:  host, nphases (1..16) isotropic phases, phase id = index.
 *  C0:      isotropic reference medium L0 (Eqs. 2.16-2.18); mu0 > 0, lambda0+2mu0 > 0.
 *  b:       dev, 3 x N body force, mean-free (Eq. 2.5), else BFCS_ERR_NONZERO_MEAN.
 *  E:       host, 6: prescribed mean strain; sets the k = 0 mode (Eq. 5.4 with
 *           the classical term of Eq. 2.24).
 *  tol:     stop once the residual r(eps^s) <= tol (tol = 0: run maxit sweeps).
 *  maxit:   >= 0 sweeps at most.
 *  eps_init: dev 6 x N warm start or NULL (NULL: eps^0 = eps^{b(0)} + E).
 *  eps_out: dev 6 x N, the returned strain eps^S (S = sweeps run).
 *  sig_out: dev 6 x N or NULL, sigma^S = L(x) eps^S.
 *  u_out:   dev 3 x N or NULL, the periodic displacement with sym grad u =
 *           eps^S - <eps^S> and zero mean (Eqs. 2.9-2.10).
 *  info:    host, filled on return (may be NULL).
 * Sweep s forms tau^s = (L - L0) eps^s, its transform, the residual r(eps^s)
 * and eps^{s+1}; the call stops after the first sweep with r(eps^s) <= tol,
 * or when the residual has not dropped by 10% over 100 sweeps (a stalled
 * fixed point, e.g. the FP32 rounding floor; status NOT_CONVERGED, info.stalled = 1).
 * Residual (reading of Eq. 5.11): r = ||i xi.sigma_hat + b_hat|| / D over modes
 * with xi != 0, D = ||b_hat|| + (2 pi / max N_a) |sigma_hat(0)|.  With a warm
 * start r(eps^0) is not evaluated (reported as +inf).
 * BFCS_MIXED plans (precision ladder): FP32 sweeps until r <= max(tol, 1e-4)
 * or the FP32 stall, then rounds of defect correction: the residual of the
 * FP64 strain is evaluated in float-float arithmetic (two floats, about
 * 48 significant bits, on the FP32 pipes; GB300's FP64 rate is a small
 * fraction of its FP32 rate) from the FP64 fields (sigma = L eps, its
 * transform, R_hat = i xi.sigma_hat + b_hat), and while it exceeds tol an FP32 solve with load R
 * and E = 0 gives a correction added to the FP64 strain and displacement
 * (at most 8 rounds; maxit bounds the FP32 sweeps of all rounds together).
 * The first round forms the FP64 strain as E + sym grad u from the FP64
 * displacement.  With tol >= 1e-9 the later rounds evaluate the defect of the
 * FP64 strain carried forward by adding each correction's FP32 strain (which
 * keeps it equal to E + sym grad u to ~1e-10 of its norm); with tol < 1e-9
 * every round re-forms it from the displacement.
 * info.resid is then that residual of the returned FP64 strain, and an
 * eps_init skips the first FP32 phase.  The FP32-only path cannot go below
 * its rounding floor (~1e-7 times the load's length scale in voxels).
 * Returns OK, NOT_CONVERGED, INVALID_ARG, NONZERO_MEAN, CUDA, TIMEOUT, DIVERGED.
 */
int bfcs_solve(bfcs_plan plan, const int8_t* phase, int nphases, const bfcs_lame* phases, bfcs_lame C0,
               const void* b, const double E[6], double tol, int maxit, const void* eps_init,
               void* eps_out, void* sig_out, void* u_out, bfcs_info* info);

/*
 * bfcs_solve_batched - `batch` independent solves sharing the plan's grid,
 * phases, C0, tol and maxit; member m reads its phase map translated by
 * problems[m].shift (phase(x) = phase0(x - chi), Eq. 3.3).
 *  problems: host array of `batch` members; infos: host array (may be NULL).
 * Returns the most severe member status.
 */
int bfcs_solve_batched(bfcs_plan plan, int batch, const bfcs_problem* problems, int nphases,
                       const bfcs_lame* phases, bfcs_lame C0, double tol, int maxit, bfcs_info* infos);

/*
 * bfcs_solve_group - batches on different grids in one loop (project feature:
 * the paper solves one problem at a time).  Item i runs items[i].batch
 * members (1..max_batch of its plan; bfcs_problem as for bfcs_solve_batched)
 * on items[i].plan, whose grid may differ from the other items'.  All plans
 * are FP32 or all FP64 (BFCS_MIXED: BFCS_ERR_UNSUPPORTED) and distinct; phases
 * and C0 are shared.  The sweeps of all items run together: one CUDA graph
 * launch per chunk of sweeps advances every item (the items' launches are
 * parallel branches of the graph, one stream per plan), and the loop ends when
 * every member of every item is done.  Each plan's stream waits for the loop
 * and finalises its own members; the call returns when all are written.
 * infos (per item, host, batch entries) may be NULL.  Returns the most severe
 * member status.  nitems in 1..BFCS_MAX_GROUP.
 */
#define BFCS_MAX_GROUP 8
typedef struct {
  bfcs_plan plan;
  int batch;
  const bfcs_problem* problems;
  bfcs_info* infos;
} bfcs_group_item;
int bfcs_solve_group(int nitems, const bfcs_group_item* items, int nphases, const bfcs_lame* phases,
                     bfcs_lame C0, double tol, int maxit);

/*
 * bfcs_translate_average - translated averaging (Eqs. 3.3-3.6) and the
 * dataset record of Eq. 3.7: for each integer shift chi_m (host, 3*nshift int32,
 * (x, y, z)) the microstructure phase(x) = phase0(x - chi_m) is solved with b
 * fixed, and the fields are summed in FP64 and divided by nshift:
 *  avg_out: dev, 30 x N double: <u> (3), <u>^(1) (3), <eps> (6), <eps>^(1) (6),
 *           <sigma> (6), <sigma>^(1) (6); ^(1) = weighted by the inclusion
 *           indicator V(x, chi) and still divided by nshift (Eqs. 3.5-3.6).
 *  hits_out: dev, N int32 or NULL: number of shifts with V(x, chi) = 1.
 *  infos: host, nshift entries or NULL.
 */
int bfcs_translate_average(bfcs_plan plan, const int8_t* phase, int nphases, const bfcs_lame* phases,
                           bfcs_lame C0, const void* b, const double E[6], int nshift,
                           const int32_t* shifts, double tol, int maxit, double* avg_out,
                           int32_t* hits_out, bfcs_info* infos);

/*
 * bfcs_ensemble_average - the ensemble dataset of Eq. 3.8: the fixed load b is
 * applied to each of nconf deterministic configurations X^j (phase maps with
 * no relation to one another, e.g. different samples), each is solved, and
 * the fields are averaged over the configurations as bfcs_translate_average
 * averages over translations (same 30 FP64 output fields; ^(1) weighted by
 * each configuration's own inclusion indicator, still divided by nconf).
 *  configs: host array of nconf device pointers, each N int8 phase ids.
 *  hits_out: dev, N int32 or NULL: number of configurations with phase != 0.
 *  infos:   host, nconf entries or NULL.
 * Other arguments and the batching (max_batch configurations per batched
 * solve) as bfcs_translate_average.
 */
int bfcs_ensemble_average(bfcs_plan plan, int nconf, const int8_t* const* configs, int nphases,
                          const bfcs_lame* phases, bfcs_lame C0, const void* b, const double E[6], double tol,
                          int maxit, double* avg_out, int32_t* hits_out, bfcs_info* infos);

/*
 * bfcs_radial_profile - the RVE diagnostic of Def. 2.2: for shells k = 0 ..
 * nbins-1 about `centre`, prof_out[k] = the largest pointwise norm of `field`
 * over the voxels whose periodic minimum-image distance d from the centre
 * satisfies k <= d < k + 1 (voxel centres at i + 0.5).
 *  field:   dev, ncomp x N in the plan's real type (float for BFCS_FP32,
 *           double for BFCS_FP64 and BFCS_MIXED), component-major.
 *  ncomp:   3 (vector: Euclidean norm) or 6 (symmetric tensor: sqrt(f : f),
 *           shears counted twice).
 *  centre:  host, 3 doubles in voxel units on the half-voxel lattice (2 c
 *           integral), so that every shell is decided in integer arithmetic.
 *  nbins:   1 .. 2048.
 *  prof_out: host, nbins doubles (0 for empty shells); counts_out: host, nbins
 *           voxel counts, or NULL.
 * Uses a plan-owned scratch (allocated on first use).  Errors: INVALID_ARG,
 * OOM, CUDA, TIMEOUT.
 */
int bfcs_radial_profile(bfcs_plan plan, const void* field, int ncomp, const double centre[3], int nbins,
                        double* prof_out, int64_t* counts_out);

/*
 * bfcs_rve_size - the RVE-size loop (Def. 2.2; Sec. 5: a body-force unit cell
 * that does not hold the RVE is enlarged and the problem solved again).  For
 * each cubic grid n = sizes[i] (ascending, multiples of the microstructure
 * cell cx x cy x cz; spheres as for bfcs_voxelize, tiled over the grid) the
 * BFCS problem (bfcs_body_force of support radius a, centred at the cell
 * corner nearest the grid centre, E = 0) is solved on a fresh plan with
 * `flags`, tol and maxit; bfcs_radial_profile of eps and sigma about the
 * centre over shells k < n/2 gives the RVE radius r: the smallest r such that
 * both profiles stay at most tol_f times their largest value in every shell
 * r <= k < n/2 (the fields vanish outside the RVE, relative to their maximum);
 * the grid holds the RVE when r + a/2 <= n/2 (room for an annulus of half the
 * support radius), and the loop stops there.
 *  records:  host, nsizes entries, filled for the grids solved.
 *  profiles: host, nsizes x 2 x (max sizes / 2) doubles (eps then sigma
 *            profile per grid, zero beyond n/2), or NULL.
 *  accepted: host, the index of the grid that holds the RVE, -1 if none.
 *  stream:   cudaStream_t of the plans and helper calls (NULL = default).
 * Allocates a plan and the grid's fields per step and frees them.
 * Returns the most severe solve status, or an error.
 */
typedef struct {
  int n;              /* cubic grid n^3 of this step */
  int r_rve;          /* RVE radius in voxels; -1: the fields do not fall below tol_f inside the grid */
  int contained;      /* 1: r_rve + a/2 <= n/2 (the loop stops at this grid) */
  int iters;          /* sweeps of the solve */
  int status;         /* status of the solve */
  double centre[3];   /* load centre (voxel units) */
  double resid;       /* residual of the returned strain */
  double eps_max;     /* largest shell maximum of |eps| */
  double sig_max;     /* largest shell maximum of |sigma| */
} bfcs_rve_record;
int bfcs_rve_size(int cx, int cy, int cz, int nsph, const int32_t* spheres, int nphases, const bfcs_lame* phases,
                  bfcs_lame C0, double a, int nsizes, const int* sizes, int flags, double tol, int maxit,
                  double tol_f, bfcs_rve_record* records, double* profiles, int* accepted, void* stream);

/*
 * bfcs_kernel_fit - the paper's nonlocal surrogate (Eqs. 6.5-6.6) for the
 * displacement operator (gamma = b): a radial kernel K(r) = sum_m c_m
 * B_m(r / delta), B_m the Bernstein basis of degree `degree` (0..7), zero for
 * r >= delta, defines L[u](x) = sum over voxel offsets 0 < |xi| < delta of
 * K(|xi|) (u(x + xi) - u(x)) on the periodic grid (voxel volume 1), and
 *   J(c) = sum_k sum_x |L[u_k](x) - Gamma_k(x)|^2 + lam |c|^2
 * (Tikhonov regularisation) is minimised by Adam (Kingma and Ba; betas 0.9,
 * 0.999, eps 1e-8, step lr, `iters` steps from c = 0); the exact minimiser
 * (G + lam I)^-1 g of the same quadratic is returned beside it.  Typically u_k
 * is the averaged displacement <u> of translated averaging or of an ensemble
 * (Eqs. 3.7-3.8) and Gamma_k = -b_k.  The sums over x are evaluated in Fourier
 * space (Parseval; K is even, so its transform is real).
 *  plan:    BFCS_FP64 or BFCS_MIXED plan of the grid (FP64 transforms; else
 *           BFCS_ERR_UNSUPPORTED); 2 delta < min(nx, ny, nz).
 *  u, gamma: host arrays of nload device pointers, each 3 x N double.
 *  coef_out: host, degree+1 (the Adam iterate); exact_out: host, degree+1 or
 *           NULL; loss_out: host, 2 (J of the Adam iterate, J of the exact
 *           minimiser) or NULL; gram_out: host (degree+1)^2 (G) or NULL;
 *           rhs_out: host degree+1 (g) or NULL.
 * Allocates its working arrays per call.
 */
int bfcs_kernel_fit(bfcs_plan plan, int nload, const void* const* u, const void* const* gamma, double delta,
                    int degree, double lam, int iters, double lr, double* coef_out, double* exact_out,
                    double* loss_out, double* gram_out, double* rhs_out);

/*
 * bfcs_kernel_apply - evaluates the nonlocal operator L[u] of bfcs_kernel_fit
 * for the kernel with Bernstein coefficients coef (host, degree+1) and
 * horizon delta: u, out dev 3 x N double (same plan requirements).
 */
int bfcs_kernel_apply(bfcs_plan plan, int degree, const double* coef, double delta, const void* u, void* out);

/*
 * bfcs_effective_stiffness - effective stiffness L* and inclusion strain
 * concentration A* of the periodic microstructure (Eqs. 6.1-6.3 and Eq. 3.2):
 * the classical problem (b = 0, Eq. 2.24) is solved under the six unit mean
 * strains E_J (J = xx yy zz yz xz xy, tensorial: a unit shear sets both
 * symmetric entries to 1), min(max_batch, 6) members at a time through
 * bfcs_solve_batched, and the fields are averaged in FP64 on the device.
 *  phase:  dev, N int8 phase ids; phases, C0, tol, maxit as for bfcs_solve.
 *  Lstar:  host, 36 doubles, row-major: Lstar[6 I + J] = <sigma_I> (cell
 *          average) for E = E_J, i.e. <sigma> = Lstar <eps> in tensorial
 *          components.
 *  Astar:  host, 36 doubles or NULL: Astar[6 I + J] = average of eps_I over
 *          the inclusion voxels (phase != 0) for E = E_J; NaN when there is
 *          no inclusion voxel.
 *  infos:  host, 6 entries (one per E_J) or NULL.
 * Uses the plan's translated-averaging scratch (allocated on first use).
 * Returns the most severe member status (as bfcs_solve_batched).
 */
int bfcs_effective_stiffness(bfcs_plan plan, const int8_t* phase, int nphases, const bfcs_lame* phases,
                             bfcs_lame C0, double tol, int maxit, double* Lstar, double* Astar,
                             bfcs_info* infos);

/*
 * Learned warm start / surrogate.  The paper proposes replacing the solver by
 * a learned map of the averaged nonlocal response (Sec. 6, Eqs. 6.9-6.10,
 * Fig. 5) without fixing a model; this library's model is a 4-level 3D U-net
 * on periodic volumes (BFCS_NET_PARAMS = 523654 parameters):
 *   input  4 channels: b / max|b| (3) and mu(x) / mu_max - 1/2;
 *   output 6 channels: eps mu_max / max|b| (normalised strain);
 *   widths 32, 32, 32, 48; two circular 3^3 convolutions per level with leaky
 *   ReLU (slope 0.1); 2^3 average pooling; 2^3 stride-2 transposed
 *   convolutions; skip concatenation [upsampled, skip]; 1^3 head.
 * Parameters ("params"): dev, BFCS_NET_PARAMS float (FP32 master copy); per
 * layer in the order e0a e0b e1a e1b e2a e2b e3a e3b u2 d2a d2b u1 d1a d1b u0
 * d0a d0b head, the weight in PyTorch's shape (conv: cout, cin, k, k, k;
 * transposed conv: cin, cout, 2, 2, 2) then the bias.  Every call rounds the
 * weights to BF16 on the device; activations are BF16, accumulation FP32.
 * Grids: nx, ny, nz multiples of 8 (three 2^3 poolings), any size otherwise.
 * Network tensors (x, y, target) are FP32, sample-major then channel-major:
 * element (sample s, channel c, voxel v) at [(s*C + c)*N + v].
 */
#define BFCS_NET_PARAMS 523654
#define BFCS_NET_TRAIN 1              /* bfcs_net_create: keep what the backward pass needs */

typedef struct bfcs_net_s* bfcs_net;

/* Number of parameters (BFCS_NET_PARAMS). */
long long bfcs_net_param_count(void);

/* Create a network context for nx x ny x nz grids and up to max_batch (1..1024)
 * samples per call; flags 0 (inference) or BFCS_NET_TRAIN.  The context owns
 * its activations (about 370 bytes per voxel and sample with BFCS_NET_TRAIN,
 * 180 without) and orders all work on stream.  Errors: INVALID_ARG, OOM. */
int bfcs_net_create(bfcs_net* out, int nx, int ny, int nz, int max_batch, int flags, void* stream);
int bfcs_net_destroy(bfcs_net net);

/* Waits for the context's stream and reports whether any network kernel gave
 * up a bounded wait (BFCS_ERR_TIMEOUT; its outputs are then unspecified).  The
 * condition is sticky: once set, the context's tensor-core convolutions return
 * without work and every later status call reports it; destroy and re-create
 * the context to continue. */
int bfcs_net_status(bfcs_net net);

/* Network input of one sample: x_out (dev, 4 x N float) from the body force b
 * (dev, 3 x N, float for BFCS_FP32 or double for BFCS_FP64 = precision) and
 * the phase map (dev, N int8; shear moduli from phases, host).  With eps (dev
 * 6 x N, same type as b) also the training target (dev, 6 x N float)
 * eps mu_max / max|b|; eps NULL: target_out unused. */
int bfcs_net_prepare(bfcs_net net, int precision, const void* b, const int8_t* phase, int nphases,
                     const bfcs_lame* phases, const void* eps, float* x_out, float* target_out);

/* y (dev, batch x 6 x N float) = network(x) for x (dev, batch x 4 x N float). */
int bfcs_net_forward(bfcs_net net, const float* params, int batch, const float* x, float* y);

/* Loss L = mean over the batch of ||y - target||^2 / ||target||^2 and its
 * gradient grad (dev, BFCS_NET_PARAMS float, overwritten) with respect to
 * params; loss_dev (dev, 1 double) or NULL.  Needs BFCS_NET_TRAIN.  The
 * result is deterministic (fixed-order reductions). */
int bfcs_net_grad(bfcs_net net, const float* params, int batch, const float* x, const float* target,
                  float* grad, double* loss_dev);

/* One Adam step (Kingma and Ba 2014; beta1 0.9, beta2 0.999, eps 1e-8, bias
 * correction for step t >= 1) on params with moments m, v (dev, float,
 * BFCS_NET_PARAMS each, zero before step 1). */
int bfcs_net_adam(bfcs_net net, float* params, const float* grad, float* m, float* v, long long t, float lr);

/* bfcs_net_grad followed by bfcs_net_adam (grad is the caller's scratch). */
int bfcs_net_train_step(bfcs_net net, float* params, float* grad, float* m, float* v, long long t, float lr,
                        int batch, const float* x, const float* target, double* loss_dev);

/* Predicted strain for batch samples (host arrays of dev pointers): b[i]
 * (3 x N), phase[i] (N int8), eps_out[i] (6 x N), element type float for
 * precision BFCS_FP32 or double for BFCS_FP64; processed max_batch at a time.
 * The result is a warm start for bfcs_solve / bfcs_problem.eps_init. */
int bfcs_net_predict(bfcs_net net, const float* params, int precision, int batch, const void* const* b,
                     const int8_t* const* phase, int nphases, const bfcs_lame* phases, void* const* eps_out);

/*
 * bfcs_surrogate_infer - the network's strain prediction on the plan's grid:
 * eps_pred (dev, 6 x N, element type of the plan: float for BFCS_FP32, double
 * otherwise) from b (dev, 3 x N, same type) and phase (dev, N int8).
 * weights: dev, BFCS_NET_PARAMS float (layout above).  The plan keeps an
 * inference context (created on the first call, ~180 bytes per voxel).
 * Errors: INVALID_ARG (grid not a multiple of 8, bad pointers or phases), OOM.
 */
int bfcs_surrogate_infer(bfcs_plan plan, const void* weights, const void* b, const int8_t* phase,
                         int nphases, const bfcs_lame* phases, void* eps_pred);

/*
 * Two steps of a sweep on their own, so that a sweep can be assembled around
 * transforms made elsewhere (e.g. a library FFT, kept as a comparison of the
 * fused passes).  Both run asynchronously on the plan's stream, in the plan's
 * real type (float for BFCS_FP32, double otherwise).
 *
 * bfcs_polarize - the polarization of Eq. 5.7, tau = (L(x) - L0) : eps, pointwise.
 *  phase:  dev, N int8 phase ids in [0, nphases) (ids outside the table read
 *          phase 0's moduli); phases, C0 as in bfcs_solve.
 *  eps:    dev, 6 x N (xx yy zz yz xz xy, tensorial shears); tau: dev, 6 x N
 *          (may alias eps).  C0 = {0, 0} is rejected; for sigma = L eps use
 *          bfcs_solve's outputs.
 *  Errors: INVALID_ARG (null pointers, invalid moduli), CUDA.
 *
 * bfcs_green_apply - the Green step of Algorithm 1 (Eq. 5.9 with U0 of Eqs.
 *  2.16-2.18 and the reference strain of Eqs. 2.8-2.9) on a dense half
 *  spectrum: complex values [c][z][y][kx], kx in [0, nx/2], rows of nx/2 + 1
 *  (the layout of a real-to-complex 3D transform), unnormalised (Eq. 4.3).
 *  spec:   dev, 6 components: tau_hat on entry, eps_hat^{s+1} on exit =
 *          U0 tau_hat + eps_hat^{b(0)} on modes with xi != 0 (reading R1 of xi),
 *          N E at k = 0, 0 on the other modes with xi = 0; unnormalised (an
 *          inverse transform that divides by N gives eps^{s+1}).
 *  b_hat:  dev, 3 components of the same layout: the transformed body force.
 *  E:      host, 6: prescribed mean strain.
 *  d_prev: dev, 3 components, or NULL: on entry xi . tau_hat of the previous
 *          sweep (zeros before the first), on exit that of this sweep;
 *  num_out: dev, 1 double, or NULL (with d_prev): the residual numerator of
 *          Eq. 5.11 (reading R4) of the strain whose polarization is on entry,
 *          sum over modes with xi != 0 of w |xi.tau_hat - d_prev|^2 (w = 1 on
 *          the kx = 0 and nx/2 planes, 2 elsewhere: the full spectrum's sum).
 *  Errors: INVALID_ARG (null pointers, only one of d_prev / num_out, invalid
 *          C0), CUDA.
 */
int bfcs_polarize(bfcs_plan plan, const int8_t* phase, int nphases, const bfcs_lame* phases, bfcs_lame C0,
                  const void* eps, void* tau);
int bfcs_green_apply(bfcs_plan plan, bfcs_lame C0, const double E[6], const void* b_hat, void* spec,
                     void* d_prev, double* num_out);

/*
 * bfcs_fft3d - the solver's 3D real transform on its own (Eqs. 4.3-4.4):
 *  direction -1: real (ncomp x N) -> half spectrum (ncomp x nz x ny x (nx/2+1)
 *  complex, unnormalised, Eq. 4.3); +1: half spectrum -> real with the 1/|N| of
 *  Eq. 4.4 NOT applied (multiply by 1/N yourself).  ncomp in 1..6.
 */
int bfcs_fft3d(bfcs_plan plan, int direction, int ncomp, const void* in, void* out);

/* Measurement hooks.
 * bfcs_kernel_launches: number of kernels this library has launched in the
 *   process so far (every launch, including sweeps skipped on device after
 *   convergence).
 * bfcs_profile_kernel: kind 0 = off, 1 = x pass, 2 = y passes, 3 = fused
 *   z/Green pass.  While on, every launch of that kind inside an executed sweep
 *   of a solve on this plan is bracketed by CUDA events on the plan's stream.
 * bfcs_profile_read: launches timed and their summed duration (ms) since the
 *   last read; resets the totals.  Both return a status.
 * bfcs_profile_green_io: with kind 3, how many of the timed z/Green launches
 *   (summed over members) read the previous sweep's divergence d_prev (3
 *   complex values per mode) and how many wrote d (the same size); every
 *   launch also reads and writes the 6-component spectrum and reads b_hat.
 *   Waits for the plan's stream; resets the counts. */
long long bfcs_kernel_launches(void);
int bfcs_profile_kernel(bfcs_plan plan, int kind);
int bfcs_profile_read(bfcs_plan plan, long long* launches, double* total_ms);
int bfcs_profile_green_io(bfcs_plan plan, long long* d_reads, long long* d_writes);

/* bfcs_plan_tuning - the plan's choice for the y passes of its FP32 sweeps
 * (project feature, not in the paper): variant 0..5 = column tile of 16, 8 or
 * 32 kx columns per block, then the same three with the two radices of the
 * line length ny = R1 R2 in the other order; 6 and 7 = tiles of 8 and 16
 * columns brought into shared memory by one tensor-memory-access copy per
 * block (when the driver provides the tensor-map encoder).  With
 * BFCS_AUTOTUNE the plan timed every variant valid for ny on its own buffers
 * and kept the fastest (variant_ms: 8 doubles, ms per y forward + inverse
 * pair, 0 = not timed); without it the variant is 0.  Any output pointer may
 * be NULL. */
int bfcs_plan_tuning(bfcs_plan plan, int* col_variant, int* col_tile, int* col_swap, double* variant_ms);

/* Residual history of the last solve on the plan: copies min(cap, iters)
 * values r(eps^s) into hist (host); returns the count or a negative status. */
int bfcs_last_history(bfcs_plan plan, double* hist, int cap);

/* bfcs_twiddles - host-only diagnostic (no device work): the twiddle table a
 * plan uploads for a line of length n (one of the grid sizes above) in
 * precision BFCS_FP32 (float pairs), BFCS_FP64 (double pairs) or BFCS_MIXED
 * (the ladder's float-float table: per entry the float pairs (hi, lo) of the
 * real part, then of the imaginary part), written to host memory `out` as
 * interleaved (re, im) values.  Entries 0..n-1 are
 * W^j = exp(-2 pi i j / n), the factors of the forward transform of Eq. 4.3.
 * Then, for each distinct first radix r of the line's four-step split that is
 * a multiple of 4 and at least 8 (the split's first radix, then its second),
 * a block [entry][n2] of (r/4 + 2) * (n/r) values: W^((n2 b) mod n) for
 * b = 1..3, then W^((4 n2 a) mod n) for a = 1..r/4-1, n2 < n/r; the
 * transform's first step reads them with consecutive n2 in consecutive
 * threads.  A float-float table holds instead one block [k1 - 1][n2] =
 * W^((n2 k1) mod n), k1 = 1..r1-1, n2 < n/r1, for the split's first radix r1.
 * Returns the number of complex entries (a NULL out or a too small cap only
 * returns the count) or BFCS_ERR_INVALID_ARG. */
int bfcs_twiddles(int n, int precision, void* out, int cap);

const char* bfcs_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* BFCS_H */
