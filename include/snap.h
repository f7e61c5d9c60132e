/*
 * snap.h -- C ABI of the B300 batched nonlinear constraint projection library (libsnap.so).
 *
 * The library computes, for every sample b of a batch, the projection of eq. (2) of the
 * paper (Sampling section; restated in "Jacobian Structure"):
 *
 *     u_b = argmin_u 1/2 || u - u_hat_b ||^2   subject to  h(u; theta_b) = 0,
 *
 * by Newton iterations on the KKT conditions of Appendix B ("newtonKKTsystem"):
 *
 *     [ W  J^T ] [du  ]     [ u - u_hat + J^T lambda ]
 *     [ J  0   ] [dlam] = - [ h(u)                   ],  W = I + sum_r lambda_r Hess h_r,
 *
 * with L = f + lambda^T h.  The Jacobian of h has a fixed block-sparse pattern: blocks are
 * independent across samples ("Jacobian Structure": block-diagonal over the batch) and,
 * for the families here, across time slices / frames too.
 *
 * Conventions for every entry point:
 *   - All numeric arrays are IEEE FP64, C order, and live in DEVICE memory unless the
 *     argument says "host".  The caller allocates and owns every buffer; the library
 *     never allocates inside snap_project / snap_project_backward / snap_constraint_residual
 *     / snap_batch_project, so those calls can be enqueued on a stream and captured into
 *     a CUDA graph.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls
 *     that take a stream are asynchronous with respect to the host; results are ready
 *     when the stream reaches that point.
 *   - Errors in arguments are reported by the return code and a thread-local message
 *     (snap_last_error).  Per-sample numerical outcomes (non-convergence, non-finite
 *     input, ...) are NOT call errors: they are written to snap_stats.status.
 *   - Device code never traps and never spins on other blocks (a programmatic dependent
 *     launch waits for its primary grid through griddepcontrol.wait, a hardware wait).
 *
 * Layouts (x fastest, the flattening of Appendix C):
 *   1-D families A/B:  u[b][k][i], k < nt time slices, i < nx points, x_i = i/nx periodic,
 *                      t_k = k/(nt-1).
 *   1-D families D/E:  u[b][k][i] as A/B, but x_i = i/(nx-1) on [0, 1] (both ends on the
 *                      grid; family E's flux update takes periodic neighbours).
 *   2-D family C:      w[b][f][c][j][i], f < nt frames, c = 0 (u) / 1 (v), j = y, i = x,
 *                      N x N periodic grid, dx = 1/N, t_f = f/(nt-1).
 *   Multipliers lambda[b][r] in the nominal row order (rows implied by other rows are
 *   listed but carry lambda = 0):
 *     A/B: IC rows (nx) | mass rows (nt) | energy rows (nt) | boundary rows (nt, family B)
 *          (only the row types enabled in snap_problem_desc.rows, in this order)
 *     C:   divergence rows [f][j][i] (nt*N*N) | kinetic-energy rows (nt)
 *     D:   Dirichlet rows (nt) | mass rows (nt) | Neumann rows (nt)
 *     E:   IC rows (nx) | mass rows (nt; slices 0..K implied) | flux rows [k-1][i] (K*nx)
 *   Parameters params[b][*]:
 *     A/B: g[0..nx-1] (IC values), r (energy decay rate), c[0..nt-1] (family B only)
 *     C:   K0, r2  (kinetic energy K_f = K0 exp(-r2 t_f))
 *     D:   u_L, m0 (Dirichlet value, mass target)
 *     E:   g[0..nx-1] (IC values; the mass target is dx sum g)
 */
#ifndef SNAP_H
#define SNAP_H

#include <stddef.h>

#if defined(__GNUC__)
#define SNAP_API __attribute__((visibility("default")))
#else
#define SNAP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct snap_problem *snap_problem_t;
typedef struct snap_batch *snap_batch_t;
typedef void *snap_stream_t; /* cudaStream_t */

typedef enum {
  SNAP_OK = 0,
  SNAP_ERR_INVALID_ARG = 1,  /* bad descriptor, null pointer, size out of range */
  SNAP_ERR_UNSUPPORTED = 2,  /* valid request this build does not implement */
  SNAP_ERR_CUDA = 3,         /* a CUDA runtime call failed (message has the CUDA error) */
  SNAP_ERR_NO_MEMORY = 4,    /* host or device allocation failed in a create call */
  SNAP_ERR_WORKSPACE = 5,    /* workspace pointer missing or smaller than required */
  SNAP_ERR_NOT_READY = 6     /* object used before it was completed (e.g. unbound batch) */
} snap_status;

/* Constraint families (Table I constraint types; Appendix A/C/D discretisations). */
typedef enum {
  /* 1-D space-time field: IC u(x_i,0) = g_i; per-slice mass dx sum_i u_{k,i} = M,
   * M = dx sum g; per-slice energy dx sum_i u_{k,i}^2 = E_k,
   * E_k = max(E0 exp(-r t_k), M^2 + energy_floor), E0 = dx sum g^2. */
  SNAP_FAMILY_A_MASS_ENERGY = 0,
  /* A plus the two-sided boundary invariant u_{k,0}^2 + u_{k,nx/2}^2 = c_k. */
  SNAP_FAMILY_B_BURGERS_BOUNDARY = 1,
  /* 2-D velocity per frame: central-difference divergence
   * (u_{i+1,j} - u_{i-1,j} + v_{i,j+1} - v_{i,j-1}) / (2 dx) = 0 and kinetic energy
   * 1/2 dx^2 sum(u^2 + v^2) = K0 exp(-r2 t_f). */
  SNAP_FAMILY_C_DIV_ENERGY = 2,
  /* Appendix C worked example (IC + left-Riemann mass differences).  Pattern queries
   * only; snap_project returns SNAP_ERR_UNSUPPORTED for it. */
  SNAP_FAMILY_TOY_LEFT_RIEMANN = 3,
  /* Boundary-condition regime of the Burgers problem (Appendix A; discretisation of
   * Appendix D): 1-D field on [0, 1], x_i = i dx, dx = 1 / (nx - 1), per slice k the
   * Dirichlet row u_{k,0} = u_L, the mass row dx sum_i u_{k,i} = m0 and the Neumann row
   * u_{k,nx-1} = u_{k,nx-2}.  params[b] = {u_L, m0}; rows grouped by type (nt Dirichlet, nt
   * mass, nt Neumann); nx in [4, 65536] (any parity), desc.rows must be 0.  Linear rows:
   * one Newton step; the adjoint applies the same projector to dL/du (grad_params =
   * dL/d(u_L, m0)). */
  SNAP_FAMILY_D_BURGERS_BC = 4,
  /* IC regime of the Burgers problem with Godunov flux rows (Appendix A "IC, mass,
   * Flux(k)"; the flux residual of Appendix D): 1-D field on x_i = i dx, dx = 1 / (nx - 1),
   * periodic neighbours, t_k = k dt, dt = 1 / (nt - 1), c = dt / dx.  Rows, in this order:
   * IC u^0_i = g_i (nx); mass dx sum_i u^k_i = M, M = dx sum_i g_i (nt); flux
   * u^k_i = G(u^{k-1})_i for k = 1..K, K = desc.n_flux (K nx rows, slice-major), with
   * G(v)_i = v_i - c (F(v_i, v_{i+1}) - F(v_{i-1}, v_i)) and F the Godunov flux of u^2/2
   * (minimum of u^2/2 over [a, b] when a <= b, maximum over [b, a] when a > b).  The mass
   * rows of slices 0..K are implied by the others (lambda 0; counted in h_inf).
   * params[b] = g[0..nx-1]; nx in [3, 512], 1 <= n_flux <= nt - 1, desc.rows must be 0.
   * The KKT point is evaluated directly (forward Godunov steps, backward substitution for
   * the multipliers; stats.iters = 1).  Adjoint: dL/du_hat is 0 on slices 0..K and
   * gbar - mean(gbar) on the others; grad_params = dL/dg.  u0 must be NULL. */
  SNAP_FAMILY_E_BURGERS_FLUX = 5,
  /* Heat equation, second constraint regime (Appendix A "Heat Equation Problems"; the
   * energy-evolution identity of the appendix "Energy Evolution Constraint"): 1-D field on
   * the periodic [0, 2 pi), x_i = i dx, dx = 2 pi / nx, t_k = k dt, dt = 1 / (nt - 1).  Rows,
   * in this order: IC u^0_i = g_i (nx); mass dx sum_i u^k_i = dx sum_i g_i (nt); PDE residual
   * (u^k_i - u^{k-1}_i) / dt - alpha/2 (D2 u^k + D2 u^{k-1})_i, k = 1..nt-1 (Crank-Nicolson,
   * (nt - 1) nx rows, slice-major; D2 the periodic second difference / dx^2); energy
   * evolution (E^k - E^{k-1}) / dt + alpha dx sum_i ((ubar_{i+1} - ubar_i) / dx)^2,
   * E^k = 1/2 dx sum_i (u^k_i)^2, ubar = (u^k + u^{k-1}) / 2, k = 1..nt-1 (nt - 1 rows).  The
   * mass and energy rows are implied by the IC and PDE rows (summation by parts: lambda 0,
   * counted in h_inf); the active rows are square, so the projection is the Crank-Nicolson
   * solution from g for every u_hat, and lambda solves J^T lambda = u_hat - u (backward
   * substitution in time; stats.iters = 1, kkt_inf = the largest active-row residual).
   * params[b] = {g_0..g_{nx-1}, alpha}, alpha >= 0 (else INFEASIBLE_PARAMS); nx in [3, 512];
   * desc.rows must be 0; u0 must be NULL.  Adjoint: dL/du_hat = 0, grad_params = dL/d(g,
   * alpha).  No workspace. */
  SNAP_FAMILY_F_HEAT_ENERGY = 6
} snap_family;

/* Row-type bits for snap_problem_desc.rows (1-D families). */
enum {
  SNAP_ROW_IC = 1,
  SNAP_ROW_MASS = 2,
  SNAP_ROW_ENERGY = 4,
  SNAP_ROW_BOUNDARY = 8
};

/* Per-sample outcome codes (snap_stats.status). */
enum {
  SNAP_SAMPLE_OK = 0,                /* ||F||_inf <= tol_kkt and ||h||_inf <= tol_h */
  SNAP_SAMPLE_MAXITER = 1,           /* max_iter Newton steps without convergence */
  SNAP_SAMPLE_LINESEARCH = 2,        /* no Armijo step within max_backtracks halvings */
  SNAP_SAMPLE_NONFINITE = 3,         /* NaN/Inf met in the input or the iteration */
  SNAP_SAMPLE_INFEASIBLE_PARAMS = 4, /* parameters admit no feasible point (c_k < 0) */
  SNAP_SAMPLE_RESIDUAL = 5,          /* KKT converged but some nominal row (one left out of
                                        the solve) has |h| > tol_h: inconsistent params */
  SNAP_SAMPLE_SINGULAR = 6,          /* singular Newton-KKT matrix */
  SNAP_SAMPLE_NOT_MINIMUM = 7,       /* converged to a KKT point whose KKT matrix has the
                                        wrong inertia (second-order condition fails) */
  SNAP_SAMPLE_DEVICE_WAIT = 8        /* a bounded wait inside a kernel ran out (an asynchronous
                                        copy did not complete): the slice was not solved */
};

/* Solver paths for snap_options.path. */
enum {
  SNAP_PATH_AUTO = 0,     /* fastest path valid for the call */
  SNAP_PATH_GENERAL = 1,  /* per-element FP64 Newton-KKT (any u0) */
  SNAP_PATH_MOMENT = 2,   /* moment-reduced Newton-KKT, FP64 throughout (u0 = u_hat only) */
  SNAP_PATH_MIXED = 3     /* moment-reduced Newton-KKT with the moments and the early Newton
                             steps on the FP32 pipe (float, then double-float), FP64 write
                             (u0 = u_hat only); AUTO picks it when u0 is NULL */
};

typedef struct {
  int family;          /* snap_family */
  int nx;              /* 1-D: points per slice (even, 4..512); 2-D: N (even, 4..64 in this
                          build; the uneven batch takes 4, 8, 16, 32 and 64) */
  int ny;              /* 2-D: must equal nx; 1-D: ignored */
  int nt;              /* 1-D: time slices; 2-D: frames (>= 2) */
  unsigned rows;       /* 1-D: SNAP_ROW_* mask (IC required); 0 = family default */
  double energy_floor; /* 1-D: floor in E_k (the workloads use 0.05) */
  int max_batch;       /* 0, or an upper bound on B checked by every call */
  int n_flux;          /* family E: Godunov flux steps K (1..nt-1); other families: 0 */
} snap_problem_desc;

typedef struct {
  int n_vars;              /* unknowns per sample */
  int n_rows_nominal;      /* rows per sample, including implied rows (lambda length) */
  int n_rows_active;       /* rows in the Newton-KKT system per sample */
  int n_params;            /* parameters per sample */
  long long pattern_nnz;   /* nonzeros of the Jacobian pattern over the nominal rows */
  int n_blocks;            /* independent blocks per sample (1-D: nt, 2-D: nt frames) */
} snap_info;

typedef struct {
  int iters;        /* Newton steps taken (max over the sample's blocks) */
  int backtracks;   /* line-search halvings (sum over blocks) */
  int status;       /* SNAP_SAMPLE_* (worst over blocks) */
  int corrections;  /* inertia corrections (sum over blocks) */
  double h_inf;     /* ||h(u)||_inf over ALL nominal rows at the returned u */
  double kkt_inf;   /* ||F||_inf over the active system at the returned (u, lambda) */
  double obj;       /* 1/2 ||u - u_hat||^2 */
} snap_stats;

typedef struct {
  double tol_kkt;      /* stop when ||F||_inf <= tol_kkt (default 1e-10) */
  double tol_h;        /* SNAP_SAMPLE_RESIDUAL threshold on ||h||_inf (default 1e-8) */
  int max_iter;        /* default 50 (at most 10000) */
  int max_backtracks;  /* default 30 (at most 200) */
  double armijo_c1;    /* accept t when phi(t) <= (1 - 2 c1 t) phi(0); default 1e-4 */
  double delta0;       /* first inertia-correction shift W + delta I (default 1e-8) */
  int max_corrections; /* 0 (default): plain Newton-Raphson on F = 0; 1..100: shift W until
                          the inertia of K is (n, m, 0), delta x10 each time */
  int path;            /* SNAP_PATH_* (default AUTO) */
  double w_keep;       /* each step keeps every diagonal entry of W at >= w_keep times its
                          current value (default 0.01; 0 disables) */
} snap_options;

/* Bounds-checked build (library libsnap_bc.so, compiled with -DSNAP_BOUNDS_CHECK): the
 * kernels' indexed global accesses are checked against their arrays' extents; the first
 * failing access is recorded in a device error word (bits 63..48: the access site, bits
 * 47..0: the index) and skipped instead of trapping.  Writes the word to *word (0: no
 * failure) and clears it when clear != 0; synchronous.  The paper has no counterpart: this is
 * a diagnostic build.  Errors: UNSUPPORTED in the normal build (word set to 0), CUDA. */
SNAP_API snap_status snap_bounds_error(unsigned long long *word, int clear);

/* Message of the last failed call on this host thread ("" if none).  Never NULL. */
SNAP_API const char *snap_last_error(void);

/* Library version string. */
SNAP_API const char *snap_version(void);

/* Fill *opt with the defaults listed in snap_options.  Returns SNAP_ERR_INVALID_ARG if
 * opt is NULL. */
SNAP_API snap_status snap_options_default(snap_options *opt);

/* Build a problem: validates the descriptor, fixes the row list and the Jacobian
 * sparsity pattern over the nominal rows ("Jacobian Structure": the pattern does not change
 * across iterations), marks the rows implied by others (left out of the solve), and builds
 * the symbolic structure once (1-D: per-slice 3x3 Schur blocks; 2-D: the constant
 * divergence Schur factor, see snap_problem_info).  Host call; allocates device memory for
 * shared constant data.  *out is set only on success.  Errors: INVALID_ARG (bad sizes,
 * ny != nx for C, IC bit missing, boundary bit for family A), NO_MEMORY, CUDA. */
SNAP_API snap_status snap_problem_create(const snap_problem_desc *desc, snap_problem_t *out);

/* Release a problem (NULL is a no-op).  Must not be in use by queued work. */
SNAP_API void snap_problem_destroy(snap_problem_t p);

/* Sizes of a problem.  Host call. */
SNAP_API snap_status snap_problem_info(snap_problem_t p, snap_info *info);

/* Sparsity pattern of the Jacobian over the nominal rows, CSR, HOST arrays:
 * row_ptr[n_rows_nominal + 1], col_idx[pattern_nnz] (columns ascending in a row).
 * Defined for every family (including the Appendix C toy family). */
SNAP_API snap_status snap_problem_pattern(snap_problem_t p, int *row_ptr, int *col_idx);

/* Which nominal rows take part in the solve (host array active[n_rows_nominal], 1/0). */
SNAP_API snap_status snap_problem_active_rows(snap_problem_t p, unsigned char *active);

/* Workspace bytes a call with batch size B needs (snap_project, snap_project_backward and
 * snap_constraint_residual share one requirement). */
SNAP_API snap_status snap_workspace_size(snap_problem_t p, int B, size_t *bytes);

/* Forward projection of B samples (eq. (2) solved by the Newton-KKT iteration of
 * Appendix B with an Armijo line search on phi = 1/2 ||F||^2 and per-block convergence
 * masks).
 *   u_hat   [B][n_vars]    targets (device, read)
 *   params  [B][n_params]  per-sample constraint parameters (device, read)
 *   u0      [B][n_vars]    starting point, or NULL for u0 = u_hat (device, read)
 *   u       [B][n_vars]    projected samples (device, written; may not alias inputs)
 *   lambda  [B][n_rows_nominal] multipliers, sign of L = f + lambda^T h (device, written)
 *   stats   [B]            per-sample statistics (device, written) or NULL
 *   opt                    NULL for defaults (host)
 *   workspace              snap_workspace_size(p, B) bytes of device scratch
 * Errors: INVALID_ARG (B < 0, B > max_batch, null required pointer, bad options),
 * WORKSPACE, UNSUPPORTED (toy family; MOMENT path with u0 != NULL), CUDA (launch failed).
 * B = 0 is a no-op. */
SNAP_API snap_status snap_project(snap_problem_t p, int B, const double *u_hat, const double *params,
                         const double *u0, double *u, double *lambda, snap_stats *stats,
                         const snap_options *opt, void *workspace, size_t workspace_bytes,
                         snap_stream_t stream);

/* Backward pass of the projection by the implicit-function theorem on
 * F(u, lambda; u_hat, theta) = 0 (Appendix B system at the solution, no inertia shift):
 *     K [a ; b] = [grad_u ; 0],  dL/du_hat = a,  dL/dtheta = -b^T dh/dtheta.
 * The per-block factors of K are rebuilt from (u, lambda): storing them in the forward pass and
 * reading them back measured slower than rebuilding them.
 *   grad_u      [B][n_vars]    upstream gradient dL/du (device, read)
 *   u, lambda   forward outputs (device, read)
 *   params      forward parameters (device, read)
 *   stats       forward stats (device) or NULL; samples whose status is not OK get NaN
 *   grad_u_hat  [B][n_vars]    (device, written; may not alias grad_u or u)
 *   grad_params [B][n_params]  (device, written; may not alias params) or NULL; layout of
 *                              params
 *   workspace   snap_workspace_size(p, B) bytes
 * Errors as snap_project. */
SNAP_API snap_status snap_project_backward(snap_problem_t p, int B, const double *grad_u,
                                  const double *u, const double *lambda, const double *params,
                                  const snap_stats *stats, double *grad_u_hat,
                                  double *grad_params, void *workspace, size_t workspace_bytes,
                                  snap_stream_t stream);

/* Constraint residual h(u; theta) of every nominal row (the per-type constraint error of
 * the Additional Results section is computed from it).
 *   h      [B][n_rows_nominal] (device, written) or NULL
 *   h_inf  [B] max_r |h_r| (device, written) or NULL */
SNAP_API snap_status snap_constraint_residual(snap_problem_t p, int B, const double *u,
                                     const double *params, double *h, double *h_inf,
                                     void *workspace, size_t workspace_bytes,
                                     snap_stream_t stream);

/* ---------------- the sampling loop around the projection ---------------- */

/* Workspace of snap_pcfm_sample (device, 256-byte aligned). */
SNAP_API snap_status snap_pcfm_workspace_size(snap_problem_t p, int B, size_t *bytes);

/* One PCFM sampling pass of the three-step variant (Sampling section, Eqs. 1-3): for
 * tau = k / n_steps, k = 0 .. n_steps-1: forward shoot u_hat_1 = u_tau + (1 - tau) v,
 * projection u_1 = argmin 1/2 ||u - u_hat_1||^2 s.t. h(u; params) = 0 (snap_project's
 * forward path, start u_hat_1), OT pull-back u_tau' = u_0 + tau' (u_1 - u_0).  The flow
 * model is replaced by the analytic velocity v(u, tau) = (x1 - u_0) + sigma0 (1 - tau) xi
 * (the straight-path OT velocity from the prior sample u_0 to the data sample x1, plus a
 * decaying perturbation along xi).
 *   u0, x1, xi: device [B][n_vars] (16-byte aligned); params as snap_project.  With this
 *   velocity u_0 cancels from the shoot after the pull-back (u_hat_1 = tau u_1 + (1 - tau) x1
 *   + sigma0 (1 - tau)^2 xi), so u0 is validated but not read.
 *   u: device [B][n_vars] out: u_1 of the last step (= the sample at tau = 1); it also holds
 *   the running u_1 between steps.  lambda, stats: of the last projection.
 * Asynchronous on stream, no allocation or synchronisation (capturable in a CUDA graph).
 * Errors: as snap_project; INVALID_ARG for n_steps outside [1, 100000] or a NaN sigma0. */
SNAP_API snap_status snap_pcfm_sample(snap_problem_t p, int B, int n_steps, double sigma0,
                                      const double *u0, const double *x1, const double *xi,
                                      const double *params, double *u, double *lambda,
                                      snap_stats *stats, const snap_options *opt,
                                      void *workspace, size_t workspace_bytes,
                                      snap_stream_t stream);

/* ---------------- forward projection without any allocation ---------------- */

/* Bytes of the library's static device scratch used by snap_project_noalloc (8 MiB). */
#define SNAP_NOALLOC_SCRATCH_BYTES 8388608

/* The 1-D forward projection of snap_project (families A and B, start u0 = u_hat, the path of
 * opt->path or the mixed-pipe path for AUTO/GENERAL), with its scratch memory taken from a
 * fixed library-owned device array instead of a caller-provided workspace.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate device memory where
 * they project (a host callback or plugin where cudaMalloc is not permitted, or an embedding
 * with no allocator of its own that cannot size a workspace per batch).  The caller still
 * passes all inputs and outputs, with the meaning and layout of snap_project.
 *   - It calls no cudaMalloc / cudaFree or any other allocating routine.
 *   - Limit: snap_workspace_size(p, B) must not exceed SNAP_NOALLOC_SCRATCH_BYTES (about
 *     80 bytes per time slice plus 64 per sample: e.g. B * nt <= 100,000 slices); larger
 *     batches are rejected with SNAP_ERR_WORKSPACE and a message.
 *   - The scratch is one file-scope __device__ array: every GPU that loads the library holds
 *     it until the process exits.  The first call on a device looks up its device address
 *     (cudaGetSymbolAddress, with that device current) and caches it; make that first call
 *     before any stream capture.
 *   - All calls share the array and it keeps the previous call's contents; nothing in it needs
 *     to start at zero (every byte a call reads was written earlier in the same call).  Calls
 *     whose work overlaps on the GPU (other streams, other threads) race on the array: order
 *     them on one stream or synchronise between them.
 * Errors: as snap_project (INVALID_ARG also when u aliases u_hat, or lambda aliases u or
 * u_hat: in-place calls are refused), plus UNSUPPORTED for families C, D and E.  Like every
 * entry point it clears snap_last_error() and snap_last_launch_count() on entry. */
SNAP_API snap_status snap_project_noalloc(snap_problem_t p, int B, const double *u_hat,
                                          const double *params, double *u, double *lambda,
                                          snap_stats *stats, const snap_options *opt,
                                          snap_stream_t stream);

/* ---------------- uneven batches in one persistent launch ---------------- */

/* A batch of instances of differing grid sizes and constraint families, projected together
 * (the block-diagonal batch of independent samples of Section 3, "Jacobian Structure",
 * extended to samples of different shapes and families): instance
 * i is one sample of problem probs[inst_problem[i]].  Supported families: A and B (1-D, the
 * mixed-pipe moment path, start u0 = u_hat) and C (2-D).  Instances of one problem form a
 * group; groups differ in shape.  snap_batch_project runs every instance in ONE persistent
 * kernel launch (after one memset of the workspace header): 2-D frames are taken from a work
 * queue by whole blocks, 1-D tiles of 32 time slices by single warps, and the last unit of an
 * instance to finish reduces that instance's statistics.  No allocation, no synchronisation:
 * capturable in a CUDA graph (see snap_batch_capture_graph).  Results are those of
 * snap_project on each instance (the same device code runs per slice / frame). */

/* How the persistent launch orders and shapes its work (the autotuner's search space). */
typedef struct {
  int ctas_per_sm;   /* resident blocks of 256 threads per SM (1 or 2; clamped to occupancy) */
  int order;         /* 0: 2-D frames first, then 1-D tiles;  1: 1-D tiles first */
  int pack_1d;       /* 1: a 1-D tile's 32 slices may span consecutive instances of a group;
                        0: tiles end at instance boundaries */
  int sort_1d;       /* 1-D groups in the queue: 0 creation order, 1 widest grid (nx) first */
  int tile_1d;       /* slices per 1-D work item: 16, 32 or 64 (a 64-slice item is two
                        32-slice tiles run by the same warp) */
  int lanes_1d;      /* lanes per slice of the 1-D load and write-back passes (2, 4 or 8) set
                        for every 1-D group; 0 keeps each group's own value (forward kernel;
                        the adjoint uses 4) */
} snap_batch_schedule;

/* Per-group lanes per slice (groups in problem order, n_groups entries as snap_batch_info
 * reports; 2-D groups read 0 and ignore what is set).  Set: each 1-D entry 2, 4 or 8, else
 * INVALID_ARG.  Host only, synchronous (uploads the group table). */
SNAP_API snap_status snap_batch_get_group_lanes(snap_batch_t b, int *lanes);
SNAP_API snap_status snap_batch_set_group_lanes(snap_batch_t b, const int *lanes);

/* Host arrays probs[n_problems], inst_problem[n_inst]; the problems must outlive the batch.
 * Allocates the batch's device tables on the current device (bind and project use it).
 * Errors: INVALID_ARG (null arrays, index out of range, n_inst < 0), UNSUPPORTED (a family
 * other than A, B, C, or a family C grid side other than 4, 8, 16, 32, 64), NO_MEMORY / CUDA
 * (device allocation). */
SNAP_API snap_status snap_batch_create(int n_problems, const snap_problem_t *probs, int n_inst,
                                       const int *inst_problem, snap_batch_t *out);
SNAP_API void snap_batch_destroy(snap_batch_t b);

/* Bind the device buffers of every instance (host arrays of device pointers, length n_inst):
 * u_hat[i] / u[i] [n_vars], params[i] [n_params], lambda[i] [n_rows_nominal], stats[i] one
 * snap_stats (layouts as in snap_project for one sample).  1-D u_hat / u must be 16-byte
 * aligned, everything else 8-byte aligned.  Copies the pointer table to the device
 * synchronously; call again to rebind (a captured graph then uses the new pointers).
 * Errors: INVALID_ARG (null or misaligned pointer; the message names the instance). */
SNAP_API snap_status snap_batch_bind(snap_batch_t b, const double *const *u_hat,
                                     const double *const *params, double *const *u,
                                     double *const *lambda, snap_stats *const *stats);

/* Workspace of snap_batch_project and snap_batch_project_grouped (device, 256-byte aligned). */
SNAP_API snap_status snap_batch_workspace_size(snap_batch_t b, size_t *bytes);

/* Project every bound instance in one persistent launch on stream.  t_ns (device,
 * [n_inst][2]) or NULL receives each instance's first-start and finish %globaltimer stamps
 * (ns).  opt: as snap_project (the path field is ignored).  Errors: NOT_READY (unbound),
 * WORKSPACE, INVALID_ARG (options), CUDA. */
SNAP_API snap_status snap_batch_project(snap_batch_t b, const snap_options *opt,
                                        unsigned long long *t_ns, void *workspace,
                                        size_t workspace_bytes, snap_stream_t stream);

/* The same work as snap_batch_project as plain snap_project launches, one per group (the
 * comparison baseline).  Needs each group's bound buffers to be contiguous and in instance
 * order (instance j+1 of a group directly after instance j, in every array); else
 * UNSUPPORTED. */
SNAP_API snap_status snap_batch_project_grouped(snap_batch_t b, const snap_options *opt,
                                                void *workspace, size_t workspace_bytes,
                                                snap_stream_t stream);

/* Current schedule / set one (host only: rebuilds and uploads the work lists, synchronous). */
SNAP_API snap_status snap_batch_get_schedule(snap_batch_t b, snap_batch_schedule *s);
SNAP_API snap_status snap_batch_set_schedule(snap_batch_t b, const snap_batch_schedule *s);

/* Autotuner: times snap_batch_project (CUDA events on stream, `reps` launches after one
 * warm-up, best of them) over the search space in three stages -- the 16 combinations of
 * ctas_per_sm, order, pack_1d and sort_1d (32-slice items, 4 lanes per slice); then tile_1d
 * in {16, 32, 64}; then, one 1-D group at a time, its lanes per slice in {2, 4, 8} --, keeps
 * the fastest on the batch and returns it in *best (lanes_1d = 0: the chosen per-group values
 * are in the batch, snap_batch_get_group_lanes) and its time in *best_ms (either may be
 * NULL).  Runs the
 * projection on the bound buffers (outputs are overwritten with the same results);
 * synchronous.  Errors: as snap_batch_project. */
SNAP_API snap_status snap_batch_autotune(snap_batch_t b, const snap_options *opt, void *workspace,
                                         size_t workspace_bytes, snap_stream_t stream, int reps,
                                         snap_batch_schedule *best, double *best_ms);

/* Capture snap_batch_project(b, opt, t_ns, workspace) into a CUDA graph owned by the batch
 * (replacing an earlier one) / launch that graph on stream.  The graph reads the bound
 * pointer table when it runs, so rebinding needs no new capture; a new schedule does. */
SNAP_API snap_status snap_batch_capture_graph(snap_batch_t b, const snap_options *opt,
                                              unsigned long long *t_ns, void *workspace,
                                              size_t workspace_bytes);
SNAP_API snap_status snap_batch_launch_graph(snap_batch_t b, snap_stream_t stream);

/* ---- adjoint of an uneven batch ----
 * The implicit-function adjoint of every bound instance (the per-instance operation of
 * snap_project_backward, Appendix B's KKT system at the solution) in ONE persistent launch:
 * the forward's work lists and schedule, 1-D tiles per warp and 2-D frames per block, each
 * instance's dL/dparams formed by the last of its units to finish (fixed order: the bits of
 * the per-group launches).  The forward binding supplies u (the solution), lambda, params and
 * stats (a sample whose forward status is not OK gets NaN gradients); the backward binding
 * below supplies, per instance, dL/du (input, n_vars doubles), dL/du_hat (output, n_vars) and
 * dL/dparams (output, n_params, or NULL: not formed; grad_params itself may be NULL).  1-D
 * instances need dL/du and dL/du_hat 16-byte aligned, 2-D 8-byte; the pointer table is copied
 * to the device, the caller keeps ownership.  The workspace is snap_batch_workspace_size's.
 * Errors: INVALID_ARG (null or misaligned), NOT_READY (forward or backward binding missing),
 * WORKSPACE, CUDA. */
SNAP_API snap_status snap_batch_bind_backward(snap_batch_t b, const double *const *grad_u,
                                              double *const *grad_u_hat,
                                              double *const *grad_params);
SNAP_API snap_status snap_batch_project_backward(snap_batch_t b, void *workspace,
                                                 size_t workspace_bytes, snap_stream_t stream);
/* The same adjoint as plain snap_project_backward launches, one per group (the comparison
 * baseline); every group's buffers of both bindings contiguous, else UNSUPPORTED. */
SNAP_API snap_status snap_batch_project_backward_grouped(snap_batch_t b, void *workspace,
                                                         size_t workspace_bytes,
                                                         snap_stream_t stream);
/* Capture snap_batch_project_backward into a CUDA graph owned by the batch / launch it. */
SNAP_API snap_status snap_batch_capture_graph_backward(snap_batch_t b, void *workspace,
                                                       size_t workspace_bytes);
SNAP_API snap_status snap_batch_launch_graph_backward(snap_batch_t b, snap_stream_t stream);

/* Shape of the batch: groups, 1-D tiles and 2-D frames in the current schedule's queues. */
SNAP_API snap_status snap_batch_info(snap_batch_t b, int *n_groups, int *n_tiles_1d,
                                     int *n_frames_2d);

/* ---------------- measurement helpers ---------------- */

/* Measured FP64 FMA rate of device `device` (FMAs per second) from a short in-register
 * kernel; used to state the arithmetic roofline.  Host call, synchronous. */
SNAP_API snap_status snap_measure_fp64_rate(int device, double *fma_per_s);

/* Per-kernel timing: when enabled (on = 1), every kernel launch of the library outside stream
 * capture is bracketed by two CUDA events recorded on its stream; with on = 2 the events are
 * also recorded into graphs being captured (as event nodes: after a replay they hold that
 * replay's times).  snap_profile_read waits for the recorded events of kernel `name` (e.g.
 * "k1d_mixed") and returns their summed elapsed time and count; snap_profile_reset drops all
 * records (call it only when no captured graph that records them will be replayed again).
 * Host calls. */
SNAP_API snap_status snap_profile_enable(int on);
SNAP_API snap_status snap_profile_reset(void);
SNAP_API snap_status snap_profile_read(const char *name, double *total_ms, long long *launches);

/* Number of kernels launched by the last snap_* call on this host thread. */
SNAP_API int snap_last_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SNAP_H */
