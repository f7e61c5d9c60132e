// Internal definitions shared by the host side and the kernels of libsnap.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/snap.h"

#define SNAP_VERSION_STRING "snap-b300 0.1 (sm_103a, FP64)"

// Status ranks used when a sample's blocks are combined (worse outcome wins).
__host__ __device__ inline int snap_status_rank(int s) {
  switch (s) {
    case SNAP_SAMPLE_OK: return 0;
    case SNAP_SAMPLE_MAXITER: return 1;
    case SNAP_SAMPLE_LINESEARCH: return 2;
    case SNAP_SAMPLE_RESIDUAL: return 3;
    case SNAP_SAMPLE_INFEASIBLE_PARAMS: return 4;
    case SNAP_SAMPLE_NOT_MINIMUM: return 5;
    case SNAP_SAMPLE_SINGULAR: return 6;
    case SNAP_SAMPLE_NONFINITE: return 7;
    case SNAP_SAMPLE_DEVICE_WAIT: return 8;
    default: return 9;
  }
}

// Row-presence bits of a 1-D slice system (mass, energy, boundary).
enum { SL_MASS = 1, SL_ENERGY = 2, SL_BOUND = 4 };

// Per-block statistics kept in the workspace before the per-sample reduction.
struct BlockStat {
  int iters, backtracks, status, corrections;
  double h_inf, kkt_inf, obj;
};
static_assert(sizeof(BlockStat) == 40, "BlockStat layout");
static_assert(sizeof(snap_stats) == 40, "snap_stats layout");

// Solver options in the form the kernels read them.
struct SolverOpts {
  double tol_kkt, tol_h, c1, delta0, w_keep;
  int max_iter, max_backtracks, max_corrections, pad;
};

// Geometry of a 1-D problem as the kernels see it.
struct Geom1D {
  int nx, nt, ih;      // ih = nx / 2
  int rows;            // SL_* bits of the k >= 1 slice systems
  int has_ic;          // always 1 for families A/B
  int n_vars, n_rows, n_params;
  int off_mass, off_energy, off_bound;  // row offsets in lambda / h (-1 if absent)
  int p_rate, p_c;                      // parameter offsets (r, c_0) (-1 if absent)
  double dx, energy_floor;
};

// Workspace of the 1-D paths (device, caller-provided):
//   SampleDerived[B]  per-sample M, E0, residual of the rows at t = 0 left out of the solve
//   BlockStat[B*nt]   per-slice statistics
//   BwdContrib[B*nt]  per-slice backward contributions
//   double[B*nt]      per-slice residual maxima
struct SampleDerived {
  double M, E0, h0_inf, q;   // q = exp(-r dt): E0 exp(-r t_k) = E0 q^k
  // the same values as float pairs (hi, lo) for the double-float path; f = M^2 + floor
  float Mh, Ml, E0h, E0l, qh, ql, fh, fl;
};

// Per-slice contributions of the backward pass to dL/dtheta (summed per sample):
// b_m, b_e e^{-r t} (exp branch of E_k), b_e (floor branch), -b_e t E0 e^{-r t}.
struct BwdContrib {
  double bm, bex, bfl, br;
};

struct snap_problem {
  snap_problem_desc desc;
  snap_info info;
  Geom1D g1;
  // CSR pattern over the nominal rows (host) and the active-row flags (host)
  int *row_ptr;
  int *col_idx;
  unsigned char *active;
  // 2-D: constant Schur factor of the divergence rows (device), see kern_2d.cu
  void *dev_const;
  size_t dev_const_bytes;
  void *host_const;    // host copy of the 2-D factor (uploaded on create or first use)
  int n2d_band;        // half bandwidth of the class factor
  int n2d_m;           // unknowns of one parity-class system (M*M - 1)
};

// Error-message helpers of snap_api.cu for the other entry-point files.
snap_status snap_fail_msg(snap_status st, const char *msg);
void snap_clear_error();
snap_status snap_check_options(const snap_options &o);

// Kernel-launch bookkeeping (per host thread) and optional event timing (snap_profile.cu).
void snap_note_launch(int n);
void snap_reset_launches();
int snap_prof_begin(cudaStream_t s, const char *name);
void snap_prof_end(cudaStream_t s, int id);

// Host-side launchers (kern_1d.cu / kern_2d.cu).
cudaError_t launch_1d_forward(const snap_problem *p, int B, const double *u_hat,
                              const double *params, const double *u0, double *u, double *lambda,
                              snap_stats *stats, const SolverOpts &o, int path, void *ws,
                              cudaStream_t s);
cudaError_t launch_1d_backward(const snap_problem *p, int B, const double *grad_u,
                               const double *u, const double *lambda, const double *params,
                               const snap_stats *stats, double *grad_u_hat, double *grad_params,
                               void *ws, cudaStream_t s);
cudaError_t launch_1d_residual(const snap_problem *p, int B, const double *u,
                               const double *params, double *h, double *h_inf, void *ws,
                               cudaStream_t s);
size_t ws_bytes_1d(const snap_problem *p, int B);
void launch_1d_bwd_mixed(const Geom1D &g, int B, const double *grad_u, const double *u,
                         const double *lambda, const double *params, const snap_stats *stats,
                         const SampleDerived *sd, double *grad_u_hat, double *grad_params,
                         BwdContrib *contrib, cudaStream_t s);
void launch_1d_mixed(const Geom1D &g, int B, const double *u_hat, const double *params,
                     const SampleDerived *sd, double *u, double *lambda, BlockStat *bst,
                     const SolverOpts &o, int blocks_per_sm, cudaStream_t s);

cudaError_t setup_2d(snap_problem *p);
cudaError_t ensure_2d_factor(const snap_problem *p);
void teardown_2d(snap_problem *p);
cudaError_t launch_2d_forward(const snap_problem *p, int B, const double *w_hat,
                              const double *params, const double *w0, double *w, double *lambda,
                              snap_stats *stats, const SolverOpts &o, int path, void *ws,
                              cudaStream_t s);
cudaError_t launch_2d_backward(const snap_problem *p, int B, const double *grad_w,
                               const double *w, const double *lambda, const double *params,
                               const snap_stats *stats, double *grad_w_hat, double *grad_params,
                               void *ws, cudaStream_t s);
cudaError_t launch_2d_residual(const snap_problem *p, int B, const double *w,
                               const double *params, double *h, double *h_inf, void *ws,
                               cudaStream_t s);
size_t ws_bytes_2d(const snap_problem *p, int B);
bool supported_2d(int N);
void launch_finalize_stats(int B, int nblk, const BlockStat *bst, double tol_h, snap_stats *stats,
                           cudaStream_t s);

// Family D (kern_1dbc.cu).
size_t ws_bytes_1dbc(const snap_problem *p, int B);
cudaError_t launch_1dbc_forward(const snap_problem *p, int B, const double *u_hat,
                                const double *params, double *u, double *lambda,
                                snap_stats *stats, const SolverOpts &o, void *ws,
                                cudaStream_t s);
cudaError_t launch_1dbc_backward(const snap_problem *p, int B, const double *grad_u,
                                 const snap_stats *stats, double *grad_u_hat, double *grad_params,
                                 void *ws, cudaStream_t s);
cudaError_t launch_1dbc_residual(const snap_problem *p, int B, const double *u,
                                 const double *params, double *h, double *h_inf, void *ws,
                                 cudaStream_t s);

// Family F (kern_heat.cu).
cudaError_t launch_heat_forward(const snap_problem *p, int B, const double *u_hat,
                                const double *params, double *u, double *lambda,
                                snap_stats *stats, double tol_h, cudaStream_t s);
cudaError_t launch_heat_residual(const snap_problem *p, int B, const double *u,
                                 const double *params, double *h, double *h_inf, cudaStream_t s);
cudaError_t launch_heat_backward(const snap_problem *p, int B, const double *grad_u,
                                 const double *u, const double *params, const snap_stats *stats,
                                 double *grad_u_hat, double *grad_params, cudaStream_t s);

// Alignment helper for workspace carving.
inline size_t snap_align256(size_t x) { return (x + 255) & ~(size_t)255; }
