// The PCFM sampling loop around the projection (the three-step variant of the Sampling
// section): for tau_k = k / N, k = 0 .. N-1,
//   forward shoot   u_hat_1 = u_tau + (1 - tau) v(u_tau, tau)                 (Eq. 1)
//   projection      u_1 = argmin 1/2 ||u - u_hat_1||^2  s.t.  h(u) = 0       (Eq. 2)
//   OT pull-back    u_tau' = u_0 + tau' (u_1 - u_0),  tau' = tau_{k+1}        (Eq. 3)
// with the velocity model replaced by an analytic field (no trained flow model here): the
// straight-path OT velocity from the prior sample u_0 to a data sample x_1, plus a decaying
// perturbation,  v(u, tau) = (x_1 - u_0) + sigma0 (1 - tau) xi.
// The pull-back of step k and the shoot of step k + 1 are one elementwise kernel (u_tau is
// never stored): u_hat_1 = u_0 + tau (u_1 - u_0) + (1 - tau) v.  With this field u_0 cancels
// (v is the straight OT path from u_0): u_hat_1 = tau u_1 + (1 - tau) x_1 + sigma0 (1 - tau)^2 xi,
// three FP64 operations per value (FP64 is B300's scarce pipe) and three streams read instead
// of four; at tau = 0 (the first step) u_1 is not read.  The projection is the library's
// forward path.  One sampling pass = N x (this kernel + the projection kernels), all on one
// stream without allocation or synchronisation, so a pass can be captured in a CUDA graph.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kern_1dflux.h"
#include "snap_internal.h"

namespace {

// u_hat_1 for step tau over n values (pairs, then the odd last value); first = (tau == 0).
__global__ void __launch_bounds__(256)
k_pcfm_step(long long n, double tau, double sigma0, int first, const double2 *__restrict__ u1,
            const double2 *__restrict__ x1, const double2 *__restrict__ xi,
            double2 *__restrict__ uh) {
  const double rest = 1.0 - tau;
  const double s2 = sigma0 * rest * rest;
  const long long n2 = n >> 1;
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const long long j = n - 1;
    const double b = first ? 0.0 : ((const double *)u1)[j];
    ((double *)uh)[j] = fma(s2, ((const double *)xi)[j], fma(rest, ((const double *)x1)[j], tau * b));
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 x = __ldg(x1 + i), z = __ldg(xi + i);
    const double2 b = first ? make_double2(0.0, 0.0) : u1[i];
    double2 r;
    r.x = fma(s2, z.x, fma(rest, x.x, tau * b.x));
    r.y = fma(s2, z.y, fma(rest, x.y, tau * b.y));
    uh[i] = r;
  }
}

bool aligned16p(const void *p) { return ((uintptr_t)p & 15u) == 0; }

size_t pcfm_ws_bytes(const snap_problem *p, int B) {
  const size_t proj = (p->desc.family == SNAP_FAMILY_C_DIV_ENERGY)   ? ws_bytes_2d(p, B)
                      : (p->desc.family == SNAP_FAMILY_D_BURGERS_BC)   ? ws_bytes_1dbc(p, B)
                      : (p->desc.family == SNAP_FAMILY_E_BURGERS_FLUX) ? ws_bytes_1dflux(p, B)
                                                                       : ws_bytes_1d(p, B);
  return snap_align256(sizeof(double) * (size_t)B * p->info.n_vars) + proj;
}

}  // namespace

extern "C" {

SNAP_API snap_status snap_pcfm_workspace_size(snap_problem_t p, int B, size_t *bytes) {
  if (!p || !bytes || B < 0) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null argument or B < 0");
  if (p->desc.family == SNAP_FAMILY_TOY_LEFT_RIEMANN)
    return snap_fail_msg(SNAP_ERR_UNSUPPORTED, "the toy family supports pattern queries only");
  *bytes = pcfm_ws_bytes(p, B);
  return SNAP_OK;
}

SNAP_API snap_status snap_pcfm_sample(snap_problem_t p, int B, int n_steps, double sigma0,
                                      const double *u0, const double *x1, const double *xi,
                                      const double *params, double *u, double *lambda,
                                      snap_stats *stats, const snap_options *opt,
                                      void *workspace, size_t workspace_bytes,
                                      snap_stream_t stream) {
  snap_reset_launches();
  if (!p) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null problem");
  if (p->desc.family == SNAP_FAMILY_TOY_LEFT_RIEMANN)
    return snap_fail_msg(SNAP_ERR_UNSUPPORTED, "the toy family supports pattern queries only");
  if (B < 0 || (p->desc.max_batch > 0 && B > p->desc.max_batch))
    return snap_fail_msg(SNAP_ERR_INVALID_ARG, "batch size out of range");
  if (n_steps < 1 || n_steps > 100000)
    return snap_fail_msg(SNAP_ERR_INVALID_ARG, "n_steps must be in [1, 100000]");
  if (!(sigma0 == sigma0)) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "sigma0 is NaN");
  snap_options o;
  snap_options_default(&o);
  if (opt) o = *opt;
  if (snap_check_options(o) != SNAP_OK) return SNAP_ERR_INVALID_ARG;
  if (B == 0) return SNAP_OK;
  if (!u0 || !x1 || !xi || !params || !u || !lambda)
    return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null u0 / x1 / xi / params / u / lambda");
  if (!aligned16p(u0) || !aligned16p(x1) || !aligned16p(xi) || !aligned16p(u))
    return snap_fail_msg(SNAP_ERR_INVALID_ARG, "u0, x1, xi and u must be 16-byte aligned");
  if (u == u0 || u == x1 || u == xi)
    return snap_fail_msg(SNAP_ERR_INVALID_ARG, "u may not alias an input");
  const size_t need = pcfm_ws_bytes(p, B);
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255u))
    return snap_fail_msg(SNAP_ERR_WORKSPACE, "pcfm workspace missing, unaligned or too small");
  double *uh = (double *)workspace;
  void *pws = (char *)workspace + snap_align256(sizeof(double) * (size_t)B * p->info.n_vars);
  SolverOpts so;
  so.tol_kkt = o.tol_kkt;
  so.tol_h = o.tol_h;
  so.c1 = o.armijo_c1;
  so.delta0 = o.delta0;
  so.w_keep = o.w_keep;
  so.max_iter = o.max_iter;
  so.max_backtracks = o.max_backtracks;
  so.max_corrections = o.max_corrections;
  so.pad = 0;
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = (long long)B * p->info.n_vars;
  long long blocks = (n / 2 + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 148LL * 8) blocks = 148LL * 8;
  int launches = 0;
  for (int k = 0; k < n_steps; ++k) {
    const double tau = (double)k / (double)n_steps;
    k_pcfm_step<<<(int)blocks, 256, 0, s>>>(n, tau, sigma0, k == 0, (const double2 *)u,
                                           (const double2 *)x1, (const double2 *)xi,
                                           (double2 *)uh);
    launches++;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
      if (p->desc.family == SNAP_FAMILY_C_DIV_ENERGY)
        e = launch_2d_forward(p, B, uh, params, nullptr, u, lambda, stats, so,
                              SNAP_PATH_MIXED, pws, s);
      else if (p->desc.family == SNAP_FAMILY_D_BURGERS_BC)
        e = launch_1dbc_forward(p, B, uh, params, u, lambda, stats, so, pws, s);
      else if (p->desc.family == SNAP_FAMILY_E_BURGERS_FLUX)
        e = launch_1dflux_forward(p, B, uh, params, u, lambda, stats, so, pws, s);
      else
        e = launch_1d_forward(p, B, uh, params, nullptr, u, lambda, stats, so,
                              SNAP_PATH_MIXED, pws, s);
    }
    if (e != cudaSuccess) return snap_fail_msg(SNAP_ERR_CUDA, cudaGetErrorString(e));
  }
  snap_note_launch(launches);
  return SNAP_OK;
}

}  // extern "C"
