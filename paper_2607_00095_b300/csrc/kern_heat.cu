// Family F: the heat equation with IC, mass, Crank-Nicolson PDE-residual and energy-evolution
// rows (the paper's second heat-equation constraint operator, Appendix A; the energy identity
// of the appendix "Energy Evolution Constraint").
//
// Grid: x_i = i dx on the periodic [0, 2 pi), dx = 2 pi / nx; t_k = k dt, dt = 1 / (nt - 1).
// With A = I - (alpha dt / 2) D2 and B = I + (alpha dt / 2) D2 (D2 the periodic second
// difference) the PDE row block of slice k is (A u^k - B u^{k-1}) / dt.  The IC and PDE rows
// are square and nonsingular, and imply the mass and energy rows, so the projection is the
// single feasible point, the Crank-Nicolson solution u^k = A^-1 B u^{k-1} = 2 A^-1 u^{k-1} -
// u^{k-1}, u^0 = g, and its multipliers solve J^T lambda = u_hat - u by backward substitution
// in time (r = u_hat - u):
//   lambda^{nt-1} = dt A^-1 r^{nt-1},
//   lambda^k = A^-1 (dt r^k + 2 lambda^{k+1}) - lambda^{k+1}      (k = nt-2 .. 1),
//   lambda_IC = r^0 + (2 lambda^1 - A lambda^1) / dt.
// The implicit-function adjoint solves the same transposed system with gbar in place of r.
//
// A, symmetric positive definite and circulant, factors exactly as
//   A = (kappa / rho) (I - rho S)(I - rho S^-1),   kappa = alpha dt / (2 dx^2),
//   rho = 2 kappa / ((1 + 2 kappa) + sqrt(1 + 4 kappa)) in [0, 1)
// (S the periodic shift), so every solve is two periodic first-order recurrences.  One warp
// per sample keeps the slice in registers (lane l holds i = l E + q, q < E); a recurrence is a
// local pass over the lane's E values, a five-level warp scan of the block ends and the
// periodic wrap term rho^{i+1} z_{n-1} / (1 - rho^n).  The factor is computed once per sample
// and shared by every step of both time chains.  Arithmetic FP64 throughout.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "snap_bounds.cuh"
#include "snap_internal.h"

namespace {

constexpr unsigned kAll = 0xffffffffu;

__device__ __forceinline__ double h_nan_max(double a, double b) { return (a < b || b != b) ? b : a; }

__device__ __forceinline__ double h_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kAll, v, o);
  return v;
}

__device__ __forceinline__ double h_warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = h_nan_max(v, __shfl_xor_sync(kAll, v, o));
  return v;
}

// x^m, m >= 0, by binary powering
__device__ __forceinline__ double h_pow(double x, int m) {
  double r = 1.0;
  while (m > 0) {
    if (m & 1) r *= x;
    x *= x;
    m >>= 1;
  }
  return r;
}

// Per-lane constants of the factorisation of A for one sample.
template <int E>
struct HeatFactor {
  double rho, kap, scale, inv;   // scale = rho / kappa, inv = 1 / (1 - rho^n)
  double P[5];                   // (rho^E)^(2^j): multipliers of the block-end scans
  double pl[E];                  // rho^(q+1): carry into element q from the block before
  double pr[E];                  // rho^(E-q): carry into element q from the block after
  double pf[E];                  // rho^(i+1): wrap term of the forward pass (0 beyond nx)
  double pb[E];                  // rho^(n-i): wrap term of the backward pass (0 beyond nx)
};

template <int E>
__device__ __forceinline__ void heat_factor(HeatFactor<E> &f, double alpha, double dx, double dt,
                                            int nx, int lane) {
  f.kap = alpha * dt / (2.0 * dx * dx);
  const double root = sqrt(1.0 + 4.0 * f.kap);
  f.scale = 2.0 / ((1.0 + 2.0 * f.kap) + root);
  f.rho = f.kap * f.scale;
  const double rE = h_pow(f.rho, E);
  double p = rE;
#pragma unroll
  for (int j = 0; j < 5; ++j) { f.P[j] = p; p *= p; }
  f.inv = 1.0 / (1.0 - h_pow(f.rho, nx));
  const double base = h_pow(rE, lane);   // rho^(lane E)
#pragma unroll
  for (int q = 0; q < E; ++q) {
    f.pl[q] = h_pow(f.rho, q + 1);
    f.pr[q] = h_pow(f.rho, E - q);
    const int i = lane * E + q;
    f.pf[q] = (i < nx) ? base * f.pl[q] : 0.0;
    f.pb[q] = (i < nx) ? h_pow(f.rho, nx - i) : 0.0;
  }
}

// y <- A^-1 y (values beyond nx must be 0 on entry; they are 0 on exit)
template <int E>
__device__ __forceinline__ void heat_solve(const HeatFactor<E> &f, double (&y)[E], int nx,
                                           int lane) {
  // (I - rho S)^-1: z_i = y_i + rho z_{i-1}, periodic
  double run = 0.0;
#pragma unroll
  for (int q = 0; q < E; ++q) { run = fma(f.rho, run, y[q]); y[q] = run; }
  double v = y[E - 1];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const int d = 1 << j;
    const double t = __shfl_up_sync(kAll, v, d);
    if (lane >= d) v = fma(f.P[j], t, v);
  }
  double cin = __shfl_up_sync(kAll, v, 1);
  if (lane == 0) cin = 0.0;
  const int L = (nx - 1) / E, Lq = (nx - 1) - L * E;
  double zl = 0.0;
#pragma unroll
  for (int q = 0; q < E; ++q) {
    y[q] = fma(f.pl[q], cin, y[q]);
    if (q == Lq) zl = y[q];
  }
  zl = __shfl_sync(kAll, zl, L) * f.inv;
#pragma unroll
  for (int q = 0; q < E; ++q) y[q] = (lane * E + q < nx) ? fma(f.pf[q], zl, y[q]) : 0.0;
  // (I - rho S^-1)^-1: x_i = z_i + rho x_{i+1}, periodic
  run = 0.0;
#pragma unroll
  for (int q = E - 1; q >= 0; --q) { run = fma(f.rho, run, y[q]); y[q] = run; }
  v = y[0];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const int d = 1 << j;
    const double t = __shfl_down_sync(kAll, v, d);
    if (lane + d < 32) v = fma(f.P[j], t, v);
  }
  cin = __shfl_down_sync(kAll, v, 1);
  if (lane == 31) cin = 0.0;
#pragma unroll
  for (int q = 0; q < E; ++q) y[q] = fma(f.pr[q], cin, y[q]);
  const double x0 = __shfl_sync(kAll, y[0], 0) * f.inv;
#pragma unroll
  for (int q = 0; q < E; ++q) y[q] = (lane * E + q < nx) ? f.scale * fma(f.pb[q], x0, y[q]) : 0.0;
}

// Periodic neighbours v_{i-1}, v_{i+1} of the lane's elements.
template <int E>
__device__ __forceinline__ void heat_neighbours(const double (&v)[E], double (&lft)[E],
                                                double (&rgt)[E], int nx, int lane) {
  const int L = (nx - 1) / E, Lq = (nx - 1) - L * E;
  double last = 0.0;
#pragma unroll
  for (int q = 0; q < E; ++q)
    if (q == Lq) last = v[q];
  last = __shfl_sync(kAll, last, L);             // v_{nx-1}
  const double first = __shfl_sync(kAll, v[0], 0);   // v_0
  const double up = __shfl_up_sync(kAll, v[E - 1], 1);
  const double dn = __shfl_down_sync(kAll, v[0], 1);
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int i = lane * E + q;
    lft[q] = (q > 0) ? v[q - 1] : ((lane > 0) ? up : last);
    rgt[q] = (i == nx - 1) ? first : ((q < E - 1) ? v[q + 1] : dn);
  }
}

struct HeatArgs {
  int B, nx, nt, n_rows, off_mass, off_pde, off_energy;
  double dx, dt;
  const double *uh;       // forward: u_hat; adjoint: dL/du
  const double *params;   // [B][nx + 1] = g, alpha
  const double *u;        // adjoint / residual: the projection
  double *u_out;          // forward: u
  double *lam;            // forward: lambda (nominal rows)
  double *h;              // residual: h (nominal rows) or nullptr
  double *h_inf;          // residual: per-sample ||h||_inf or nullptr
  snap_stats *stats;      // forward: per-sample statistics or nullptr
  double *grad_uh;        // adjoint
  double *grad_params;    // adjoint
  const snap_stats *fwd_stats;   // adjoint: forward statistics or nullptr
  double tol_h;
};

// Residuals of the mass, PDE and energy rows of slice k >= 1 from u^k (cur) and u^{k-1}
// (prev): returns max |h| over the slice's rows (all lanes), writes h if hrow is given.
template <int E>
__device__ __forceinline__ double heat_slice_residual(const HeatArgs &a, int k, double alpha,
                                                      double sum_g, const double (&cur)[E],
                                                      const double (&prev)[E], double &e_prev,
                                                      double *hrow, int lane) {
  const double kap = alpha * a.dt / (2.0 * a.dx * a.dx);
  double s[E], sl[E], sr[E];
#pragma unroll
  for (int q = 0; q < E; ++q) s[q] = cur[q] + prev[q];
  heat_neighbours<E>(s, sl, sr, a.nx, lane);
  double mx = 0.0, su = 0.0, su2 = 0.0, sd2 = 0.0;
  const double idt = 1.0 / a.dt;
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int i = lane * E + q;
    if (i < a.nx) {
      // (A u^k - B u^{k-1}) / dt = ((1 + 2k) u^k - (1 - 2k) u^{k-1} - k (s_{i-1} + s_{i+1})) / dt
      const double r = ((1.0 + 2.0 * kap) * cur[q] - (1.0 - 2.0 * kap) * prev[q] -
                        kap * (sl[q] + sr[q])) * idt;
      if (hrow) hrow[a.off_pde + (k - 1) * a.nx + i] = r;
      mx = h_nan_max(mx, fabs(r));
      su += cur[q];
      su2 = fma(cur[q], cur[q], su2);
      const double d = sr[q] - s[q];     // 2 dx D+ ubar
      sd2 = fma(d, d, sd2);
    }
  }
  su = h_warp_sum(su);
  su2 = h_warp_sum(su2);
  sd2 = h_warp_sum(sd2);
  const double hm = a.dx * su - a.dx * sum_g;
  const double ek = 0.5 * a.dx * su2;
  const double he = (ek - e_prev) * idt + alpha * a.dx * sd2 / (4.0 * a.dx * a.dx);
  e_prev = ek;
  if (hrow && lane == 0) {
    hrow[a.off_mass + k] = hm;
    hrow[a.off_energy + (k - 1)] = he;
  }
  return h_nan_max(h_warp_max(mx), h_nan_max(fabs(hm), fabs(he)));
}

// Forward projection: u (time chain), lambda (backward substitution), statistics.
template <int E>
__global__ void __launch_bounds__(128) k_heat_forward(HeatArgs a) {
  const int lane = threadIdx.x & 31;
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= a.B) return;
  const int nx = a.nx, nt = a.nt;
  const double *pg = a.params + (size_t)b * (nx + 1);
  const double alpha = pg[nx];
  double *ub = a.u_out + (size_t)b * nx * nt;
  const double *uhb = a.uh + (size_t)b * nx * nt;
  double *lb = a.lam + (size_t)b * a.n_rows;
  const bool bad_alpha = !(alpha >= 0.0) || isinf(alpha);
  HeatFactor<E> f;
  heat_factor<E>(f, bad_alpha ? 0.0 : alpha, a.dx, a.dt, nx, lane);
  double cur[E], prev[E];
  double sum_g = 0.0, sq_g = 0.0;
  [[maybe_unused]] const long long nvar = (long long)a.B * nx * nt;
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int i = lane * E + q;
    cur[q] = (i < nx && snap_in_bounds(SNAP_SITE_HEAT_G, (long long)b * (nx + 1) + i,
                                       (long long)a.B * (nx + 1))) ? pg[i] : 0.0;
    if (i < nx && snap_in_bounds(SNAP_SITE_HEAT_U, (long long)b * nx * nt + i, nvar)) {
      ub[i] = cur[q];
      sum_g += cur[q];
      sq_g = fma(cur[q], cur[q], sq_g);
    }
  }
  sum_g = h_warp_sum(sum_g);
  double e_prev = 0.5 * a.dx * h_warp_sum(sq_g);
  double hmax = 0.0;                                   // IC rows: u^0 = g exactly
  hmax = h_nan_max(hmax, fabs(a.dx * sum_g - a.dx * sum_g));   // mass row of slice 0
  // forward chain
  for (int k = 1; k < nt; ++k) {
#pragma unroll
    for (int q = 0; q < E; ++q) prev[q] = cur[q];
    heat_solve<E>(f, cur, nx, lane);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = lane * E + q;
      cur[q] = (i < nx) ? 2.0 * cur[q] - prev[q] : 0.0;
      if (i < nx && snap_in_bounds(SNAP_SITE_HEAT_U, (long long)b * nx * nt + (long long)k * nx + i, nvar))
        ub[(size_t)k * nx + i] = cur[q];
    }
    hmax = h_nan_max(hmax, heat_slice_residual<E>(a, k, alpha, sum_g, cur, prev, e_prev, nullptr, lane));
  }
  // backward substitution for the multipliers (u read back: written above by this warp)
  __syncwarp();
  double lam1[E], obj = 0.0;
#pragma unroll
  for (int q = 0; q < E; ++q) lam1[q] = 0.0;
  for (int k = nt - 1; k >= 1; --k) {
    double y[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = lane * E + q;
      double r = 0.0;
      if (i < nx) {
        r = uhb[(size_t)k * nx + i] - ub[(size_t)k * nx + i];
        obj = fma(r, r, obj);
      }
      y[q] = (i < nx) ? fma(a.dt, r, 2.0 * lam1[q]) : 0.0;
    }
    heat_solve<E>(f, y, nx, lane);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = lane * E + q;
      const double lk = (i < nx) ? y[q] - lam1[q] : 0.0;
      if (i < nx && snap_in_bounds(SNAP_SITE_HEAT_LAM, a.off_pde + (long long)(k - 1) * nx + i, a.n_rows))
        lb[a.off_pde + (size_t)(k - 1) * nx + i] = lk;
      lam1[q] = lk;
    }
  }
  // IC multipliers: r^0 + (2 lambda^1 - A lambda^1) / dt
  {
    double ll[E], lr[E];
    heat_neighbours<E>(lam1, ll, lr, nx, lane);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = lane * E + q;
      if (i < nx) {
        const double r0 = uhb[i] - ub[i];
        obj = fma(r0, r0, obj);
        const double alam = (1.0 + 2.0 * f.kap) * lam1[q] - f.kap * (ll[q] + lr[q]);
        lb[i] = r0 + (2.0 * lam1[q] - alam) / a.dt;
      }
    }
  }
  for (int k = lane; k < nt; k += 32) lb[a.off_mass + k] = 0.0;
  for (int k = lane; k < nt - 1; k += 32) lb[a.off_energy + k] = 0.0;
  obj = h_warp_sum(obj);
  if (a.stats && lane == 0) {
    snap_stats st;
    st.iters = 1;
    st.backtracks = 0;
    st.corrections = 0;
    st.h_inf = hmax;
    st.kkt_inf = hmax;    // active rows (IC exact, PDE rows) at the returned u
    st.obj = 0.5 * obj;
    if (bad_alpha) st.status = SNAP_SAMPLE_INFEASIBLE_PARAMS;
    else if (!(hmax == hmax) || isinf(hmax) || !(obj == obj) || isinf(obj)) st.status = SNAP_SAMPLE_NONFINITE;
    else if (!(hmax <= a.tol_h)) st.status = SNAP_SAMPLE_RESIDUAL;
    else st.status = SNAP_SAMPLE_OK;
    a.stats[b] = st;
  }
}

// h(u) of every nominal row and its per-sample maximum.
template <int E>
__global__ void __launch_bounds__(128) k_heat_residual(HeatArgs a) {
  const int lane = threadIdx.x & 31;
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= a.B) return;
  const int nx = a.nx, nt = a.nt;
  const double *pg = a.params + (size_t)b * (nx + 1);
  const double alpha = pg[nx];
  const double *ub = a.u + (size_t)b * nx * nt;
  double *hrow = a.h ? a.h + (size_t)b * a.n_rows : nullptr;
  double cur[E], prev[E];
  double sum_g = 0.0, sq = 0.0, su0 = 0.0, hmax = 0.0;
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int i = lane * E + q;
    cur[q] = (i < nx) ? ub[i] : 0.0;
    if (i < nx) {
      const double gi = pg[i];
      sum_g += gi;
      su0 += cur[q];
      sq = fma(cur[q], cur[q], sq);
      const double hic = cur[q] - gi;
      if (hrow) hrow[i] = hic;
      hmax = h_nan_max(hmax, fabs(hic));
    }
  }
  sum_g = h_warp_sum(sum_g);
  su0 = h_warp_sum(su0);
  double e_prev = 0.5 * a.dx * h_warp_sum(sq);
  const double hm0 = a.dx * su0 - a.dx * sum_g;
  if (hrow && lane == 0) hrow[a.off_mass] = hm0;
  hmax = h_nan_max(h_warp_max(hmax), fabs(hm0));
  for (int k = 1; k < nt; ++k) {
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = lane * E + q;
      prev[q] = cur[q];
      cur[q] = (i < nx) ? ub[(size_t)k * nx + i] : 0.0;
    }
    hmax = h_nan_max(hmax, heat_slice_residual<E>(a, k, alpha, sum_g, cur, prev, e_prev, hrow, lane));
  }
  if (a.h_inf && lane == 0) a.h_inf[b] = hmax;
}

// Adjoint: J^T b = gbar by the same backward substitution; dL/du_hat = 0,
// dL/dg = b_IC, dL/dalpha = sum_k b^k . 1/2 D2 (u^k + u^{k-1}).
template <int E>
__global__ void __launch_bounds__(128) k_heat_backward(HeatArgs a) {
  const int lane = threadIdx.x & 31;
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= a.B) return;
  const int nx = a.nx, nt = a.nt;
  const double *pg = a.params + (size_t)b * (nx + 1);
  const double alpha = pg[nx];
  const double *gb = a.uh + (size_t)b * nx * nt;       // dL/du
  const double *ub = a.u + (size_t)b * nx * nt;
  double *gh = a.grad_uh + (size_t)b * nx * nt;
  const bool bad = (a.fwd_stats && a.fwd_stats[b].status != SNAP_SAMPLE_OK) || !(alpha >= 0.0) ||
                   isinf(alpha);
  for (size_t i = lane; i < (size_t)nx * nt; i += 32) gh[i] = bad ? NAN : 0.0;
  double *gp = a.grad_params ? a.grad_params + (size_t)b * (nx + 1) : nullptr;
  if (bad) {
    if (gp)
      for (int i = lane; i <= nx; i += 32) gp[i] = NAN;
    return;
  }
  HeatFactor<E> f;
  heat_factor<E>(f, alpha, a.dx, a.dt, nx, lane);
  double b1[E], cur[E], nxt[E], dalpha = 0.0;
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int i = lane * E + q;
    b1[q] = 0.0;
    nxt[q] = (i < nx) ? ub[(size_t)(nt - 1) * nx + i] : 0.0;   // u^k of the step below
  }
  for (int k = nt - 1; k >= 1; --k) {
    double y[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = lane * E + q;
      y[q] = (i < nx) ? fma(a.dt, gb[(size_t)k * nx + i], 2.0 * b1[q]) : 0.0;
      cur[q] = (i < nx) ? ub[(size_t)(k - 1) * nx + i] : 0.0;   // u^{k-1}
    }
    heat_solve<E>(f, y, nx, lane);
    // b^k . 1/2 D2 (u^k + u^{k-1})
    double s[E], sl[E], sr[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = lane * E + q;
      y[q] = (i < nx) ? y[q] - b1[q] : 0.0;
      b1[q] = y[q];
      s[q] = nxt[q] + cur[q];
    }
    heat_neighbours<E>(s, sl, sr, nx, lane);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = lane * E + q;
      if (i < nx) dalpha = fma(b1[q], 0.5 * (sl[q] - 2.0 * s[q] + sr[q]) / (a.dx * a.dx), dalpha);
      nxt[q] = cur[q];
    }
  }
  dalpha = h_warp_sum(dalpha);
  if (gp) {
    double ll[E], lr[E];
    heat_neighbours<E>(b1, ll, lr, nx, lane);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = lane * E + q;
      if (i < nx) {
        const double ab = (1.0 + 2.0 * f.kap) * b1[q] - f.kap * (ll[q] + lr[q]);
        gp[i] = gb[i] + (2.0 * b1[q] - ab) / a.dt;
      }
    }
    if (lane == 0) gp[nx] = dalpha;
  }
}

template <int E>
void heat_launch(int kind, const HeatArgs &a, cudaStream_t s) {
  const unsigned blocks = (unsigned)(((long long)a.B * 32 + 127) / 128);
  if (kind == 0) k_heat_forward<E><<<blocks, 128, 0, s>>>(a);
  else if (kind == 1) k_heat_residual<E><<<blocks, 128, 0, s>>>(a);
  else k_heat_backward<E><<<blocks, 128, 0, s>>>(a);
}

cudaError_t heat_dispatch(int kind, const HeatArgs &a, cudaStream_t s) {
  const int E = (a.nx + 31) / 32;
  if (E <= 1) heat_launch<1>(kind, a, s);
  else if (E <= 2) heat_launch<2>(kind, a, s);
  else if (E <= 4) heat_launch<4>(kind, a, s);
  else if (E <= 8) heat_launch<8>(kind, a, s);
  else if (E <= 16) heat_launch<16>(kind, a, s);
  else return cudaErrorNotSupported;
  return cudaGetLastError();
}

HeatArgs heat_args(const snap_problem *p, int B) {
  HeatArgs a = {};
  a.B = B;
  a.nx = p->desc.nx;
  a.nt = p->desc.nt;
  a.n_rows = p->info.n_rows_nominal;
  a.off_mass = a.nx;
  a.off_pde = a.nx + a.nt;
  a.off_energy = a.off_pde + (a.nt - 1) * a.nx;
  a.dx = 2.0 * 3.14159265358979323846 / a.nx;
  a.dt = 1.0 / (a.nt - 1);
  return a;
}

}  // namespace

cudaError_t launch_heat_forward(const snap_problem *p, int B, const double *u_hat,
                                const double *params, double *u, double *lambda,
                                snap_stats *stats, double tol_h, cudaStream_t s) {
  HeatArgs a = heat_args(p, B);
  a.uh = u_hat;
  a.params = params;
  a.u_out = u;
  a.lam = lambda;
  a.stats = stats;
  a.tol_h = tol_h;
  const int pid = snap_prof_begin(s, "k_heat_forward");
  const cudaError_t e = heat_dispatch(0, a, s);
  snap_prof_end(s, pid);
  snap_note_launch(1);
  return e;
}

cudaError_t launch_heat_residual(const snap_problem *p, int B, const double *u,
                                 const double *params, double *h, double *h_inf, cudaStream_t s) {
  HeatArgs a = heat_args(p, B);
  a.u = u;
  a.params = params;
  a.h = h;
  a.h_inf = h_inf;
  snap_note_launch(1);
  return heat_dispatch(1, a, s);
}

cudaError_t launch_heat_backward(const snap_problem *p, int B, const double *grad_u,
                                 const double *u, const double *params, const snap_stats *stats,
                                 double *grad_u_hat, double *grad_params, cudaStream_t s) {
  HeatArgs a = heat_args(p, B);
  a.uh = grad_u;
  a.u = u;
  a.params = params;
  a.fwd_stats = stats;
  a.grad_uh = grad_u_hat;
  a.grad_params = grad_params;
  const int pid = snap_prof_begin(s, "k_heat_backward");
  const cudaError_t e = heat_dispatch(2, a, s);
  snap_prof_end(s, pid);
  snap_note_launch(1);
  return e;
}
