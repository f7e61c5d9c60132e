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

#include "df64.cuh"
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
  // grid constants formed on the host (FP64 divisions and conversions in the kernel would be
  // FP64-pipe work for every thread ahead of the time chain): dt / (2 dx^2), 1 / dt, 1 / (4 dx),
  // and dx, dx / 2, 1 / dt, dt, 1 / (2 dx^2) in double-float
  double kfac, idt, ce_fac;
  df64 dx_d, half_dx_d, idt_d, dt_d, cd2_d;
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

// ---------------------------------------------------------------------------------------------
// The time chains in double-float on the FP32 pipe (df64.cuh: ~48-bit significands), one warp per
// sample.  The FP64 pipe of a B300 SM retires 2 lanes per clock against 128 FP32 lanes, and the
// chains above are FP64-bound; here FP64 is left only for the conversion of the written u and
// lambda to double (one addition per value).  The factor constants are formed in FP64 once per
// sample and split.  The stored u and lambda are the double roundings of the double-float chain
// values, so the residual of a Crank-Nicolson step is the local error of the double-float solve
// (a few units of 2^-47 relative, times (1 + 4 kappa) / dt), far inside the FP64 stopping
// tolerance, and the stored u agrees with the FP64 chain to ~1e-12 relative.

// a b + c with one error-free transformation on the leading parts (the accuracy of df_add_fast)
__device__ __forceinline__ df64 hd_fma(df64 a, df64 b, df64 c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const df64 s = df_two_sum(p, c.hi);
  return df_fast_two_sum(s.hi, s.lo + (e + c.lo));
}

// Two independent hd_fma, statement by statement interleaved (two latency chains in flight)
__device__ __forceinline__ void hd_fma2(df64 a1, df64 b1, df64 c1, df64 a2, df64 b2, df64 c2,
                                        df64 &r1, df64 &r2) {
  const float p1 = a1.hi * b1.hi, p2 = a2.hi * b2.hi;
  float e1 = fmaf(a1.hi, b1.hi, -p1), e2 = fmaf(a2.hi, b2.hi, -p2);
  e1 = fmaf(a1.hi, b1.lo, e1);
  e2 = fmaf(a2.hi, b2.lo, e2);
  e1 = fmaf(a1.lo, b1.hi, e1);
  e2 = fmaf(a2.lo, b2.hi, e2);
  const float s1 = p1 + c1.hi, s2 = p2 + c2.hi;
  const float q1 = s1 - p1, q2 = s2 - p2;
  const float t1 = (p1 - (s1 - q1)) + (c1.hi - q1), t2 = (p2 - (s2 - q2)) + (c2.hi - q2);
  const float l1 = t1 + (e1 + c1.lo), l2 = t2 + (e2 + c2.lo);
  const float h1 = s1 + l1, h2 = s2 + l2;
  r1 = df64(h1, l1 - (h1 - s1));
  r2 = df64(h2, l2 - (h2 - s2));
}

__device__ __forceinline__ df64 hd_shfl(df64 v, int src) {
  return df64(__shfl_sync(kAll, v.hi, src), __shfl_sync(kAll, v.lo, src));
}
__device__ __forceinline__ df64 hd_shfl_up(df64 v, int d) {
  return df64(__shfl_up_sync(kAll, v.hi, d), __shfl_up_sync(kAll, v.lo, d));
}
__device__ __forceinline__ df64 hd_shfl_down(df64 v, int d) {
  return df64(__shfl_down_sync(kAll, v.hi, d), __shfl_down_sync(kAll, v.lo, d));
}
__device__ __forceinline__ df64 hd_warp_sum(df64 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = df_add_fast(v, df64(__shfl_xor_sync(kAll, v.hi, o), __shfl_xor_sync(kAll, v.lo, o)));
  return v;
}
// v[j] for a run-time j (warp-uniform) by selects: an indexed register array would go to local
// memory, and an if per element would split the caller's straight-line code into blocks
template <int E>
__device__ __forceinline__ df64 hd_pick(const df64 (&v)[E], int j) {
  df64 r = v[0];
#pragma unroll
  for (int q = 1; q < E; ++q) {
    r.hi = (j == q) ? v[q].hi : r.hi;
    r.lo = (j == q) ? v[q].lo : r.lo;
  }
  return r;
}

// NaN-propagating maximum of magnitudes (float: the residual's size, not its value, is kept)
__device__ __forceinline__ float hd_nan_max(float a, float b) { return (a < b || b != b) ? b : a; }
__device__ __forceinline__ float hd_warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = hd_nan_max(v, __shfl_xor_sync(kAll, v, o));
  return v;
}

// A double to double-float: the integer split for values in its range, the conversion
// otherwise (values outside [2^-74, 2^57], infinities and NaN, which then propagate); the
// warp takes the conversion branch only when one of its lanes needs it.
template <int E>
__device__ __forceinline__ void hd_load(const double (&x)[E], df64 (&v)[E]) {
  bool ok = true;
#pragma unroll
  for (int q = 0; q < E; ++q) ok &= df_split_trunc(x[q], v[q].hi, v[q].lo);
  if (!__all_sync(kAll, ok)) {
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = df64(x[q]);
  }
}

// The factor constants in double-float, with the lane masks folded into the multipliers so that
// the solve has no lane-dependent branch: Pf[j] / Pb[j] are the scan multipliers of level j,
// 0 on the lanes that take no contribution at that level (lane < 2^j, lane + 2^j > 31), and
// pl / pr are 0 on lane 0 / lane 31 (no block before / after).
template <int E>
struct HeatFactorDF {
  df64 rho, comb, inv;   // comb = (rho / kappa) / (1 - rho^2)
  df64 Pf[5], Pb[5];
  df64 pl[E], pr[E], pf[E], pb[E];
};

template <int E>
__device__ __forceinline__ void heat_factor_df(HeatFactorDF<E> &d, double alpha, double dx,
                                               double dt, int nx, int lane) {
  HeatFactor<E> f;
  heat_factor<E>(f, alpha, dx, dt, nx, lane);
  d.rho = df64(f.rho);
  d.comb = df64(f.scale / (1.0 - f.rho * f.rho));
  d.inv = df64(f.inv);
  const df64 zero(0.0f, 0.0f);
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    d.Pf[j] = (lane >= (1 << j)) ? df64(f.P[j]) : zero;
    d.Pb[j] = (lane + (1 << j) < 32) ? df64(f.P[j]) : zero;
  }
#pragma unroll
  for (int q = 0; q < E; ++q) {
    d.pl[q] = (lane > 0) ? df64(f.pl[q]) : zero;
    d.pr[q] = (lane < 31) ? df64(f.pr[q]) : zero;
    d.pf[q] = df64(f.pf[q]);
    d.pb[q] = df64(f.pb[q]);
  }
}

// y <- A^-1 y in double-float (values beyond nx are 0 on entry and on exit).  The two
// first-order factors commute, (I - rho S)(I - rho S^-1) has the partial fractions
//   ((I - rho S)^-1 + (I - rho S^-1)^-1 - I) / (1 - rho^2),
// so the forward and the backward periodic recurrence both run on y, independently (two
// interleaved chains instead of one after the other), and
//   A^-1 y = (rho / kappa) / (1 - rho^2) (F + G - y).
// rho solves kappa rho^2 - (1 + 2 kappa) rho + kappa = 0, i.e. kappa (1 - rho)^2 = rho, so the
// factor times the bound |F|, |G| <= |y|_inf / (1 - rho) is 1 / (1 + rho) <= 1: the rounding
// of the combination stays within a few units of 2^-47 |y|_inf.
template <int E>
__device__ __forceinline__ void heat_solve_df(const HeatFactorDF<E> &f, df64 (&y)[E], int nx,
                                              int lane) {
  const df64 zero(0.0f, 0.0f);
  df64 F[E], G[E];
  // F: z_i = y_i + rho z_{i-1}; G: x_i = y_i + rho x_{i+1} (each periodic)
  df64 rf = zero, rb = zero;
#pragma unroll
  for (int q = 0; q < E; ++q) {
    hd_fma2(f.rho, rf, y[q], f.rho, rb, y[E - 1 - q], rf, rb);
    F[q] = rf;
    G[E - 1 - q] = rb;
  }
  // block-end scans; a lane that takes no contribution has a zero multiplier (the shuffled
  // value there is its own, finite), so every lane runs the same instructions
  df64 vf = F[E - 1], vb = G[0];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const int d = 1 << j;
    const df64 tf = hd_shfl_up(vf, d);
    const df64 tb = hd_shfl_down(vb, d);
    hd_fma2(f.Pf[j], tf, vf, f.Pb[j], tb, vb, vf, vb);
  }
  const df64 cf = hd_shfl_up(vf, 1), cb = hd_shfl_down(vb, 1);   // times pl = 0 / pr = 0 at the ends
  const int L = (nx - 1) / E, Lq = (nx - 1) - L * E;
#pragma unroll
  for (int q = 0; q < E; ++q) hd_fma2(f.pl[q], cf, F[q], f.pr[q], cb, G[q], F[q], G[q]);
  // the periodic wrap terms: rho^(i+1) z_{n-1} / (1 - rho^n), rho^(n-i) x_0 / (1 - rho^n)
  const df64 zl = hd_shfl(hd_pick<E>(F, Lq), L) * f.inv;
  const df64 x0 = hd_shfl(G[0], 0) * f.inv;
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const df64 t = df_add_fast(hd_fma(f.pf[q], zl, F[q]), hd_fma(f.pb[q], x0, G[q]));
    const df64 v = f.comb * df_sub_fast(t, y[q]);
    y[q] = (lane * E + q < nx) ? v : zero;
  }
}

// Periodic neighbours in double-float (0 beyond nx).
template <int E>
__device__ __forceinline__ void heat_neighbours_df(const df64 (&v)[E], df64 (&lft)[E],
                                                   df64 (&rgt)[E], int nx, int lane) {
  const int L = (nx - 1) / E, Lq = (nx - 1) - L * E;
  const df64 last = hd_shfl(hd_pick<E>(v, Lq), L);
  const df64 first = hd_shfl(v[0], 0);
  const df64 up = hd_shfl_up(v[E - 1], 1);
  const df64 dn = hd_shfl_down(v[0], 1);
  const df64 zero(0.0f, 0.0f);
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int i = lane * E + q;
    const df64 l = (q > 0) ? v[q - 1] : ((lane > 0) ? up : last);
    const df64 r = (i == nx - 1) ? first : ((q < E - 1) ? v[q + 1] : dn);
    lft[q] = (i < nx) ? l : zero;     // 0 beyond nx: no per-element guard in the callers
    rgt[q] = (i < nx) ? r : zero;
  }
}

// Per-sample constants of the residual rows in double-float.
struct HeatRowsDF {
  df64 c1, c2, c3;     // (1 + 2 kappa) / dt, (1 - 2 kappa) / dt, kappa / dt
  df64 dx, half_dx, idt, ce;   // dx, dx / 2, 1 / dt, alpha / (4 dx)
};

__device__ __forceinline__ HeatRowsDF heat_rows_df(double alpha, const HeatArgs &a) {
  const double kap = alpha * a.kfac;
  HeatRowsDF r;
  r.c1 = df64((1.0 + 2.0 * kap) * a.idt);
  r.c2 = df64((1.0 - 2.0 * kap) * a.idt);
  r.c3 = df64(kap * a.idt);
  r.dx = a.dx_d;
  r.half_dx = a.half_dx_d;
  r.idt = a.idt_d;
  r.ce = df64(alpha * a.ce_fac);
  return r;
}

// The rows of slice k >= 1 in double-float (heat_slice_residual), lane part: the PDE rows of
// the lane's elements into the lane's running max |h| (mx), and the lane's partial sums of the
// mass and energy rows, sum u^k, sum (u^k)^2 and sum (2 dx D+ ubar)^2.  The warp sums of the
// partials are deferred to heat_rows_flush.
template <int E>
__device__ __forceinline__ void heat_slice_rows_df(const HeatRowsDF &c, const df64 (&cur)[E],
                                                   const df64 (&prev)[E], int nx, int lane,
                                                   float &mx, df64 &su, df64 &su2, df64 &sd2) {
  df64 s[E], sl[E], sr[E];
#pragma unroll
  for (int q = 0; q < E; ++q) s[q] = df_add_fast(cur[q], prev[q]);
  heat_neighbours_df<E>(s, sl, sr, nx, lane);
  su = su2 = sd2 = df64(0.0f, 0.0f);
  // every term is 0 beyond nx (u and the neighbours are), so no element guard
#pragma unroll
  for (int q = 0; q < E; ++q) {
    // ((1 + 2k) u^k - (1 - 2k) u^{k-1} - k (s_{i-1} + s_{i+1})) / dt
    const df64 t = hd_fma(-c.c2, prev[q], c.c1 * cur[q]);
    const df64 r = hd_fma(-c.c3, df_add_fast(sl[q], sr[q]), t);
    mx = hd_nan_max(mx, fabsf(r.hi));
    su = df_add_fast(su, cur[q]);
    su2 = hd_fma(cur[q], cur[q], su2);
    const df64 d = df_sub_fast(sr[q], s[q]);     // 2 dx D+ ubar
    sd2 = hd_fma(d, d, sd2);
  }
}

// Per-lane partial sums of up to 32 consecutive slices, one row per slice, padded to 33
// columns so that the transposed reads of heat_rows_flush fall in distinct banks.
struct HeatRowSums {
  df64 su[32][33], su2[32][33], sd2[32][33];
};

// The mass and energy rows of the n (<= 32) slices whose partials fill rows 0 .. n-1: lane j
// sums row j over the 32 lanes; the energy row of slice j takes E_{j-1} from lane j - 1 (lane
// 0 from e_last, the last energy of the previous group).
__device__ __forceinline__ void heat_rows_flush(const HeatRowsDF &c, const df64 &sum_g,
                                                HeatRowSums &rs, int n, df64 &e_last, float &mx,
                                                int lane) {
  __syncwarp();
  df64 su(0.0f, 0.0f), su2(0.0f, 0.0f), sd2(0.0f, 0.0f);
  const int j = lane < n ? lane : n - 1;
#pragma unroll 8
  for (int l = 0; l < 32; ++l) {
    su = df_add_fast(su, rs.su[j][l]);
    su2 = df_add_fast(su2, rs.su2[j][l]);
    sd2 = df_add_fast(sd2, rs.sd2[j][l]);
  }
  __syncwarp();
  const df64 hm = c.dx * df_sub_fast(su, sum_g);
  const df64 ek = c.half_dx * su2;
  df64 ep = hd_shfl_up(ek, 1);
  if (lane == 0) ep = e_last;
  const df64 he = hd_fma(df_sub_fast(ek, ep), c.idt, c.ce * sd2);
  if (lane < n) mx = hd_nan_max(mx, hd_nan_max(fabsf(hm.hi), fabsf(he.hi)));
  e_last = hd_shfl(ek, n - 1);
}

// df64 -> double by two conversions and one FP64 addition: three issue slots against about
// 25 integer operations for df_to_double; the FP64 pipe is otherwise idle in these chains.
__device__ __forceinline__ double hd_to_double(df64 x) { return (double)x.hi + (double)x.lo; }

// Statistics the two warps of a forward block exchange at the last barrier.
struct HeatXchg {
  double obj;
  float hmax;
  int ok;
};

// Double-buffered hand-over slots between the two warps of a block: one df64 per element of a
// slice, [parity][q][lane] (consecutive lanes, consecutive words).
template <int E>
struct HeatSlots {
  df64 u[2][E][32];   // forward chain: u^k, warp 0 -> warp 1
  df64 r[2][E][32];   // multiplier chain: dt r^k (r^0 itself), warp 1 -> warp 0
  df64 l[2][E][32];   // multiplier chain: lambda^k, warp 0 -> warp 1
};

// Forward projection of sample b in double-float, by the two warps of the block.  Warp 0 runs
// only the time chains, u^k = 2 A^-1 u^{k-1} - u^{k-1} and then the multipliers by backward
// substitution, handing each slice over through HeatSlots; warp 1 does everything off the
// chains one step behind or ahead: it converts and stores u and lambda, evaluates the rows of
// every slice (the residual statistics) and the objective, and prepares dt r^k = dt (u_hat - u)
// for the multiplier chain.  One block barrier per step; both warps run the same loops, so
// every barrier is reached by both on every path, and both return the same value: false,
// having written nothing that the FP64 path does not overwrite, when a value leaves the
// double-float range (alpha = 0 or bad alpha, an IC value up front; a residual u_hat - u).
template <int E>
__device__ __forceinline__ bool heat_forward_df(const HeatArgs &a, int b, int lane, int w,
                                                HeatRowSums &rs, HeatSlots<E> &sl,
                                                HeatXchg &xc) {
  const int nx = a.nx, nt = a.nt;
  const double *pg = a.params + (size_t)b * (nx + 1);
  const double alpha = pg[nx];
  // alpha = 0 takes the FP64 path: there u^k = g exactly, which a 48-bit significand does not
  // reproduce for every double g
  if (!(alpha > 0.0) || !(alpha <= 1e30)) return false;
  [[maybe_unused]] const long long nvar = (long long)a.B * nx * nt;
  double g[E];
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int i = lane * E + q;
    g[q] = (i < nx && snap_in_bounds(SNAP_SITE_HEAT_G, (long long)b * (nx + 1) + i,
                                     (long long)a.B * (nx + 1))) ? pg[i] : 0.0;
  }
  const df64 zero(0.0f, 0.0f);
  df64 cur[E];
  bool ok = true;
#pragma unroll
  for (int q = 0; q < E; ++q)
    ok &= df_split_trunc(g[q], cur[q].hi, cur[q].lo) && fabs(g[q]) <= 0x1p60;
  if (!__all_sync(kAll, ok)) return false;    // the same data, so the same decision, in both warps
  double *ub = a.u_out + (size_t)b * nx * nt;
  const double *uhb = a.uh + (size_t)b * nx * nt;
  double *lb = a.lam + (size_t)b * a.n_rows;
  const HeatRowsDF c = heat_rows_df(alpha, a);
  const df64 dt_d = a.dt_d;
  HeatFactorDF<E> f;
  if (w == 0) heat_factor_df<E>(f, alpha, a.dx, a.dt, nx, lane);
  // warp 1: row statistics and objective
  df64 sum_g = zero, e_last = zero, prev[E];
  float hmax = 0.0f;                  // IC rows and the mass row of slice 0 hold exactly
  double obj = 0.0;
  bool in_range = true;
  int nrow = 0;
  double xh[E];                       // u_hat of the next slice to take, loaded one step ahead
  if (w == 1) {
    df64 sg = zero, sq = zero;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = lane * E + q;
      sg = df_add_fast(sg, cur[q]);
      sq = hd_fma(cur[q], cur[q], sq);
      prev[q] = cur[q];
      if (i < nx) {
        if (snap_in_bounds(SNAP_SITE_HEAT_U, (long long)b * nx * nt + i, nvar)) ub[i] = g[q];
        const double r0 = uhb[i] - g[q];
        obj = fma(r0, r0, obj);
      }
      xh[q] = (i < nx && nt > 1) ? uhb[(size_t)nx + i] : 0.0;
    }
    sum_g = hd_warp_sum(sg);
    e_last = c.half_dx * hd_warp_sum(sq);   // energy of slice 0
  }
  // warp 1 takes slice k (1 <= k < nt) from its slot: stores u^k, adds its objective term (from
  // the stored double) and its rows (with u^{k-1} = prev)
  auto take = [&](int k) {
    df64 v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = sl.u[k & 1][q][lane];
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = lane * E + q;
      const double ud = hd_to_double(v[q]);
      if (i < nx && snap_in_bounds(SNAP_SITE_HEAT_U, (long long)b * nx * nt + (long long)k * nx + i, nvar))
        ub[(size_t)k * nx + i] = ud;
      const double rd = xh[q] - ud;                   // 0 beyond nx
      obj = fma(rd, rd, obj);
      xh[q] = (i < nx && k + 1 < nt) ? uhb[(size_t)(k + 1) * nx + i] : 0.0;
    }
    df64 su, su2, sd2;
    heat_slice_rows_df<E>(c, v, prev, nx, lane, hmax, su, su2, sd2);
    rs.su[nrow][lane] = su;
    rs.su2[nrow][lane] = su2;
    rs.sd2[nrow][lane] = sd2;
    if (++nrow == 32) {
      heat_rows_flush(c, sum_g, rs, 32, e_last, hmax, lane);
      nrow = 0;
    }
#pragma unroll
    for (int q = 0; q < E; ++q) prev[q] = v[q];
  };
  // the forward chain: iteration k computes u^k (warp 0) and takes slice k - 1 (warp 1)
  for (int k = 1; k < nt; ++k) {
    if (w == 0) {
      df64 z[E];
#pragma unroll
      for (int q = 0; q < E; ++q) z[q] = cur[q];
      heat_solve_df<E>(f, z, nx, lane);
#pragma unroll
      for (int q = 0; q < E; ++q) {
        cur[q] = df_add_fast(df_scale2(z[q], 2.0f), -cur[q]);   // 0 beyond nx
        sl.u[k & 1][q][lane] = cur[q];
      }
    } else if (k >= 2) {
      take(k - 1);
    }
    __syncthreads();
  }
  // warp 1 prepares dt r^k = dt (u_hat^k - u^k) (r^0 unscaled) into slot r[k & 1] and loads
  // slice k - 1 for the next call
  double ph[E], pu[E];
  auto prep = [&](int k) {
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = lane * E + q;
      df64 v;
      in_range &= df_split_trunc(ph[q] - pu[q], v.hi, v.lo);   // 0 beyond nx
      const df64 sv = dt_d * v;
      sl.r[k & 1][q][lane] = (k > 0) ? sv : v;
      ph[q] = (i < nx && k >= 1) ? uhb[(size_t)(k - 1) * nx + i] : 0.0;
      pu[q] = (i < nx && k >= 1) ? ub[(size_t)(k - 1) * nx + i] : 0.0;
    }
  };
  if (w == 1) {
    if (nt >= 2) take(nt - 1);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = lane * E + q;
      ph[q] = (i < nx) ? uhb[(size_t)(nt - 1) * nx + i] : 0.0;
      pu[q] = (i < nx) ? ub[(size_t)(nt - 1) * nx + i] : 0.0;
    }
    prep(nt - 1);
  }
  __syncthreads();
  // the multiplier chain: iteration k computes lambda^k (warp 0); warp 1 prepares dt r^{k-1}
  // and stores lambda^{k+1}
  df64 lam1[E];
#pragma unroll
  for (int q = 0; q < E; ++q) lam1[q] = zero;
  for (int k = nt - 1; k >= 1; --k) {
    if (w == 0) {
      df64 y[E];
#pragma unroll
      for (int q = 0; q < E; ++q) y[q] = df_add_fast(sl.r[k & 1][q][lane], df_scale2(lam1[q], 2.0f));
      heat_solve_df<E>(f, y, nx, lane);
#pragma unroll
      for (int q = 0; q < E; ++q) {
        lam1[q] = df_sub_fast(y[q], lam1[q]);         // lambda^k, 0 beyond nx
        sl.l[k & 1][q][lane] = lam1[q];
      }
    } else {
      prep(k - 1);
      if (k + 1 < nt) {
#pragma unroll
        for (int q = 0; q < E; ++q) {
          const int i = lane * E + q;
          const double v = hd_to_double(sl.l[(k + 1) & 1][q][lane]);
          if (i < nx && snap_in_bounds(SNAP_SITE_HEAT_LAM, a.off_pde + (long long)k * nx + i, a.n_rows))
            lb[a.off_pde + (size_t)k * nx + i] = v;
        }
      }
    }
    __syncthreads();
  }
  if (w == 0) {
    // IC multipliers: r^0 + (2 lambda^1 - A lambda^1) / dt = r^0 + c2 lambda^1 + c3 (l + r)
    df64 ll[E], lr[E];
    heat_neighbours_df<E>(lam1, ll, lr, nx, lane);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = lane * E + q;
      const df64 r0 = sl.r[0][q][lane];
      if (i < nx)
        lb[i] = hd_to_double(hd_fma(c.c3, df_add_fast(ll[q], lr[q]), hd_fma(c.c2, lam1[q], r0)));
    }
  } else {
    if (nt >= 2) {
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const int i = lane * E + q;
        const double v = hd_to_double(sl.l[1][q][lane]);           // lambda^1
        if (i < nx && snap_in_bounds(SNAP_SITE_HEAT_LAM, a.off_pde + i, a.n_rows))
          lb[a.off_pde + i] = v;
      }
    }
    for (int k = lane; k < nt; k += 32) lb[a.off_mass + k] = 0.0;
    for (int k = lane; k < nt - 1; k += 32) lb[a.off_energy + k] = 0.0;
    if (nrow > 0) heat_rows_flush(c, sum_g, rs, nrow, e_last, hmax, lane);
    hmax = hd_warp_max(hmax);
    obj = h_warp_sum(obj);
    in_range = __all_sync(kAll, in_range);
    if (lane == 0) {
      xc.hmax = hmax;
      xc.obj = obj;
      xc.ok = in_range;
    }
  }
  __syncthreads();                    // multipliers and statistics done
  if (!xc.ok) return false;
  if (w == 0 && lane == 0 && a.stats) {
    const double hmaxd = (double)xc.hmax;
    const double objd = 0.5 * xc.obj;
    snap_stats st;
    st.iters = 1;
    st.backtracks = 0;
    st.corrections = 0;
    st.h_inf = hmaxd;
    st.kkt_inf = hmaxd;   // active rows (IC exact, PDE rows) at the returned u
    st.obj = objd;
    if (!(hmaxd == hmaxd) || isinf(hmaxd) || !(objd == objd) || isinf(objd)) st.status = SNAP_SAMPLE_NONFINITE;
    else if (!(hmaxd <= a.tol_h)) st.status = SNAP_SAMPLE_RESIDUAL;
    else st.status = SNAP_SAMPLE_OK;
    a.stats[b] = st;
  }
  return true;
}

// Hand-over slots of the adjoint block: dt gbar^k (warp 1 -> warp 0) and b^k (warp 0 -> warp 1).
template <int E>
struct HeatAdjSlots {
  df64 y[2][E][32];
  df64 b[2][E][32];
  df64 dalpha;
  int ok0, ok1;
};

// Adjoint of sample b in double-float (heat_backward_fp64's recurrences), by the two warps of
// the block.  Warp 0 runs only the chain b^k = A^-1 (dt gbar^k + 2 b^{k+1}) - b^{k+1}; warp 1
// prepares dt gbar^k one step ahead and adds the dalpha term b^{k+1} . 1/2 D2 (u^{k+1} + u^k)
// one step behind, through HeatAdjSlots, one block barrier per step.  Both warps run the same
// loops and return the same value: false, having written nothing, when a value leaves the
// double-float range (bad samples and alpha included); the outputs are written after the last
// barrier.
template <int E>
__device__ __forceinline__ bool heat_backward_df(const HeatArgs &a, int b, int lane, int w,
                                                 HeatAdjSlots<E> &sl) {
  const int nx = a.nx, nt = a.nt;
  const double *pg = a.params + (size_t)b * (nx + 1);
  const double alpha = pg[nx];
  if ((a.fwd_stats && a.fwd_stats[b].status != SNAP_SAMPLE_OK) || !(alpha >= 0.0) ||
      !(alpha <= 1e30))
    return false;
  const double *gb = a.uh + (size_t)b * nx * nt;       // dL/du
  const double *ub = a.u + (size_t)b * nx * nt;
  double *gh = a.grad_uh + (size_t)b * nx * nt;
  double *gp = a.grad_params ? a.grad_params + (size_t)b * (nx + 1) : nullptr;
  const df64 zero(0.0f, 0.0f);
  const HeatRowsDF c = heat_rows_df(alpha, a);
  const df64 dt_d = a.dt_d;
  const df64 cd2 = a.cd2_d;
  HeatFactorDF<E> f;
  if (w == 0) heat_factor_df<E>(f, alpha, a.dx, a.dt, nx, lane);
  // warp 1 state: dt gbar of the next step and u^{k+1}, u^k, u^{k-1} around the pending term
  bool ok = true;
  df64 dalpha = zero, ua[E], uc[E];
  double xg[E], xu[E];
  auto term = [&](const df64 (&bk)[E], const df64 (&s)[E]) {   // dalpha += b . cd2 D2 s
    df64 sl_[E], sr_[E];
    heat_neighbours_df<E>(s, sl_, sr_, nx, lane);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      // 0 beyond nx (b, s and the neighbours are)
      const df64 d2 = df_sub_fast(df_add_fast(sl_[q], sr_[q]), df_scale2(s[q], 2.0f));
      dalpha = hd_fma(bk[q], cd2 * d2, dalpha);
    }
  };
  if (w == 1) {
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = lane * E + q;
      df64 v;
      ok &= df_split_trunc((i < nx && nt > 1) ? gb[(size_t)(nt - 1) * nx + i] : 0.0, v.hi, v.lo);
      sl.y[(nt - 1) & 1][q][lane] = dt_d * v;
      ok &= df_split_trunc((i < nx) ? ub[(size_t)(nt - 1) * nx + i] : 0.0, uc[q].hi, uc[q].lo);
      ua[q] = zero;
      xg[q] = (i < nx && nt > 2) ? gb[(size_t)(nt - 2) * nx + i] : 0.0;
      xu[q] = (i < nx && nt > 1) ? ub[(size_t)(nt - 2) * nx + i] : 0.0;
    }
  }
  __syncthreads();
  df64 b1[E];
#pragma unroll
  for (int q = 0; q < E; ++q) b1[q] = zero;
  for (int k = nt - 1; k >= 1; --k) {
    if (w == 0) {
      df64 y[E];
#pragma unroll
      for (int q = 0; q < E; ++q) y[q] = df_add_fast(sl.y[k & 1][q][lane], df_scale2(b1[q], 2.0f));
      heat_solve_df<E>(f, y, nx, lane);
#pragma unroll
      for (int q = 0; q < E; ++q) {
        b1[q] = df_sub_fast(y[q], b1[q]);             // b^k, 0 beyond nx
        sl.b[k & 1][q][lane] = b1[q];
      }
    } else {
      // ua = u^{k+1}, uc = u^k; xg = gbar^{k-1}, xu = u^{k-1} (loaded one step ahead)
      if (k + 1 < nt) {
        df64 bk[E], s[E];
#pragma unroll
        for (int q = 0; q < E; ++q) {
          bk[q] = sl.b[(k + 1) & 1][q][lane];
          s[q] = df_add_fast(ua[q], uc[q]);
        }
        term(bk, s);                                   // step k + 1
      }
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const int i = lane * E + q;
        df64 v;
        ok &= df_split_trunc(xg[q], v.hi, v.lo);
        sl.y[(k - 1) & 1][q][lane] = dt_d * v;         // dt gbar^{k-1} (unused for k = 1)
        ua[q] = uc[q];
        ok &= df_split_trunc(xu[q], uc[q].hi, uc[q].lo);
        xg[q] = (i < nx && k >= 3) ? gb[(size_t)(k - 2) * nx + i] : 0.0;
        xu[q] = (i < nx && k >= 2) ? ub[(size_t)(k - 2) * nx + i] : 0.0;
      }
    }
    __syncthreads();
  }
  // IC gradient (warp 0): gbar^0 + (2 b^1 - A b^1) / dt = gbar^0 + c2 b^1 + c3 (l + r)
  double gpv[E];
  if (w == 0) {
    df64 ll[E], lr[E];
    heat_neighbours_df<E>(b1, ll, lr, nx, lane);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = lane * E + q;
      df64 v0;
      ok &= df_split_trunc((i < nx) ? gb[i] : 0.0, v0.hi, v0.lo);
      gpv[q] = hd_to_double(hd_fma(c.c3, df_add_fast(ll[q], lr[q]), hd_fma(c.c2, b1[q], v0)));
    }
    ok = __all_sync(kAll, ok);
    if (lane == 0) sl.ok0 = ok;
  } else {
    if (nt >= 2) {
      df64 bk[E], s[E];
#pragma unroll
      for (int q = 0; q < E; ++q) {
        bk[q] = sl.b[1][q][lane];                      // b^1
        s[q] = df_add_fast(ua[q], uc[q]);              // u^1 + u^0
      }
      term(bk, s);                                     // step 1
    }
    dalpha = hd_warp_sum(dalpha);
    ok = __all_sync(kAll, ok);
    if (lane == 0) {
      sl.ok1 = ok;
      sl.dalpha = dalpha;
    }
  }
  __syncthreads();
  if (!(sl.ok0 && sl.ok1)) return false;               // the same verdict in both warps
  for (size_t i = threadIdx.x; i < (size_t)nx * nt; i += 64) gh[i] = 0.0;
  if (gp && w == 0) {
#pragma unroll
    for (int q = 0; q < E; ++q)
      if (lane * E + q < nx) gp[lane * E + q] = gpv[q];
    if (lane == 0) gp[nx] = hd_to_double(sl.dalpha);
  }
  return true;
}

// Forward projection of sample b in FP64: u (time chain), lambda (backward substitution),
// statistics.  The path of a sample whose values leave the double-float range.
template <int E>
__device__ __noinline__ void heat_forward_fp64(const HeatArgs &a, int b, int lane) {
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

// Adjoint of sample b in FP64: J^T b = gbar by the same backward substitution;
// dL/du_hat = 0, dL/dg = b_IC, dL/dalpha = sum_k b^k . 1/2 D2 (u^k + u^{k-1}).  The path of a
// sample whose values leave the double-float range.
template <int E>
__device__ __noinline__ void heat_backward_fp64(const HeatArgs &a, int b, int lane) {
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

// One sample per block of two warps (the samples spread over every SM): the double-float
// chains, or the FP64 chain in warp 0 for a sample whose values leave the double-float range
// (and for E > 8, where the double-float arrays would spill).
template <int E>
__global__ void __launch_bounds__(64) k_heat_forward(HeatArgs a) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = blockIdx.x;
  if (b >= a.B) return;
  if constexpr (E <= 8) {
    __shared__ HeatRowSums rs;
    __shared__ HeatSlots<E> sl;
    __shared__ HeatXchg xc;
    if (heat_forward_df<E>(a, b, lane, w, rs, sl, xc)) return;
  }
  if (w == 0) heat_forward_fp64<E>(a, b, lane);
}

template <int E>
__global__ void __launch_bounds__(64) k_heat_backward(HeatArgs a) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = blockIdx.x;
  if (b >= a.B) return;
  if constexpr (E <= 8) {
    __shared__ HeatAdjSlots<E> sl;
    if (heat_backward_df<E>(a, b, lane, w, sl)) return;
  }
  if (w == 0) heat_backward_fp64<E>(a, b, lane);
}

template <int E>
void heat_launch(int kind, const HeatArgs &a, cudaStream_t s) {
  const unsigned blocks = (unsigned)(((long long)a.B * 32 + 127) / 128);
  if (kind == 0) k_heat_forward<E><<<(unsigned)a.B, 64, 0, s>>>(a);
  else if (kind == 1) k_heat_residual<E><<<blocks, 128, 0, s>>>(a);
  else k_heat_backward<E><<<(unsigned)a.B, 64, 0, s>>>(a);
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
  a.kfac = a.dt / (2.0 * a.dx * a.dx);
  a.idt = 1.0 / a.dt;
  a.ce_fac = 1.0 / (4.0 * a.dx);
  a.dx_d = df64(a.dx);
  a.half_dx_d = df64(0.5 * a.dx);
  a.idt_d = df64(a.idt);
  a.dt_d = df64(a.dt);
  a.cd2_d = df64(0.5 / (a.dx * a.dx));
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
