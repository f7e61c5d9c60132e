// Per-sample pieces of the 1-D families A/B forward projection, executed by one full warp:
//   s1_derive     A1 parameter derivation: M = dx sum g, E0 = dx sum g^2, q = exp(-r dt), their
//                 float-pair images and the residual of the t = 0 rows that the IC rows imply
//                 (left out of the solve, as in the worked example of Appendix C);
//   s1_ic_forward the IC block (slice k = 0): the rows u_i - g_i are linear and independent per
//                 variable, so one Newton step from (u_hat, 0) lands on u = g,
//                 lambda = u_hat - g (Appendix B);
//   s1_finalize   the per-sample reduction of the per-slice statistics (fixed order, so the
//                 result does not depend on which warp runs it).
// Shared by the per-problem kernels (kern_1d.cu) and the uneven-batch kernel (kern_batch.cu),
// so that both produce the same bits.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "df64.cuh"
#include "snap_internal.h"

namespace {

__device__ __forceinline__ double s1_nan_max(double a, double b) {
  return (a < b || b != b) ? b : a;
}

__device__ __forceinline__ double s1_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double s1_warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = s1_nan_max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Derived parameters of the sample with parameters pg (every lane returns the same value:
// the butterfly sums are symmetric).
__device__ __forceinline__ SampleDerived s1_derive(const Geom1D &g, const double *__restrict__ pg,
                                                   int lane) {
  double s1 = 0.0, s2 = 0.0;
  for (int i = lane; i < g.nx; i += 32) {
    const double v = pg[i];
    s1 += v;
    s2 = fma(v, v, s2);
  }
  s1 = s1_warp_sum(s1);
  s2 = s1_warp_sum(s2);
  SampleDerived d;
  d.M = g.dx * s1;
  d.E0 = g.dx * s2;
  d.q = exp(-pg[g.p_rate] / (double)(g.nt - 1));
  const double fl = d.M * d.M + g.energy_floor;
  d.Mh = __double2float_rn(d.M);   d.Ml = __double2float_rn(d.M - (double)d.Mh);
  d.E0h = __double2float_rn(d.E0); d.E0l = __double2float_rn(d.E0 - (double)d.E0h);
  d.qh = __double2float_rn(d.q);   d.ql = __double2float_rn(d.q - (double)d.qh);
  d.fh = __double2float_rn(fl);    d.fl = __double2float_rn(fl - (double)d.fh);
  // rows at t = 0 evaluated at u_0 = g
  double hinf = 0.0;
  if (g.rows & SL_MASS) hinf = s1_nan_max(hinf, fabs(g.dx * s1 - d.M));
  if (g.rows & SL_ENERGY) {
    const double e0 = d.E0 >= d.M * d.M + g.energy_floor ? d.E0 : d.M * d.M + g.energy_floor;
    hinf = s1_nan_max(hinf, fabs(g.dx * s2 - e0));
  }
  if (g.rows & SL_BOUND) {
    const double g0 = pg[0], gh = pg[g.ih];
    hinf = s1_nan_max(hinf, fabs(g0 * g0 + gh * gh - pg[g.p_c]));
  }
  d.h0_inf = hinf;
  return d;
}

// IC block of one sample with start u0 = u_hat: row = u_hat of slice 0, out = u of slice 0,
// lb = the sample's multipliers, *st0 = statistics of slice 0 (lane 0 writes).
__device__ __forceinline__ void s1_ic_forward(const Geom1D &g, const double *__restrict__ pg,
                                              const double *__restrict__ row,
                                              double *__restrict__ out, double *__restrict__ lb,
                                              BlockStat *__restrict__ st0, double h0_inf,
                                              double tol_kkt, int lane) {
  double mx = 0.0, sq = 0.0;
  for (int i = lane; i < g.nx; i += 32) {
    const double dv = row[i] - pg[i];
    sq = fma(dv, dv, sq);
    mx = s1_nan_max(mx, fabs(dv));
  }
  mx = s1_warp_max(mx);
  sq = s1_warp_sum(sq);
  const bool take = !(mx <= tol_kkt);
  for (int i = lane; i < g.nx; i += 32) {
    out[i] = take ? pg[i] : row[i];
    lb[i] = take ? row[i] - pg[i] : 0.0;
  }
  if (lane == 0) {
    if (g.off_mass >= 0) lb[g.off_mass] = 0.0;
    if (g.off_energy >= 0) lb[g.off_energy] = 0.0;
    if (g.off_bound >= 0) lb[g.off_bound] = 0.0;
    BlockStat st;
    st.iters = take ? 1 : 0;
    st.backtracks = 0;
    st.corrections = 0;
    st.status = (mx == mx && !isinf(mx)) ? SNAP_SAMPLE_OK : SNAP_SAMPLE_NONFINITE;
    st.kkt_inf = take ? 0.0 : mx;
    st.h_inf = s1_nan_max(take ? 0.0 : mx, h0_inf);
    st.obj = take ? 0.5 * sq : 0.0;
    *st0 = st;
  }
}

// Per-sample statistics from the nblk block statistics bs[0..nblk) (lane 0 writes *out).
// kCoherent: read through L2 only (blocks written by other warps of a running kernel).
template <bool kCoherent>
__device__ __forceinline__ void s1_finalize(const BlockStat *__restrict__ bs, int nblk,
                                            double tol_h, snap_stats *__restrict__ out,
                                            int lane) {
  int iters = 0, bt = 0, corr = 0, rank = 0, status = SNAP_SAMPLE_OK;
  double hinf = 0.0, kinf = 0.0, obj = 0.0;
  for (int k = lane; k < nblk; k += 32) {
    BlockStat q;
    if (kCoherent) {
      // 40-byte records: 8-byte aligned
      const int2 a = __ldcg(reinterpret_cast<const int2 *>(bs + k));
      const int2 b = __ldcg(reinterpret_cast<const int2 *>(bs + k) + 1);
      q.iters = a.x; q.backtracks = a.y; q.status = b.x; q.corrections = b.y;
      const double *d = reinterpret_cast<const double *>(bs + k) + 2;
      q.h_inf = __ldcg(d);
      q.kkt_inf = __ldcg(d + 1);
      q.obj = __ldcg(d + 2);
    } else {
      q = bs[k];
    }
    iters = max(iters, q.iters);
    bt += q.backtracks;
    corr += q.corrections;
    const int rk = snap_status_rank(q.status);
    if (rk > rank) { rank = rk; status = q.status; }
    hinf = s1_nan_max(hinf, q.h_inf);
    kinf = s1_nan_max(kinf, q.kkt_inf);
    obj += q.obj;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    iters = max(iters, __shfl_xor_sync(0xffffffffu, iters, o));
    bt += __shfl_xor_sync(0xffffffffu, bt, o);
    corr += __shfl_xor_sync(0xffffffffu, corr, o);
    const int r2 = __shfl_xor_sync(0xffffffffu, rank, o);
    const int s2 = __shfl_xor_sync(0xffffffffu, status, o);
    if (r2 > rank || (r2 == rank && s2 < status)) { rank = r2; status = s2; }
  }
  hinf = s1_warp_max(hinf);
  kinf = s1_warp_max(kinf);
  obj = s1_warp_sum(obj);
  if (lane == 0) {
    snap_stats st;
    st.iters = iters;
    st.backtracks = bt;
    st.corrections = corr;
    st.status = status;
    if (status == SNAP_SAMPLE_OK && !(hinf <= tol_h)) st.status = SNAP_SAMPLE_RESIDUAL;
    st.h_inf = hinf;
    st.kkt_inf = kinf;
    st.obj = obj;
    *out = st;
  }
}

// dL/dparams of one sample (one warp; fixed order, so the bits do not depend on which warp
// runs it) from the per-slice contributions c[1..nt) of its adjoint: the IC block passes
// dL/du of slice 0 (g0) to dL/dg, the mass / energy rows add dx b_m, 2 dx g b_e (exponential
// branch) and 2 M dx b_fl (floor branch) to every g_i, and the rate receives sum b_r.  M is the
// sample's dx sum g.  kCoherent reads the contributions through L2 only (written by other
// warps of a running kernel).
template <bool kCoherent>
__device__ __forceinline__ void s1_param_grad(const Geom1D &g, const double *__restrict__ g0,
                                              const double *__restrict__ pg, double M,
                                              const BwdContrib *__restrict__ c, bool bad,
                                              double *__restrict__ out, int lane) {
  double sm = 0.0, sex = 0.0, sfl = 0.0, sr = 0.0;
  for (int k = 1 + lane; k < g.nt; k += 32) {
    if (kCoherent) {
      const double2 a = __ldcg(reinterpret_cast<const double2 *>(c + k));
      const double2 b = __ldcg(reinterpret_cast<const double2 *>(c + k) + 1);
      sm += a.x; sex += a.y; sfl += b.x; sr += b.y;
    } else {
      const BwdContrib q = c[k];
      sm += q.bm; sex += q.bex; sfl += q.bfl; sr += q.br;
    }
  }
  sm = s1_warp_sum(sm);
  sex = s1_warp_sum(sex);
  sfl = s1_warp_sum(sfl);
  sr = s1_warp_sum(sr);
  for (int i = lane; i < g.nx; i += 32) {
    const double v = g0[i] + g.dx * sm + 2.0 * g.dx * pg[i] * sex + 2.0 * M * g.dx * sfl;
    out[i] = bad ? NAN : v;
  }
  if (lane == 0) out[g.p_rate] = bad ? NAN : sr;
}

// sum_i row[i] of a slice over its four lanes (four lanes per slice, eight slices per warp) (lane r takes i = r, r + 4, ...), on the FP32
// and integer pipes: every value split into a float pair by integer operations (df_split_trunc,
// |x - hi - lo| < 2^-46 |x|), the pairs summed by TwoSum with the errors carried, the four lane
// sums combined in double-float.  A slice with a value outside the split range (|x| outside
// [2^-74, 2^57] and not zero, or non-finite) is summed in FP64 instead; the four lanes of a
// slice agree on the path.  The FP64 pipe (2 lanes per clock per SM on B300) otherwise spends
// one addition per element here.
__device__ __forceinline__ double s4_slice_sum(const double *row, int nx, int r, bool live) {
  float sh = 0.0f, se = 0.0f;
  int ok = 1;
  if (live) {
#pragma unroll 8
    for (int i = r; i < nx; i += 4) {
      float h, l;
      ok &= df_split_trunc(row[i], h, l);
      const float t = sh + h, bb = t - sh;
      se += ((sh - (t - bb)) + (h - bb)) + l;
      sh = t;
    }
  }
  ok &= __shfl_xor_sync(0xffffffffu, ok, 1);
  ok &= __shfl_xor_sync(0xffffffffu, ok, 2);
  df64 v = df_fast_two_sum(sh, se);
  v = v + df64(__shfl_xor_sync(0xffffffffu, v.hi, 1), __shfl_xor_sync(0xffffffffu, v.lo, 1));
  v = v + df64(__shfl_xor_sync(0xffffffffu, v.hi, 2), __shfl_xor_sync(0xffffffffu, v.lo, 2));
  double S = (double)v.hi + (double)v.lo;
  if (__any_sync(0xffffffffu, !ok)) {         // rare, warp-uniform: the FP64 sums of the warp's slices
    double T = 0.0;
    if (live)
      for (int i = r; i < nx; i += 4) T += row[i];
    T += __shfl_xor_sync(0xffffffffu, T, 1);
    T += __shfl_xor_sync(0xffffffffu, T, 2);
    if (!ok) S = T;
  }
  return S;
}

}  // namespace
