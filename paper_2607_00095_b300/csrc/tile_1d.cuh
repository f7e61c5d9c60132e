// The warp tile of the 1-D mixed-pipe moment path (families A/B, start u0 = u_hat): one warp
// projects up to 32 consecutive slices [sbase, send) of a virtual batch whose slices are
// located by the address policy Addr.  The tile of the per-problem kernel k1d_mixed
// (kern_1d_mixed.cu: rows of one batch, 4 lanes per slice, 16 loads in flight) and of the
// uneven-batch kernel (kern_batch.cu: one pointer set per instance, lanes per slice per group).
//
//   phase 1  (LPS = 2, 4 or 8 lanes per slice, 32 / LPS slices per warp instruction, 16-byte
//            loads): every u_hat_i is split into a float pair hi + lo with integer operations
//            only (|u_hat - hi - lo| < 2^-46 |u_hat|), and the interior moments
//            S1 = sum u_hat_i, S2 = sum u_hat_i^2 are accumulated in double-float
//            (error-free TwoSum / TwoProd), reduced across the LPS lanes by butterfly steps;
//   phase 2  (one slice per lane): the slice's Newton-KKT iteration in moment form,
//            first in float, then in double-float to the FP64 stopping tolerance
//            (slice_solve_mixed); E_k = E0 q^k with q = exp(-r dt) by binary powering in
//            double-float;
//   phase 3  (LPS lanes per slice): u = fma(a, u_hat, c) in FP64, 16-byte stores.
//
// Slice k = 0 (the IC block) is skipped: the caller solves it (s1_ic_forward).  A slice whose
// values leave the range of the float-pair representation (|u_hat| outside [2^-74, 2^57], exactly
// zero, or non-finite) falls back to FP64 moments and the FP64 iteration.
//
// u_hat and the parameters are read through the read-only path (__ldg): the kernel never
// writes them.
//
// Address policy Addr (all device, inlined):
//   row_in(s) / row_out(s)  u_hat / u of slice s;  slice_k(s)  its time index;
//   par(s) / lam_of(s)      the parameters / multipliers of its sample;
//   derived(s)              the sample's SampleDerived;  stat(s)  its BlockStat slot;
//   prefetch(s0, s1, lane)  L2 prefetch of the tile's u_hat;
//   before_solve(s0, s1, lane)  hook run by the whole warp between phases 1 and 2;
//   row_ok(site, s, i) / slice_ok(s)  the bounds-checked build's checks of the accesses to
//                                      elements i, i + 1 of slice s / of slice s (true otherwise).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "slice_newton.cuh"
#include "snap_bounds.cuh"
#include "snap_internal.h"

namespace {

enum { T1_KIND_MOMENT = 0, T1_KIND_NONE = 3 };

__device__ __forceinline__ double t1_nan_max(double a, double b) { return (a < b || b != b) ? b : a; }

// x^k for k >= 0 by binary powering in double-float
__device__ __forceinline__ df64 t1_df_pow(df64 x, int k) {
  df64 r(1.0f, 0.0f);
  while (k > 0) {
    if (k & 1) r = r * x;
    x = x * x;
    k >>= 1;
  }
  return r;
}

__device__ __forceinline__ df64 t1_shfl_df(df64 v, int off) {
  return df64(__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off));
}

// Phase 2 for one slice k >= 1 (one lane): the slice's Newton-KKT iteration from its interior
// moments (m1, m2: S1, S2 in double-float; mmx, mmn: interior extremes; mok: every value in
// the float-pair range), u_hat at i = 0 and i = nx/2 (uh0, uhh) and the sample's derived
// values; writes the slice's multipliers into lb and its statistics into *stat.  Returns u = A u_hat + Cc on the interior, P0 / PH at i = 0 /
// nx/2.  row (u_hat of the slice, any address space) is read only by the FP64 fallback.
__device__ __forceinline__ void t1_solve_slice(
    const Geom1D &g, int k, const df64 &m1, const df64 &m2, float mmx, float mmn, int mok,
    double uh0, double uhh, const double *row, const double *__restrict__ pg,
    const SampleDerived &dv, double *__restrict__ lb, BlockStat *__restrict__ stat,
    const SolverOpts &o, const SliceOptsT<float> &so_f,
    const SliceOptsT<df64> &so_d, const df64 &dxd, double &A, double &Cc, double &P0,
    double &PH) {
  const int nx = g.nx, ih = g.ih;
  BlockStat st;
  const double C = (g.rows & SL_BOUND) ? __ldg(pg + g.p_c + k) : 0.0;
  double hm, he, hb, res, S1d, S2d;
  SliceResult R;
  double lmd, led, lbd;
  float u0h, u0l, uhh_h, uhh_l, ch, cl;
  const bool range_ok = mok && df_split(uh0, u0h, u0l) && df_split(uhh, uhh_h, uhh_l) &&
                        df_split(C, ch, cl);
  if (range_ok) {
    SliceIn<df64> d;
    d.S1 = m1; d.S2 = m2;
    d.mx = df64(mmx, 0.0f); d.mn = df64(mmn, 0.0f);
    d.uh0 = df64(u0h, u0l); d.uhh = df64(uhh_h, uhh_l);
    d.n = df64((float)(nx - 2), 0.0f);
    d.nint = nx - 2;
    d.dx = dxd;
    d.M = df64(dv.Mh, dv.Ml);
    df64 E(0.0f, 0.0f);
    if (g.rows & SL_ENERGY) {
      const df64 e = df64(dv.E0h, dv.E0l) * t1_df_pow(df64(dv.qh, dv.ql), k);
      const df64 fl = df64(dv.fh, dv.fl);
      E = (e >= fl) ? e : fl;
    }
    d.E = E;
    d.C = df64(ch, cl);
    d.rows = g.rows;
    const df64 zero(0.0f, 0.0f);
    const bool infeasible = ((g.rows & SL_BOUND) && ch < 0.0f) ||
                            ((g.rows & SL_ENERGY) && E < ((g.rows & SL_MASS) ? d.M * d.M : zero));
    SliceZ<df64> z{df64(1.0f, 0.0f), zero, d.uh0, d.uhh, zero, zero, zero};
    SliceEval<df64> e;
    if (infeasible) {
      slice_eval(d, z, e);
      R = SliceResult{0, 0, SNAP_SAMPLE_INFEASIBLE_PARAMS, 0};
    } else {
      R = slice_solve_mixed(d, z, e, o, so_f, so_d);
    }
    A = (double)z.a; Cc = (double)z.c; P0 = (double)z.p0; PH = (double)z.ph;
    lmd = (double)z.lm; led = (double)z.le; lbd = (double)z.lb;
    // statistics in double-float, one conversion each
    const df64 hmx = sl_max(sl_max(sl_abs(e.hm), sl_abs(e.he)), sl_abs(e.hb));
    const df64 am1 = z.a - df64(1.0f, 0.0f);
    const df64 d0 = z.p0 - d.uh0, dh = z.ph - d.uhh;
    const df64 obj = (am1 * am1 * d.S2 + df64(2.0f, 0.0f) * am1 * z.c * d.S1 + z.c * z.c * d.n +
                      d0 * d0 + dh * dh) * df64(0.5f, 0.0f);
    st.iters = R.iters;
    st.backtracks = R.backtracks;
    st.status = R.status;
    st.corrections = R.corrections;
    st.kkt_inf = (double)e.res;
    st.h_inf = (double)hmx;
    st.obj = (double)obj;
    if (e.res != e.res) st.kkt_inf = NAN;
    if (hmx != hmx) st.h_inf = NAN;
  } else {
    // FP64 fallback: moments in FP64 by this lane, FP64 iteration
    double a1 = 0.0, a2 = 0.0, mx = -INFINITY, mn = INFINITY;
    for (int i = 0; i < nx; ++i) {
      if (i == 0 || i == ih) continue;
      const double v = row[i];
      a1 += v;
      a2 = fma(v, v, a2);
      mx = fmax(mx, v);
      mn = fmin(mn, v);
      if (v != v) mx = v;
    }
    SliceIn<double> d;
    d.S1 = a1; d.S2 = a2; d.mx = mx; d.mn = mn;
    d.uh0 = uh0; d.uhh = uhh;
    d.n = (double)(nx - 2);
    d.nint = nx - 2;
    d.dx = g.dx;
    d.M = dv.M;
    double E = 0.0;
    if (g.rows & SL_ENERGY) {
      const double e = dv.E0 * exp(-__ldg(pg + g.p_rate) * ((double)k / (double)(g.nt - 1)));
      const double fl = dv.M * dv.M + g.energy_floor;
      E = e >= fl ? e : fl;
    }
    d.E = E;
    d.C = C;
    d.rows = g.rows;
    const bool infeasible = ((g.rows & SL_BOUND) && C < 0.0) ||
                            ((g.rows & SL_ENERGY) && E < ((g.rows & SL_MASS) ? dv.M * dv.M : 0.0));
    SliceZ<double> z{1.0, 0.0, uh0, uhh, 0.0, 0.0, 0.0};
    SliceEval<double> e;
    if (infeasible) {
      slice_eval(d, z, e);
      R = SliceResult{0, 0, SNAP_SAMPLE_INFEASIBLE_PARAMS, 0};
    } else {
      R = slice_newton(d, z, e, o);
    }
    A = z.a; Cc = z.c; P0 = z.p0; PH = z.ph;
    lmd = z.lm; led = z.le; lbd = z.lb;
    hm = e.hm; he = e.he; hb = e.hb; res = e.res;
    S1d = a1; S2d = a2;
  }
  if (!range_ok) {
    st.iters = R.iters;
    st.backtracks = R.backtracks;
    st.status = R.status;
    st.corrections = R.corrections;
    st.kkt_inf = res;
    st.h_inf = t1_nan_max(t1_nan_max(fabs(hm), fabs(he)), fabs(hb));
    const double am1 = A - 1.0;
    st.obj = 0.5 * (am1 * am1 * S2d + 2.0 * am1 * Cc * S1d + Cc * Cc * (double)(nx - 2) +
                    (P0 - uh0) * (P0 - uh0) + (PH - uhh) * (PH - uhh));
  }
  if (g.off_mass >= 0) lb[g.off_mass + k] = lmd;
  if (g.off_energy >= 0) lb[g.off_energy + k] = led;
  if (g.off_bound >= 0) lb[g.off_bound + k] = lbd;
  *stat = st;
}

// LPS = 2^lg lanes per slice in phases 1 and 3 (2, 4 or 8): 32 / LPS slices per round, LPS
// rounds.  LPS_LOG2 > 0 fixes lg at compile time (the per-problem kernel); LPS_LOG2 = 0 takes
// lg = lps_log2 at run time, so that one instance of the tile serves every group of the uneven
// batch.  A different LPS sums the moments in a different order (results agree to rounding).
// CH: 16-byte loads in flight per lane in phases 1 and 3.
template <class Addr, int LPS_LOG2 = 0, int CH = 8>
__device__ __forceinline__ void mixed_tile(const Geom1D &g, const Addr &ad, long long sbase,
                                           long long send, const SolverOpts &o,
                                           const SliceOptsT<float> &so_f,
                                           const SliceOptsT<df64> &so_d, const df64 &dxd,
                                           int lps_log2) {
  const int lg = LPS_LOG2 > 0 ? LPS_LOG2 : lps_log2;
  const int LPS = 1 << lg;
  const int SPR = 32 >> lg;         // slices per round
  const int lane = threadIdx.x & 31;
  const int q = lane >> lg;         // group: slice SPR*rho + q of round rho
  const int r = lane & (LPS - 1);   // lane within the group
  const int nx = g.nx, ih = g.ih;
  // ---------------- phase 1 ----------------
  ad.prefetch(sbase, send, lane);
  df64 m1(0.0f, 0.0f), m2(0.0f, 0.0f);
  float mmx = -INFINITY, mmn = INFINITY;
  int mok = 1;
#pragma unroll 1
  for (int rho = 0; rho < LPS; ++rho) {
    const long long s = sbase + SPR * rho + q;
    float s1h = 0.0f, s1e = 0.0f, s2h = 0.0f, s2e = 0.0f;
    float pmx = -INFINITY, pmn = INFINITY;
    int ok = 1;
    if (s < send) {
      const int k = ad.slice_k(s);
      const double *row = ad.row_in(s);
      if (k == 0) {
        // the IC slice is handled by the per-sample prepare kernel
      } else {
        // CH independent 16-byte loads in flight per lane, then the accumulation
        for (int i0 = 2 * r; i0 < nx; i0 += 2 * LPS * CH) {
          double2 v[CH];
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const int i = i0 + 2 * LPS * c;
            v[c] = (i < nx && ad.row_ok(SNAP_SITE_MOMENT_ROW, s, i))
                       ? __ldg(reinterpret_cast<const double2 *>(row + i)) : make_double2(0.0, 0.0);
          }
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const int i = i0 + 2 * LPS * c;
            if (i >= nx) break;
            float h0, l0, h1, l1;
            ok &= df_split_trunc_fast(v[c].x, h0, l0);
            ok &= df_split_trunc_fast(v[c].y, h1, l1);
            if (i == 0 || i == ih) { h0 = 0.0f; l0 = 0.0f; }
            if (i + 1 == ih) { h1 = 0.0f; l1 = 0.0f; }
            else { pmx = fmaxf(pmx, h1); pmn = fminf(pmn, h1); }
            if (i != 0 && i != ih) { pmx = fmaxf(pmx, h0); pmn = fminf(pmn, h0); }
            // S1 += h + l (TwoSum on the leading parts, errors accumulated in s1e)
            {
              float t = s1h + h0, bb = t - s1h;
              s1e += ((s1h - (t - bb)) + (h0 - bb)) + l0;
              s1h = t;
              t = s1h + h1; bb = t - s1h;
              s1e += ((s1h - (t - bb)) + (h1 - bb)) + l1;
              s1h = t;
            }
            // S2 += (h + l)^2 = h^2 (TwoProd) + 2 h l (+ l^2, below 2^-48 relative)
            {
              float p = h0 * h0;
              float pe = fmaf(h0, h0, -p);
              pe = fmaf(h0 + h0, l0, pe);
              float t = s2h + p, bb = t - s2h;
              s2e += ((s2h - (t - bb)) + (p - bb)) + pe;
              s2h = t;
              p = h1 * h1;
              pe = fmaf(h1, h1, -p);
              pe = fmaf(h1 + h1, l1, pe);
              t = s2h + p; bb = t - s2h;
              s2e += ((s2h - (t - bb)) + (p - bb)) + pe;
              s2h = t;
            }
          }
        }
      }
    }
    df64 a1 = df_fast_two_sum(s1h, s1e);
    df64 a2 = df_fast_two_sum(s2h, s2e);
#pragma unroll
    for (int off = 1; off < LPS; off <<= 1) {
      a1 = a1 + t1_shfl_df(a1, off);
      a2 = a2 + t1_shfl_df(a2, off);
      pmx = fmaxf(pmx, __shfl_xor_sync(0xffffffffu, pmx, off));
      pmn = fminf(pmn, __shfl_xor_sync(0xffffffffu, pmn, off));
      ok &= __shfl_xor_sync(0xffffffffu, ok, off);
    }
    if (r == rho) {
      m1 = a1; m2 = a2; mmx = pmx; mmn = pmn; mok = ok;
    }
  }
  ad.before_solve(sbase, send, lane);
  // ---------------- phase 2: one slice per lane ----------------
  const long long s = sbase + SPR * r + q;
  int kind = T1_KIND_NONE;
  double A = 1.0, Cc = 0.0, P0 = 0.0, PH = 0.0;
  if (s < send && ad.slice_ok(s)) {
    const int k = ad.slice_k(s);
    if (k != 0) {     // IC slice (k = 0): solved by the caller
      const double *row = ad.row_in(s);
      kind = T1_KIND_MOMENT;
      t1_solve_slice(g, k, m1, m2, mmx, mmn, mok, __ldg(row), __ldg(row + g.ih), row,
                     ad.par(s), ad.derived(s), ad.lam_of(s), ad.stat(s), o, so_f,
                     so_d, dxd, A, Cc, P0, PH);
    }
  }
  // ---------------- phase 3: write-back, LPS lanes per slice ----------------
#pragma unroll 1
  for (int rho = 0; rho < LPS; ++rho) {
    const int src = LPS * q + rho;
    const double a = __shfl_sync(0xffffffffu, A, src);
    const double c0 = __shfl_sync(0xffffffffu, Cc, src);
    const double p0 = __shfl_sync(0xffffffffu, P0, src);
    const double ph = __shfl_sync(0xffffffffu, PH, src);
    const int kd = __shfl_sync(0xffffffffu, kind, src);
    const long long s2 = sbase + SPR * rho + q;
    if (s2 >= send || kd == T1_KIND_NONE) continue;
    const double *row = ad.row_in(s2);
    double *out = ad.row_out(s2);
    if (kd == T1_KIND_MOMENT) {
      for (int i0 = 2 * r; i0 < nx; i0 += 2 * LPS * CH) {
        double2 v[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const int i = i0 + 2 * LPS * c;
          v[c] = (i < nx) ? __ldg(reinterpret_cast<const double2 *>(row + i)) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const int i = i0 + 2 * LPS * c;
          if (i >= nx) break;
          double2 w;
          w.x = (i == 0) ? p0 : ((i == ih) ? ph : fma(a, v[c].x, c0));
          w.y = (i + 1 == ih) ? ph : fma(a, v[c].y, c0);
          if (ad.row_ok(SNAP_SITE_MIXED_ROW, s2, i)) *reinterpret_cast<double2 *>(out + i) = w;
        }
      }
    }
  }
}

}  // namespace
