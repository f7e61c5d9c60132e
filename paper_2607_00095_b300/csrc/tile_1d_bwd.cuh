// The warp tile of the 1-D implicit-function adjoint (families A/B): one warp, up to 32
// consecutive slices of a virtual batch whose slices are located by the address policy Bwd.
// Used by the per-problem adjoint kernel k1d_bwd_mixed (kern_1d_bwd_mixed.cu) and by the
// uneven-batch adjoint kernel (kern_batch.cu), so that both produce the same bits.
//
// For every slice k >= 1 the adjoint solves K [a; b] = [gbar; 0] with the KKT matrix of
// Appendix B at the solution (W = diag(w interior, wb at i in {0, h})):
//     S b = J W^-1 gbar,   a = W^-1 (gbar - J^T b),   S = J W^-1 J^T.
// J W^-1 gbar needs the interior sums sum gbar_i and sum u_i gbar_i, and S is rebuilt from
// sum u_i and sum u_i^2 (storing the forward's factors and reading them back measured slower
// than rebuilding S here):
//   phase 1  (4 lanes per slice): float-pair split of u and gbar with integer operations only
//            (|x - hi - lo| < 2^-46 |x|), double-float sums;
//   phase 2  (one slice per lane): S rebuilt and S b = v solved in double-float; the
//            per-slice contributions to dL/dtheta;
//   phase 3  (4 lanes per slice): a_i = gbar_i / w - (dx b_m + 2 dx u_i b_e) / w with two
//            FP64 FMAs per element.
// IC slices (a = 0) are not live: the caller writes them.  A slice whose values leave the
// float-pair range is done by its owner lane in FP64.
//
// Address policy Bwd (all device, inlined):
//   live(s)                  slice s exists and is not an IC slice
//   slice_k(s)               its time index
//   row_u(s) / row_g(s)      u and dL/du of the slice;  row_out(s)  dL/du_hat of the slice
//   lam_of(s)                the sample's multipliers;  bad(s)  its forward status is not OK
//   derived(s)               the sample's SampleDerived
//   contrib_at(s)            the slice's BwdContrib slot
//   gp_of(s)                 the sample's dL/dparams row or nullptr
//   before_solve(lane)       hook run by the whole warp between phases 1 and 2
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "slice_newton.cuh"
#include "snap_internal.h"

namespace {

__device__ __forceinline__ df64 tb_shfl_df(df64 v, int off) {
  return df64(__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off));
}

// error-free accumulation of h into (s, e): s + e tracks the running sum
__device__ __forceinline__ void tb_acc2(float &s, float &e, float h, float l) {
  const float t = s + h, bb = t - s;
  e += ((s - (t - bb)) + (h - bb)) + l;
  s = t;
}

// (xh + xl)(yh + yl) accumulated into (s, e): TwoProd of the leading parts plus cross terms
__device__ __forceinline__ void tb_acc_prod(float &s, float &e, float xh, float xl, float yh,
                                            float yl) {
  const float p = xh * yh;
  float pe = fmaf(xh, yh, -p);
  pe = fmaf(xh, yl, pe);
  pe = fmaf(xl, yh, pe);
  const float t = s + p, bb = t - s;
  e += ((s - (t - bb)) + (p - bb)) + pe;
  s = t;
}

// L2 residency hint for the adjoint tile: u and dL/du are read twice (the sums of phase 1,
// the write-back of phase 3) and the whole batch's u and dL/du are in flight at once, so the
// second reads and the dL/du_hat stores mark their lines for early eviction (evict_first): the
// outputs stream through L2 without pushing out inputs that other tiles have still to re-read.
// The second reads take the non-coherent path: the kernel never writes u or dL/du (the entry
// point refuses outputs that alias them).
__device__ __forceinline__ unsigned long long tb_policy_drop() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ double2 tb_ld2(const double *p, unsigned long long pol) {
  double2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
               : "=d"(v.x), "=d"(v.y)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void tb_st2(double *p, double2 v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p), "d"(v.x),
               "d"(v.y), "l"(pol)
               : "memory");
}

__device__ __forceinline__ df64 tb_df_pow(df64 x, int k) {
  df64 r(1.0f, 0.0f);
  while (k > 0) {
    if (k & 1) r = r * x;
    x = x * x;
    k >>= 1;
  }
  return r;
}

__device__ __forceinline__ df64 tb_split_df(double x, bool &ok) {
  float h, l;
  ok &= df_split(x, h, l);
  return df64(h, l);
}

// Coefficients of the write-back a_i = gbar_i iw + u_i kx + k0 (interior) and
// gbar_i iwb + u_i kxb + k0b (i = 0, nx/2) of one slice.
struct BwdCoef {
  double iw, iwb, kx, k0, kxb, k0b;
};

// Phase 2 of one live slice s (one lane): S b = J W^-1 gbar from the slice's interior sums
// (mg = sum gbar_i, mug = sum u_i gbar_i, mu / muu = sum u_i / u_i^2; mok: every value in the
// float-pair range), the slice's rows urow / grow (any address
// space: the boundary values, and the FP64 fallback, read them); writes the slice's
// contribution to dL/dparams and its boundary-parameter gradient, returns the write-back
// coefficients (NaN for a failed sample).
template <class Bwd>
__device__ __forceinline__ BwdCoef bwd_slice(const Geom1D &g, const Bwd &ad, long long s,
                                             const df64 &mg, const df64 &mug, const df64 &mu,
                                             const df64 &muu, int mok, const double *urow,
                                             const double *grow, const df64 &dxd) {
  const int nx = g.nx, ih = g.ih;
  BwdCoef out;
  double ciw = 0.0, ciwb = 0.0, ckx = 0.0, ck0 = 0.0, ckxb = 0.0, ck0b = 0.0;
  {
  const int k = ad.slice_k(s);
  const bool bad = ad.bad(s);
  const double *lb = ad.lam_of(s);
  const double u0 = urow[0], uhv = urow[ih], g0 = grow[0], ghv = grow[ih];
  const double lme = (g.rows & SL_ENERGY) ? lb[g.off_energy + k] : 0.0;
  const double lbb = (g.rows & SL_BOUND) ? lb[g.off_bound + k] : 0.0;
  bool ok = mok;
  const df64 U0 = tb_split_df(u0, ok), UH = tb_split_df(uhv, ok), G0 = tb_split_df(g0, ok), GH = tb_split_df(ghv, ok);
  const df64 LE = tb_split_df(lme, ok), LB = tb_split_df(lbb, ok);
  const df64 two(2.0f, 0.0f), one(1.0f, 0.0f), zero(0.0f, 0.0f);
  double bm = 0.0, be = 0.0, bbv = 0.0, w = 1.0, wb = 1.0;
  if (ok) {
    const df64 W = one + two * dxd * LE;
    const df64 WB = W + two * LB;
    const df64 iw = df64(1.0f, 0.0f) / W, iwb = df64(1.0f, 0.0f) / WB;
    // v = J W^-1 gbar
    const df64 pg2 = U0 * G0 + UH * GH;
    const bool hm = g.rows & SL_MASS, he = g.rows & SL_ENERGY, hbnd = g.rows & SL_BOUND;
    const df64 v0 = hm ? dxd * (mg * iw + (G0 + GH) * iwb) : zero;
    const df64 v1 = he ? two * dxd * (mug * iw + pg2 * iwb) : zero;
    const df64 v2 = hbnd ? two * pg2 * iwb : zero;
    Ldl3<df64> f;
    SliceIn<df64> d;
    d.dx = dxd;
    d.n = df64((float)(nx - 2), 0.0f);
    d.rows = g.rows;
    d.nint = nx - 2;
    SliceZ<df64> z;
    z.p0 = U0; z.ph = UH;
    df64 s00, s01, s02, s11, s12, s22;
    slice_schur(d, z, mu, muu, iw, iwb, s00, s01, s02, s11, s12, s22);
    if (ldl3_factor(s00, s01, s02, s11, s12, s22, f)) {
      df64 xm, xe, xb;
      ldl3_solve(f, v0, v1, v2, xm, xe, xb);
      if (!hm) xm = zero;
      if (!he) xe = zero;
      if (!hbnd) xb = zero;
      bm = (double)xm; be = (double)xe; bbv = (double)xb;
      w = (double)W; wb = (double)WB;
      // a = W^-1 (gbar - dx b_m - 2 dx u b_e [- 2 u b_b at the boundary])
      const df64 kx = -(two * dxd * xe) * iw, k0 = -(dxd * xm) * iw;
      const df64 kxb = -(two * dxd * xe + two * xb) * iwb, k0b = -(dxd * xm) * iwb;
      ciw = (double)iw; ciwb = (double)iwb;
      ckx = (double)kx; ck0 = (double)k0; ckxb = (double)kxb; ck0b = (double)k0b;
    } else {
      ciw = ciwb = ckx = ck0 = ckxb = ck0b = NAN;
      bm = be = bbv = NAN;
    }
  } else {
    // FP64 by this lane: sums, S and the solve
    double sgd = 0.0, sugd = 0.0, sud = 0.0, suud = 0.0;
    for (int i = 0; i < nx; ++i) {
      if (i == 0 || i == ih) continue;
      const double uv = urow[i], gv = grow[i];
      sgd += gv;
      sugd = fma(uv, gv, sugd);
      sud += uv;
      suud = fma(uv, uv, suud);
    }
    w = 1.0 + 2.0 * g.dx * lme;
    wb = w + 2.0 * lbb;
    const double iw = 1.0 / w, iwb = 1.0 / wb;
    const double pg2 = u0 * g0 + uhv * ghv;
    const bool hm = g.rows & SL_MASS, he = g.rows & SL_ENERGY, hbnd = g.rows & SL_BOUND;
    const double v0 = hm ? g.dx * (sgd * iw + (g0 + ghv) * iwb) : 0.0;
    const double v1 = he ? 2.0 * g.dx * (sugd * iw + pg2 * iwb) : 0.0;
    const double v2 = hbnd ? 2.0 * pg2 * iwb : 0.0;
    SliceIn<double> d;
    d.dx = g.dx;
    d.n = (double)(nx - 2);
    d.rows = g.rows;
    d.nint = nx - 2;
    SliceZ<double> z;
    z.p0 = u0; z.ph = uhv;
    double s00, s01, s02, s11, s12, s22;
    slice_schur(d, z, sud, suud, iw, iwb, s00, s01, s02, s11, s12, s22);
    Ldl3<double> f;
    if (ldl3_factor(s00, s01, s02, s11, s12, s22, f)) {
      ldl3_solve(f, v0, v1, v2, bm, be, bbv);
      if (!hm) bm = 0.0;
      if (!he) be = 0.0;
      if (!hbnd) bbv = 0.0;
    } else {
      bm = be = bbv = NAN;
    }
    ciw = iw; ciwb = iwb;
    ckx = -2.0 * g.dx * be * iw; ck0 = -g.dx * bm * iw;
    ckxb = -(2.0 * g.dx * be + 2.0 * bbv) * iwb; ck0b = -g.dx * bm * iwb;
  }
  if (bad) { ciw = ciwb = ckx = ck0 = ckxb = ck0b = NAN; }
  out = BwdCoef{ciw, ciwb, ckx, ck0, ckxb, ck0b};
  BwdContrib c{bm, 0.0, 0.0, 0.0};
  if (g.rows & SL_ENERGY) {
    const SampleDerived dv = ad.derived(s);
    const double t = (double)k / (double)(g.nt - 1);
    const double ex = (double)tb_df_pow(df64(dv.qh, dv.ql), k);
    const bool expb = dv.E0 * ex >= dv.M * dv.M + g.energy_floor;
    c.bex = expb ? be * ex : 0.0;
    c.bfl = expb ? 0.0 : be;
    c.br = expb ? -be * t * dv.E0 * ex : 0.0;
  }
  *ad.contrib_at(s) = c;
  double *gpr = ad.gp_of(s);
  if (gpr && (g.rows & SL_BOUND)) gpr[g.p_c + k] = bad ? NAN : bbv;
  (void)w;
  (void)wb;

  }
  return out;
}

template <class Bwd>
// dxd: dx in double-float, converted on the host (a conversion here would hold the FP64 pipe
// ahead of the tile's first loads)
__device__ __forceinline__ void bwd_tile(const Geom1D &g, const Bwd &ad, long long sbase,
                                         const df64 &dxd) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int q = lane >> 2;
  const int r = lane & 3;
  const int nx = g.nx, ih = g.ih;
  const unsigned long long pol_drop = tb_policy_drop();
  // ---------------- phase 1: sums over the interior ----------------
  df64 mg(0.0f, 0.0f), mug(0.0f, 0.0f), mu(0.0f, 0.0f), muu(0.0f, 0.0f);
  int mok = 1;
#pragma unroll 1
  for (int rho = 0; rho < 4; ++rho) {
    const long long s = sbase + 8 * rho + q;
    float sg = 0.f, eg = 0.f, sug = 0.f, eug = 0.f, su = 0.f, eu = 0.f, suu = 0.f, euu = 0.f;
    int ok = 1;
    if (ad.live(s)) {
      const double *urow = ad.row_u(s);
      const double *grow = ad.row_g(s);
      constexpr int CH = 8;
      for (int i0 = 2 * r; i0 < nx; i0 += 8 * CH) {
        double2 vu[CH], vg[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const int i = i0 + 8 * c;
          vu[c] = (i < nx) ? *reinterpret_cast<const double2 *>(urow + i) : make_double2(0.0, 0.0);
          vg[c] = (i < nx) ? *reinterpret_cast<const double2 *>(grow + i) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const int i = i0 + 8 * c;
          if (i >= nx) break;
          float uh0, ul0, uh1, ul1, gh0, gl0, gh1, gl1;
          ok &= df_split_trunc(vu[c].x, uh0, ul0);
          ok &= df_split_trunc(vu[c].y, uh1, ul1);
          ok &= df_split_trunc(vg[c].x, gh0, gl0);
          ok &= df_split_trunc(vg[c].y, gh1, gl1);
          if (i == 0 || i == ih) { uh0 = ul0 = gh0 = gl0 = 0.0f; }
          if (i + 1 == ih) { uh1 = ul1 = gh1 = gl1 = 0.0f; }
          tb_acc2(sg, eg, gh0, gl0);
          tb_acc2(sg, eg, gh1, gl1);
          tb_acc_prod(sug, eug, uh0, ul0, gh0, gl0);
          tb_acc_prod(sug, eug, uh1, ul1, gh1, gl1);
          tb_acc2(su, eu, uh0, ul0);
          tb_acc2(su, eu, uh1, ul1);
          tb_acc_prod(suu, euu, uh0, ul0, uh0, ul0);
          tb_acc_prod(suu, euu, uh1, ul1, uh1, ul1);
        }
      }
    }
    df64 a_g = df_fast_two_sum(sg, eg), a_ug = df_fast_two_sum(sug, eug);
    df64 a_u = df_fast_two_sum(su, eu), a_uu = df_fast_two_sum(suu, euu);
#pragma unroll
    for (int off = 1; off < 4; off <<= 1) {
      a_g = a_g + tb_shfl_df(a_g, off);
      a_ug = a_ug + tb_shfl_df(a_ug, off);
      a_u = a_u + tb_shfl_df(a_u, off);
      a_uu = a_uu + tb_shfl_df(a_uu, off);
      ok &= __shfl_xor_sync(FULL, ok, off);
    }
    if (r == rho) { mg = a_g; mug = a_ug; mu = a_u; muu = a_uu; mok = ok; }
  }
  // ---------------- phase 2: one slice per lane ----------------
  ad.before_solve(lane);
  const long long s = sbase + 8 * r + q;
  int live = 0;
  double ciw = 0.0, ciwb = 0.0, ckx = 0.0, ck0 = 0.0, ckxb = 0.0, ck0b = 0.0;
  if (ad.live(s)) {
    live = 1;
    const BwdCoef cf = bwd_slice(g, ad, s, mg, mug, mu, muu, mok, ad.row_u(s), ad.row_g(s), dxd);
    ciw = cf.iw; ciwb = cf.iwb; ckx = cf.kx; ck0 = cf.k0; ckxb = cf.kxb; ck0b = cf.k0b;
  }
  // ---------------- phase 3: a = W^-1 (gbar - J^T b), 4 lanes per slice ----------------
#pragma unroll 1
  for (int rho = 0; rho < 4; ++rho) {
    const int src = 4 * q + rho;
    const double iw = __shfl_sync(FULL, ciw, src);
    const double iwb = __shfl_sync(FULL, ciwb, src);
    const double kx = __shfl_sync(FULL, ckx, src);
    const double k0 = __shfl_sync(FULL, ck0, src);
    const double kxb = __shfl_sync(FULL, ckxb, src);
    const double k0b = __shfl_sync(FULL, ck0b, src);
    const int lv = __shfl_sync(FULL, live, src);
    const long long s2 = sbase + 8 * rho + q;
    if (!lv) continue;
    const double *urow = ad.row_u(s2);
    const double *grow = ad.row_g(s2);
    double *out = ad.row_out(s2);
    constexpr int CH = 8;
    for (int i0 = 2 * r; i0 < nx; i0 += 8 * CH) {
      double2 vu[CH], vg[CH];
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int i = i0 + 8 * c;
        vu[c] = (i < nx) ? tb_ld2(urow + i, pol_drop) : make_double2(0.0, 0.0);
        vg[c] = (i < nx) ? tb_ld2(grow + i, pol_drop) : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int i = i0 + 8 * c;
        if (i >= nx) break;
        const bool b0 = (i == 0 || i == ih), b1 = (i + 1 == ih);
        double2 w;
        w.x = fma(vg[c].x, b0 ? iwb : iw, fma(vu[c].x, b0 ? kxb : kx, b0 ? k0b : k0));
        w.y = fma(vg[c].y, b1 ? iwb : iw, fma(vu[c].y, b1 ? kxb : kx, b1 ? k0b : k0));
        tb_st2(out + i, w, pol_drop);
      }
    }
  }
}

}  // namespace
