// Newton-KKT for one 1-D time slice (k >= 1) of families A/B in moment form.
//
// Rows of slice k (Appendix B notation, L = f + lambda^T h, f = 1/2 ||u - u_hat||^2):
//   mass     h_m = dx sum_i u_i - M
//   energy   h_e = dx sum_i u_i^2 - E
//   boundary h_b = u_0^2 + u_h^2 - C          (h = nx/2)
// grad_u L = u - u_hat + dx lam_m 1 + 2 dx lam_e u + 2 lam_b (u_0 e_0 + u_h e_h)
// W = diag(alpha on the interior, beta at i in {0, h}), alpha = 1 + 2 dx lam_e,
// beta = alpha + 2 lam_b.
//
// Moment form.  W is uniform on the interior (i not in {0, h}) and grad_u L_i is affine in
// (u_i, u_hat_i) with coefficients shared by the interior, so a Newton step maps an interior
// iterate of the form u_i = a u_hat_i + c to another one of the same form.  Starting from
// u = u_hat (a = 1, c = 0), every iterate, line-search trial and the solution are therefore
// described by (a, c, u_0, u_h, lam_m, lam_e, lam_b), and every sum the Newton-KKT step
// needs reduces to the interior moments S1 = sum u_hat_i, S2 = sum u_hat_i^2 (and the
// interior max / min of u_hat for the infinity norm of F).  The iteration below is the
// same sequence of Newton-KKT steps, line-search trials and stopping tests as the dense
// per-element iteration, evaluated in O(1) per step.
//
// Newton step through the Schur complement of the KKT matrix of Appendix B:
//   S dlam = h - J W^-1 grad L,  S = J W^-1 J^T (3x3),  du = -W^-1 (grad L + J^T dlam).
// Inertia of K = In(W) + In(-S) (Haynsworth); the required inertia is (nx, m, 0).
// Globalisation: Armijo on phi = 1/2 ||F||^2, first trial capped so that W stays positive
// definite (both of its diagonal values keep >= w_keep of their current value); the
// second-order condition is checked at the converged point.
//
// Stationarity kept along the iteration.  The iteration starts at u = u_hat, lam = 0, where
// grad_u L = 0, and every trial point is (u(lam_t), lam_t) with lam_t = lam + t dlam and
// u(lam) = argmin_u L(u, lam): interior u_i = (u_hat_i - dx lam_m) / alpha, boundary
// u_j = (u_hat_j - dx lam_m) / beta, i.e. a = 1/alpha, c = -dx lam_m / alpha (slice_stationary).
// With grad_u L = 0 the Newton-KKT step above reduces to S dlam = h.  W stays positive definite
// (the cap), so L(., lam) is strictly convex and a KKT point reached this way is the unique
// global minimiser of the slice's projection: the result does not depend on the path.
//
// The scalar type T is double (FP64 pipe), float, or df64 (double-float on the FP32 pipe,
// df64.cuh).  slice_solve_mixed runs the iteration in float while float steps make reliable
// progress, then continues in df64 to the FP64 stopping tolerance: the same Newton-KKT
// iteration, with the early (inexact) steps taken in a cheaper precision.
#pragma once

#include "df64.cuh"
#include "snap_internal.h"

template <class T>
struct SliceIn {
  T S1, S2, mx, mn;   // interior moments / extremes of u_hat
  T uh0, uhh;         // u_hat at i = 0 and i = nx/2
  T n;                // interior count nx - 2
  T dx, M, E, C;      // rhs of the slice rows
  int rows;           // SL_* bits
  int nint;           // interior count as an integer
};

template <class T>
struct SliceZ {
  T a, c, p0, ph, lm, le, lb;
};

template <class T>
struct SliceEval {
  T alpha, beta, P, Q, su, su2, g0, gh, hm, he, hb, phi, res;
};

// option values converted once per slice
template <class T>
struct SliceOptsT {
  T tol, c1x2, delta0, w_keep1;   // tol, 2 c1, delta0, 1 - w_keep
  int max_iter, max_backtracks, max_corrections;
  bool cap;
};

template <class T>
DF_INL T sl_abs(T x) { return x < T(0) ? -x : x; }

// 1/x: exact division in FP64, the hardware reciprocal approximation in float (df_rcp; the
// float phase is a predictor whose steps are refined in double-float), the double-float
// quotient in df64
DF_INL double sl_rcp(double x) { return 1.0 / x; }
DF_INL float sl_rcp(float x) { return df_rcp(x); }
DF_INL df64 sl_rcp(df64 x) { return df64(1.0f, 0.0f) / x; }

template <class T>
DF_INL T sl_max(T x, T y) { return (x < y) ? y : x; }

DF_INL bool sl_finite(double x) { return isfinite(x); }
DF_INL bool sl_finite(float x) { return isfinite(x); }
DF_INL bool sl_finite(df64 x) { return isfinite(x.hi); }

template <class T>
DF_INL T sl_from(double x);
template <>
DF_INL double sl_from<double>(double x) { return x; }
template <>
DF_INL float sl_from<float>(double x) { return df_d2f(x); }
template <>
DF_INL df64 sl_from<df64>(double x) { return df64(x); }

DF_INL double sl_to_double(double x) { return x; }
DF_INL double sl_to_double(float x) { return (double)x; }
DF_INL double sl_to_double(df64 x) { return (double)x; }

template <class T>
DF_INL SliceOptsT<T> slice_opts(const SolverOpts &o, double tol) {
  SliceOptsT<T> s;
  s.tol = sl_from<T>(tol);
  s.c1x2 = sl_from<T>(2.0 * o.c1);
  s.delta0 = sl_from<T>(o.delta0);
  s.w_keep1 = sl_from<T>(1.0 - o.w_keep);
  s.cap = o.w_keep > 0.0;
  s.max_iter = o.max_iter;
  s.max_backtracks = o.max_backtracks;
  s.max_corrections = o.max_corrections;
  return s;
}

// phi and ||F||_inf at z; NaN propagates into res
template <class T>
DF_INL void slice_eval(const SliceIn<T> &d, const SliceZ<T> &z,
                                           SliceEval<T> &e) {
  const T two = T(2), one = T(1);
  e.alpha = one + two * d.dx * z.le;
  e.beta = e.alpha + two * z.lb;
  e.P = e.alpha * z.a - one;
  e.Q = e.alpha * z.c + d.dx * z.lm;
  e.su = z.a * d.S1 + z.c * d.n;
  e.su2 = z.a * z.a * d.S2 + two * z.a * z.c * d.S1 + z.c * z.c * d.n;
  e.g0 = e.beta * z.p0 - d.uh0 + d.dx * z.lm;
  e.gh = e.beta * z.ph - d.uhh + d.dx * z.lm;
  const T pp = z.p0 * z.p0 + z.ph * z.ph;
  e.hm = (d.rows & SL_MASS) ? d.dx * (e.su + z.p0 + z.ph) - d.M : T(0);
  e.he = (d.rows & SL_ENERGY) ? d.dx * (e.su2 + pp) - d.E : T(0);
  e.hb = (d.rows & SL_BOUND) ? pp - d.C : T(0);
  T gi2 = e.P * e.P * d.S2 + two * e.P * e.Q * d.S1 + e.Q * e.Q * d.n;
  if (gi2 < T(0)) gi2 = T(0);
  const T ginf = sl_max(sl_abs(e.P * d.mx + e.Q), sl_abs(e.P * d.mn + e.Q));
  e.phi = (gi2 + e.g0 * e.g0 + e.gh * e.gh + e.hm * e.hm + e.he * e.he + e.hb * e.hb) * T(0.5f);
  T r = ginf;
  T c;
  c = sl_abs(e.g0); r = (r < c || c != c) ? c : r;
  c = sl_abs(e.gh); r = (r < c || c != c) ? c : r;
  c = sl_abs(e.hm); r = (r < c || c != c) ? c : r;
  c = sl_abs(e.he); r = (r < c || c != c) ? c : r;
  c = sl_abs(e.hb); r = (r < c || c != c) ? c : r;
  if (e.phi != e.phi) r = e.phi;
  e.res = r;
}

// df64 evaluation: the residual components, which cancel as the iteration converges, are
// formed in df64; the merit phi (compared by the Armijo test against a factor 1 - 2 c1 t,
// far above float rounding) and ||F||_inf are then formed from their float images.
DF_INL void slice_eval(const SliceIn<df64> &d, const SliceZ<df64> &z, SliceEval<df64> &e) {
  const df64 two(2.0f, 0.0f), one(1.0f, 0.0f);
  e.alpha = one + two * d.dx * z.le;
  e.beta = e.alpha + two * z.lb;
  e.P = e.alpha * z.a - one;
  e.Q = e.alpha * z.c + d.dx * z.lm;
  e.su = z.a * d.S1 + z.c * d.n;
  e.su2 = z.a * z.a * d.S2 + two * z.a * z.c * d.S1 + z.c * z.c * d.n;
  e.g0 = e.beta * z.p0 - d.uh0 + d.dx * z.lm;
  e.gh = e.beta * z.ph - d.uhh + d.dx * z.lm;
  const df64 pp = z.p0 * z.p0 + z.ph * z.ph;
  const df64 zero(0.0f, 0.0f);
  e.hm = (d.rows & SL_MASS) ? d.dx * (e.su + z.p0 + z.ph) - d.M : zero;
  e.he = (d.rows & SL_ENERGY) ? d.dx * (e.su2 + pp) - d.E : zero;
  e.hb = (d.rows & SL_BOUND) ? pp - d.C : zero;
  const float P = e.P.hi, Q = e.Q.hi, g0 = e.g0.hi, gh = e.gh.hi;
  const float hm = e.hm.hi, he = e.he.hi, hb = e.hb.hi;
  float gi2 = P * P * d.S2.hi + 2.0f * P * Q * d.S1.hi + Q * Q * d.n.hi;
  if (gi2 < 0.0f) gi2 = 0.0f;
  const float phi = 0.5f * (gi2 + g0 * g0 + gh * gh + hm * hm + he * he + hb * hb);
  float r = fmaxf(fabsf(P * d.mx.hi + Q), fabsf(P * d.mn.hi + Q));
  r = fmaxf(r, fmaxf(fmaxf(fabsf(g0), fabsf(gh)), fmaxf(fmaxf(fabsf(hm), fabsf(he)), fabsf(hb))));
  if (phi != phi) r = phi;
  e.phi = df64(phi, 0.0f);
  e.res = df64(r, 0.0f);
}

// 3x3 symmetric LDL^T without pivoting; returns false on a zero pivot.  The reciprocals of
// the pivots are kept for the solve.
template <class T>
struct Ldl3 {
  T d0, d1, d2, l10, l20, l21, i0, i1, i2;
};

template <class T>
DF_INL bool ldl3_factor(T s00, T s01, T s02, T s11, T s12, T s22, Ldl3<T> &f) {
  f.d0 = s00;
  if (f.d0 == T(0)) return false;
  f.i0 = sl_rcp(f.d0);
  f.l10 = s01 * f.i0;
  f.l20 = s02 * f.i0;
  f.d1 = s11 - f.l10 * s01;
  if (f.d1 == T(0)) return false;
  f.i1 = sl_rcp(f.d1);
  const T t12 = s12 - f.l20 * s01;
  f.l21 = t12 * f.i1;
  f.d2 = s22 - f.l20 * s02 - f.l21 * t12;
  if (f.d2 == T(0)) return false;
  f.i2 = sl_rcp(f.d2);
  return true;
}

template <class T>
DF_INL void ldl3_solve(const Ldl3<T> &f, T r0, T r1, T r2, T &x0, T &x1, T &x2) {
  const T y0 = r0;
  const T y1 = r1 - f.l10 * y0;
  const T y2 = r2 - f.l20 * y0 - f.l21 * y1;
  x2 = y2 * f.i2;
  x1 = y1 * f.i1 - f.l21 * x2;
  x0 = y0 * f.i0 - f.l10 * x1 - f.l20 * x2;
}

// Schur complement S = J W^-1 J^T of the slice rows at z with W diagonal (w interior, wb at
// the two boundary points); absent rows get an identity row so their dlam is 0.
template <class T>
DF_INL void slice_schur(const SliceIn<T> &d, const SliceZ<T> &z, T su,
                                            T su2, T iw, T iwb, T &s00, T &s01, T &s02, T &s11,
                                            T &s12, T &s22) {
  const T two = T(2), four = T(4);
  const T pp = z.p0 * z.p0 + z.ph * z.ph;
  const T ps = z.p0 + z.ph;
  const T dx2 = d.dx * d.dx;
  const bool hm = d.rows & SL_MASS, he = d.rows & SL_ENERGY, hb = d.rows & SL_BOUND;
  s00 = hm ? dx2 * (d.n * iw + two * iwb) : T(1);
  s01 = (hm && he) ? two * dx2 * (su * iw + ps * iwb) : T(0);
  s02 = (hm && hb) ? two * d.dx * ps * iwb : T(0);
  s11 = he ? four * dx2 * (su2 * iw + pp * iwb) : T(1);
  s12 = (he && hb) ? four * d.dx * pp * iwb : T(0);
  s22 = hb ? four * pp * iwb : T(1);
}

// Inertia test of K via In(W) + In(-S).  nint = interior count, m = rows present.
template <class T>
DF_INL bool slice_inertia_ok(const Ldl3<T> &f, T w, T wb, int nint,
                                                 int m_present, int n_absent) {
  if (w == T(0) || wb == T(0)) return false;
  const int npW = (w > T(0) ? nint : 0) + (wb > T(0) ? 2 : 0);
  const int nnW = (w < T(0) ? nint : 0) + (wb < T(0) ? 2 : 0);
  int npS = (f.d0 > T(0)) + (f.d1 > T(0)) + (f.d2 > T(0)) - n_absent;
  int nnS = (f.d0 < T(0)) + (f.d1 < T(0)) + (f.d2 < T(0));
  return (npW + nnS == nint + 2) && (nnW + npS == m_present);
}

struct SliceResult {
  int iters, backtracks, status, corrections;
};

// Second-order sufficient condition at z: inertia of K = (nx, m, 0).
template <class T>
DF_INL bool slice_sosc(const SliceIn<T> &d, const SliceZ<T> &z, const SliceEval<T> &e) {
  const int m_present = ((d.rows & SL_MASS) != 0) + ((d.rows & SL_ENERGY) != 0) +
                        ((d.rows & SL_BOUND) != 0);
  if (e.alpha == T(0) || e.beta == T(0)) return false;
  T s00, s01, s02, s11, s12, s22;
  slice_schur(d, z, e.su, e.su2, sl_rcp(e.alpha), sl_rcp(e.beta), s00, s01, s02, s11, s12, s22);
  Ldl3<T> f;
  return ldl3_factor(s00, s01, s02, s11, s12, s22, f) &&
         slice_inertia_ok(f, e.alpha, e.beta, d.nint, m_present, 3 - m_present);
}

template <class L, class T>
DF_INL L sl_cast(T x);
template <>
DF_INL double sl_cast<double, double>(double x) { return x; }
template <>
DF_INL float sl_cast<float, float>(float x) { return x; }
template <>
DF_INL float sl_cast<float, df64>(df64 x) { return x.hi; }
template <>
DF_INL df64 sl_cast<df64, float>(float x) { return df64(x, 0.0f); }
template <>
DF_INL df64 sl_cast<df64, df64>(df64 x) { return x; }

// u(lam) = argmin_u L(u, lam) in moment form, from z.lm, z.le, z.lb (W positive definite).
template <class T>
DF_INL void slice_stationary(const SliceIn<T> &d, SliceZ<T> &z) {
  const T one = T(1.0f), two = T(2.0f);
  const T al = one + two * d.dx * z.le;
  const T be = al + two * z.lb;
  const T ia = sl_rcp(al), ib = sl_rcp(be);
  const T dlm = d.dx * z.lm;
  z.a = ia;
  z.c = -(dlm * ia);
  z.p0 = (d.uh0 - dlm) * ib;
  z.ph = (d.uhh - dlm) * ib;
}

// Newton-KKT direction at z in precision L: solve S dlam = h - J W^-1 grad L and form
// du = -W^-1 (grad L + J^T dlam) from the residual components of e.  Returns false when
// the Schur complement is singular (or cannot be corrected).
template <class L>
DF_INL bool slice_direction(const SliceIn<L> &d, const SliceZ<L> &z, const SliceEval<L> &e,
                            int max_corrections, L delta0, SliceZ<L> &dz, int &corrections) {
  const int m_present = ((d.rows & SL_MASS) != 0) + ((d.rows & SL_ENERGY) != 0) +
                        ((d.rows & SL_BOUND) != 0);
  const L two = L(2);
  L delta = L(0);
  Ldl3<L> f;
  bool ok = false;
  L iw = L(1), iwb = L(1);
  // max_corrections = 0: plain Newton-Raphson (Appendix B); > 0: shift W + delta I until
  // the inertia of K is (nx, m, 0)
  for (int corr = 0; corr <= max_corrections; ++corr) {
    const L w = e.alpha + delta, wb = e.beta + delta;
    if (!(w == L(0)) && !(wb == L(0))) {
      iw = sl_rcp(w);
      iwb = sl_rcp(wb);
      L s00, s01, s02, s11, s12, s22;
      slice_schur(d, z, e.su, e.su2, iw, iwb, s00, s01, s02, s11, s12, s22);
      if (ldl3_factor(s00, s01, s02, s11, s12, s22, f) &&
          (max_corrections == 0 || slice_inertia_ok(f, w, wb, d.nint, m_present, 3 - m_present))) {
        ok = true;
        break;
      }
    }
    delta = (delta == L(0)) ? delta0 : delta * L(10);
    corrections++;
  }
  if (!ok) return false;
  const L sg = e.P * d.S1 + e.Q * d.n;                                     // sum_int gL
  const L sug = z.a * e.P * d.S2 + (z.a * e.Q + z.c * e.P) * d.S1 + z.c * e.Q * d.n;
  const L pg = z.p0 * e.g0 + z.ph * e.gh;
  const L r0 = (d.rows & SL_MASS) ? e.hm - d.dx * (sg * iw + (e.g0 + e.gh) * iwb) : L(0);
  const L r1 = (d.rows & SL_ENERGY) ? e.he - two * d.dx * (sug * iw + pg * iwb) : L(0);
  const L r2 = (d.rows & SL_BOUND) ? e.hb - two * pg * iwb : L(0);
  L dlm, dle, dlb;
  ldl3_solve(f, r0, r1, r2, dlm, dle, dlb);
  dz.lm = dlm; dz.le = dle; dz.lb = dlb;
  const L dxlm = d.dx * dlm, dxle2 = two * d.dx * dle;
  dz.a = -(e.P + dxle2 * z.a) * iw;
  dz.c = -(e.Q + dxlm + dxle2 * z.c) * iw;
  dz.p0 = -(e.g0 + dxlm + (dxle2 + two * dlb) * z.p0) * iwb;
  dz.ph = -(e.gh + dxlm + (dxle2 + two * dlb) * z.ph) * iwb;
  return true;
}

// Newton-KKT iterations from z (already evaluated in e) until e.res <= so.tol, a failure,
// or `budget` steps; R accumulates counts and receives the status.  F and the merit are
// evaluated in T; the Newton system is assembled and solved in L (L = T: plain Newton;
// L = float with T = df64: Newton steps solved in float against a double-float residual,
// i.e. mixed-precision iterative refinement of the step).
template <class T, class L>
DF_INL void slice_newton_phase(const SliceIn<T> &d, const SliceIn<L> &dl, SliceZ<T> &z,
                               SliceEval<T> &e, const SliceOptsT<T> &so, const SliceOptsT<L> &sl,
                               int budget, SliceResult &R) {
  for (int it = 0;; ++it) {
    if (!sl_finite(e.res)) { R.status = SNAP_SAMPLE_NONFINITE; return; }
    if (e.res <= so.tol) { R.status = SNAP_SAMPLE_OK; return; }
    if (it >= budget) { R.status = SNAP_SAMPLE_MAXITER; return; }
    SliceZ<L> zl{sl_cast<L>(z.a), sl_cast<L>(z.c), sl_cast<L>(z.p0), sl_cast<L>(z.ph),
                 sl_cast<L>(z.lm), sl_cast<L>(z.le), sl_cast<L>(z.lb)};
    SliceEval<L> el;
    el.alpha = sl_cast<L>(e.alpha); el.beta = sl_cast<L>(e.beta);
    el.P = sl_cast<L>(e.P); el.Q = sl_cast<L>(e.Q);
    el.su = sl_cast<L>(e.su); el.su2 = sl_cast<L>(e.su2);
    el.g0 = sl_cast<L>(e.g0); el.gh = sl_cast<L>(e.gh);
    el.hm = sl_cast<L>(e.hm); el.he = sl_cast<L>(e.he); el.hb = sl_cast<L>(e.hb);
    SliceZ<L> dzl;
    if (!slice_direction(dl, zl, el, sl.max_corrections, sl.delta0, dzl, R.corrections)) {
      R.status = SNAP_SAMPLE_SINGULAR;
      return;
    }
    // first trial: the largest t <= 1 keeping both diagonal values of W at >= w_keep times
    // their current value (W is linear in lambda: alpha(t) = alpha + t 2 dx dlam_e,
    // beta(t) = beta + t (2 dx dlam_e + 2 dlam_b))
    L tl = L(1);
    if (sl.cap) {
      const L da = L(2) * dl.dx * dzl.le;
      const L db = da + L(2) * dzl.lb;
      if (el.alpha > L(0) && da < L(0)) {
        const L tm = sl.w_keep1 * el.alpha * sl_rcp(-da);
        if (tm < tl) tl = tm;
      }
      if (el.beta > L(0) && db < L(0)) {
        const L tm = sl.w_keep1 * el.beta * sl_rcp(-db);
        if (tm < tl) tl = tm;
      }
    }
    const SliceZ<T> dz{sl_cast<T>(dzl.a), sl_cast<T>(dzl.c), sl_cast<T>(dzl.p0), sl_cast<T>(dzl.ph),
                       sl_cast<T>(dzl.lm), sl_cast<T>(dzl.le), sl_cast<T>(dzl.lb)};
    T t = sl_cast<T>(tl);
    // Armijo backtracking on phi = 1/2 ||F||^2
    int nb = 0;
    bool accepted = false;
    SliceZ<T> zt;
    SliceEval<T> et;
    for (;;) {
      zt.lm = z.lm + t * dz.lm;  zt.le = z.le + t * dz.le;  zt.lb = z.lb + t * dz.lb;
      slice_stationary(d, zt);
      slice_eval(d, zt, et);
      if (et.phi <= (T(1) - so.c1x2 * t) * e.phi) { accepted = true; break; }
      if (nb >= so.max_backtracks) break;
      nb++;
      t = t * T(0.5f);
    }
    R.backtracks += nb;
    if (!accepted) { R.status = SNAP_SAMPLE_LINESEARCH; return; }
    z = zt;
    e = et;
    R.iters++;
  }
}

// The whole iteration in one precision T (FP64 reference path), with the polishing step (one
// more Newton step after the stopping test, kept when ||F||_inf does not increase).
template <class T>
DF_INL SliceResult slice_newton(const SliceIn<T> &d, SliceZ<T> &z, SliceEval<T> &e,
                                           const SolverOpts &o) {
  SliceResult R{0, 0, SNAP_SAMPLE_OK, 0};
  const SliceOptsT<T> so = slice_opts<T>(o, o.tol_kkt);
  slice_eval(d, z, e);
  slice_newton_phase<T, T>(d, d, z, e, so, so, o.max_iter, R);
  if (R.status == SNAP_SAMPLE_OK) {
    SliceZ<T> dz;
    int corr = 0;
    if (slice_direction(d, z, e, 0, so.delta0, dz, corr)) {
      SliceZ<T> zt;
      zt.lm = z.lm + dz.lm; zt.le = z.le + dz.le; zt.lb = z.lb + dz.lb;
      slice_stationary(d, zt);
      SliceEval<T> et;
      slice_eval(d, zt, et);
      if (et.res <= e.res && et.alpha > T(0) && et.beta > T(0)) {
        z = zt;
        e = et;
      }
    }
  }
  if (R.status == SNAP_SAMPLE_OK && !slice_sosc(d, z, e)) R.status = SNAP_SAMPLE_NOT_MINIMUM;
  return R;
}

template <class T, class S>
DF_INL SliceIn<T> slice_in_cast(const SliceIn<S> &s) {
  SliceIn<T> d;
  d.S1 = sl_from<T>(sl_to_double(s.S1)); d.S2 = sl_from<T>(sl_to_double(s.S2));
  d.mx = sl_from<T>(sl_to_double(s.mx)); d.mn = sl_from<T>(sl_to_double(s.mn));
  d.uh0 = sl_from<T>(sl_to_double(s.uh0)); d.uhh = sl_from<T>(sl_to_double(s.uhh));
  d.n = sl_from<T>(sl_to_double(s.n)); d.dx = sl_from<T>(sl_to_double(s.dx));
  d.M = sl_from<T>(sl_to_double(s.M)); d.E = sl_from<T>(sl_to_double(s.E));
  d.C = sl_from<T>(sl_to_double(s.C));
  d.rows = s.rows;
  d.nint = s.nint;
  return d;
}

DF_INL df64 df_from_float(float x) { return df64(x, 0.0f); }

// Row residuals at the stationary point u(lam) of the current multipliers.  Along the
// iteration u = u(lam) (slice_stationary), so grad_u L = 0 up to rounding (relative 2^-23 in
// float, 2^-46 in double-float, both far below the phase tolerances) and F = (0, h): the loop
// evaluates h and phi = 1/2 ||h||^2 only, and the full ||F||_inf (with grad_u L) is evaluated
// once at the returned point.
template <class T>
struct SliceH {
  T alpha, beta, su, su2, hm, he, hb;
  float phi, res;
};

DF_INL float sl_hi(float x) { return x; }
DF_INL float sl_hi(df64 x) { return x.hi; }

template <class T>
DF_INL void slice_eval_h(const SliceIn<T> &d, const SliceZ<T> &z, SliceH<T> &e) {
  const T one = sl_cast<T, float>(1.0f), two = sl_cast<T, float>(2.0f);
  const T zero = sl_cast<T, float>(0.0f);
  e.alpha = one + two * d.dx * z.le;
  e.beta = e.alpha + two * z.lb;
  e.su = z.a * d.S1 + z.c * d.n;
  e.su2 = z.a * z.a * d.S2 + two * z.a * z.c * d.S1 + z.c * z.c * d.n;
  const T pp = z.p0 * z.p0 + z.ph * z.ph;
  e.hm = (d.rows & SL_MASS) ? d.dx * (e.su + z.p0 + z.ph) - d.M : zero;
  e.he = (d.rows & SL_ENERGY) ? d.dx * (e.su2 + pp) - d.E : zero;
  e.hb = (d.rows & SL_BOUND) ? pp - d.C : zero;
  const float hm = sl_hi(e.hm), he = sl_hi(e.he), hb = sl_hi(e.hb);
  e.phi = 0.5f * (hm * hm + he * he + hb * hb);
  float r = fmaxf(fmaxf(fabsf(hm), fabsf(he)), fabsf(hb));
  if (e.phi != e.phi) r = e.phi;
  e.res = r;
}

// The multiplier step S dlam = h (Appendix B's Newton-KKT step with grad_u L = 0), the
// Schur complement assembled at the float image of the current point.  False when S is
// singular.
DF_INL bool slice_step_h(const SliceIn<float> &d, const SliceZ<float> &z, float alpha,
                         float beta, float su, float su2, float hm, float he, float hb,
                         float &dlm, float &dle, float &dlb) {
  if (alpha == 0.0f || beta == 0.0f) return false;
  float s00, s01, s02, s11, s12, s22;
  slice_schur(d, z, su, su2, sl_rcp(alpha), sl_rcp(beta), s00, s01, s02, s11, s12, s22);
  Ldl3<float> f;
  if (!ldl3_factor(s00, s01, s02, s11, s12, s22, f)) return false;
  ldl3_solve(f, (d.rows & SL_MASS) ? hm : 0.0f, (d.rows & SL_ENERGY) ? he : 0.0f,
             (d.rows & SL_BOUND) ? hb : 0.0f, dlm, dle, dlb);
  return true;
}

// Newton steps in the multipliers from z (evaluated in e) until e.res <= tol, a failure or
// `budget` steps, with the residuals and trial points in precision T and every step solved in
// float (T = df64: mixed-precision iterative refinement of the step).  First trial capped so
// that both diagonal values of W keep >= w_keep of their value, Armijo on phi.
template <class T>
DF_INL void slice_newton_h(const SliceIn<T> &d, const SliceIn<float> &d32, SliceZ<T> &z,
                           SliceH<T> &e, float tol, float c1x2, float w_keep1, bool cap,
                           int max_backtracks, int budget, SliceResult &R) {
  for (int it = 0;; ++it) {
    if (!isfinite(e.res)) { R.status = SNAP_SAMPLE_NONFINITE; return; }
    if (e.res <= tol) { R.status = SNAP_SAMPLE_OK; return; }
    if (it >= budget) { R.status = SNAP_SAMPLE_MAXITER; return; }
    const SliceZ<float> zf{sl_hi(z.a), sl_hi(z.c), sl_hi(z.p0), sl_hi(z.ph),
                           sl_hi(z.lm), sl_hi(z.le), sl_hi(z.lb)};
    float dlm, dle, dlb;
    if (!slice_step_h(d32, zf, sl_hi(e.alpha), sl_hi(e.beta), sl_hi(e.su), sl_hi(e.su2),
                      sl_hi(e.hm), sl_hi(e.he), sl_hi(e.hb), dlm, dle, dlb)) {
      R.status = SNAP_SAMPLE_SINGULAR;
      return;
    }
    float t = 1.0f;
    if (cap) {
      const float da = 2.0f * d32.dx * dle, db = da + 2.0f * dlb;
      const float al = sl_hi(e.alpha), be = sl_hi(e.beta);
      if (al > 0.0f && da < 0.0f) t = fminf(t, w_keep1 * al * df_rcp(-da));
      if (be > 0.0f && db < 0.0f) t = fminf(t, w_keep1 * be * df_rcp(-db));
    }
    int nb = 0;
    bool accepted = false;
    SliceZ<T> zt;
    SliceH<T> et;
    for (;;) {
      const T tt = sl_cast<T, float>(t);
      zt.lm = z.lm + tt * sl_cast<T, float>(dlm);
      zt.le = z.le + tt * sl_cast<T, float>(dle);
      zt.lb = z.lb + tt * sl_cast<T, float>(dlb);
      slice_stationary(d, zt);
      slice_eval_h(d, zt, et);
      if (et.phi <= (1.0f - c1x2 * t) * e.phi) { accepted = true; break; }
      if (nb >= max_backtracks) break;
      nb++;
      t *= 0.5f;
    }
    R.backtracks += nb;
    if (!accepted) { R.status = SNAP_SAMPLE_LINESEARCH; return; }
    z = zt;
    e = et;
    R.iters++;
  }
}

// Polishing step after the stopping test: the test bounds ||h||, and the multipliers only
// through the conditioning of S, which is large on slices whose boundary circle is nearly
// degenerate (c_k ~ 1e-6: S ~ 1e7 there).  One more Newton step on the multipliers leaves them
// at the rounding level.  S is first factored in float at the float image of z: when its
// pivots over the rows present are within a factor 1e3 of each other and its multipliers l are
// below 1e2 (S well conditioned), the multipliers are already within ~1e3 ||F|| of converged
// and no step is taken; otherwise S is assembled, factored and solved in double-float, and
// the step is kept when it does not increase ||h||_inf and leaves W positive.
DF_INL void slice_polish(const SliceIn<df64> &d, const SliceIn<float> &d32, SliceZ<df64> &z,
                         SliceH<df64> &e) {
  const df64 zero(0.0f, 0.0f), one(1.0f, 0.0f);
  if (!(e.alpha > zero) || !(e.beta > zero)) return;
  const bool hm = d.rows & SL_MASS, he = d.rows & SL_ENERGY, hb = d.rows & SL_BOUND;
  const SliceZ<float> zf{z.a.hi, z.c.hi, z.p0.hi, z.ph.hi, z.lm.hi, z.le.hi, z.lb.hi};
  float f00, f01, f02, f11, f12, f22;
  slice_schur(d32, zf, e.su.hi, e.su2.hi, df_rcp(e.alpha.hi), df_rcp(e.beta.hi), f00, f01, f02,
              f11, f12, f22);
  Ldl3<float> ff;
  bool cheap = false;
  if (ldl3_factor(f00, f01, f02, f11, f12, f22, ff)) {
    const float a0 = fabsf(ff.d0), a1 = fabsf(ff.d1), a2 = fabsf(ff.d2);
    const float dmax = fmaxf(hm ? a0 : 0.0f, fmaxf(he ? a1 : 0.0f, hb ? a2 : 0.0f));
    const float dmin = fminf(hm ? a0 : INFINITY, fminf(he ? a1 : INFINITY, hb ? a2 : INFINITY));
    const float lmax = fmaxf(fabsf(ff.l10), fmaxf(fabsf(ff.l20), fabsf(ff.l21)));
    cheap = dmax <= 1e3f * dmin && lmax <= 1e2f;
  }
  // a well-conditioned S: the multipliers at the stopping point are within cond(S) ||F|| of
  // converged, far inside their tolerance, and the step is not taken
  if (cheap) return;
  df64 dlm, dle, dlb;
  {
    df64 s00, s01, s02, s11, s12, s22;
    slice_schur(d, z, e.su, e.su2, one / e.alpha, one / e.beta, s00, s01, s02, s11, s12, s22);
    Ldl3<df64> f;
    if (!ldl3_factor(s00, s01, s02, s11, s12, s22, f)) return;
    ldl3_solve(f, hm ? e.hm : zero, he ? e.he : zero, hb ? e.hb : zero, dlm, dle, dlb);
  }
  SliceZ<df64> zt;
  zt.lm = z.lm + dlm;
  zt.le = z.le + dle;
  zt.lb = z.lb + dlb;
  slice_stationary(d, zt);
  SliceH<df64> et;
  slice_eval_h(d, zt, et);
  if (et.res <= e.res && et.alpha > zero && et.beta > zero) {
    z = zt;
    e = et;
  }
}

// The full residual (grad_u L included) at z from the row residuals h already evaluated there
// (the same values slice_eval forms): the gradient coefficients P, Q, g0, gh in double-float,
// phi and ||F||_inf from their float images.
DF_INL void slice_eval_from_h(const SliceIn<df64> &d, const SliceZ<df64> &z,
                              const SliceH<df64> &h, SliceEval<df64> &e) {
  const df64 one(1.0f, 0.0f);
  e.alpha = h.alpha;
  e.beta = h.beta;
  e.su = h.su;
  e.su2 = h.su2;
  e.hm = h.hm;
  e.he = h.he;
  e.hb = h.hb;
  e.P = e.alpha * z.a - one;
  e.Q = e.alpha * z.c + d.dx * z.lm;
  e.g0 = e.beta * z.p0 - d.uh0 + d.dx * z.lm;
  e.gh = e.beta * z.ph - d.uhh + d.dx * z.lm;
  const float P = e.P.hi, Q = e.Q.hi, g0 = e.g0.hi, gh = e.gh.hi;
  const float hm = e.hm.hi, he = e.he.hi, hb = e.hb.hi;
  float gi2 = P * P * d.S2.hi + 2.0f * P * Q * d.S1.hi + Q * Q * d.n.hi;
  if (gi2 < 0.0f) gi2 = 0.0f;
  const float phi = 0.5f * (gi2 + g0 * g0 + gh * gh + hm * hm + he * he + hb * hb);
  float r = fmaxf(fabsf(P * d.mx.hi + Q), fabsf(P * d.mn.hi + Q));
  r = fmaxf(r, fmaxf(fmaxf(fabsf(g0), fabsf(gh)), fmaxf(fmaxf(fabsf(hm), fabsf(he)), fabsf(hb))));
  if (phi != phi) r = phi;
  e.phi = df64(phi, 0.0f);
  e.res = df64(r, 0.0f);
}

// Start of the multiplier iteration inside the region W > 0, where the KKT point is unique
// (so the start changes the path, not the result): with mass and energy rows, the
// multipliers of the slice projection without the boundary row (hyperplane and sphere:
// u = M + rho w / ||w|| over all nx points, alpha = ||w|| / rho, lam_m = (mean - alpha M) / dx
// in the per-point scaling), and with the boundary row the lam_b that puts the two boundary
// values on the circle u_0^2 + u_h^2 = C at that lam_m (beta = |u_hat_b - dx lam_m| / sqrt(C)).
// Left at lam = 0 (u = u_hat) when any of these is not finite or leaves W positive definite.
DF_INL void slice_warm_start(const SliceIn<float> &d, SliceZ<float> &z) {
  if ((d.rows & (SL_MASS | SL_ENERGY)) != (SL_MASS | SL_ENERGY)) return;
  const float N = d.n + 2.0f;
  const float s1 = d.S1 + d.uh0 + d.uhh;
  const float s2 = d.S2 + d.uh0 * d.uh0 + d.uhh * d.uhh;
  const float mean = s1 / N;
  const float w2 = s2 - N * mean * mean;
  const float mbar = d.M / (N * d.dx);
  const float rho2 = d.E / d.dx - N * mbar * mbar;
  if (!(w2 > 0.0f && rho2 > 0.0f)) return;
  const float al = sqrtf(w2 / rho2);
  const float lm = (mean - al * mbar) / d.dx;
  const float le = (al - 1.0f) / (2.0f * d.dx);
  float lb = 0.0f;
  if ((d.rows & SL_BOUND) && d.C > 0.0f) {
    const float v0 = d.uh0 - d.dx * lm, vh = d.uhh - d.dx * lm;
    const float be = sqrtf((v0 * v0 + vh * vh) / d.C);
    if (be > 1e-3f * al && be < 1e30f) lb = 0.5f * (be - al);
  }
  if (!(al > 0.0f && isfinite(lm) && isfinite(le) && isfinite(lb))) return;
  z.lm = lm;
  z.le = le;
  z.lb = lb;
  slice_stationary(d, z);
}

// Mixed precision: float steps while they make reliable progress, then steps whose residuals
// and merit are evaluated in df64 while the step is still solved in float (iterative
// refinement of the Newton step), to o.tol_kkt.  The float phase stops when
// ||h||_inf <= max(1e-5 ||h(z0)||_inf, 1e-6 * scale) (scale = the largest magnitude among
// the slice data; float rounding puts a floor near 1e-7 * scale under ||h||), when a line
// search needs more than 8 halvings (the float merit is then at its rounding floor), or when
// only 8 steps of the iteration budget are left.  dd holds the inputs in df64; the result z is
// returned in df64 and e is the full evaluation (grad_u L included) at it.
DF_INL SliceResult slice_solve_mixed(const SliceIn<df64> &dd, SliceZ<df64> &z,
                                     SliceEval<df64> &e, const SolverOpts &o,
                                     const SliceOptsT<float> &sf, const SliceOptsT<df64> &sd) {
  (void)sd;
  SliceResult R{0, 0, SNAP_SAMPLE_OK, 0};
  SliceIn<float> d32;
  d32.S1 = dd.S1.hi; d32.S2 = dd.S2.hi; d32.mx = dd.mx.hi; d32.mn = dd.mn.hi;
  d32.uh0 = dd.uh0.hi; d32.uhh = dd.uhh.hi; d32.n = dd.n.hi; d32.dx = dd.dx.hi;
  d32.M = dd.M.hi; d32.E = dd.E.hi; d32.C = dd.C.hi;
  d32.rows = dd.rows;
  d32.nint = dd.nint;
  const float c1x2 = sf.c1x2, wk1 = sf.w_keep1;
  SliceZ<float> z32{z.a.hi, z.c.hi, z.p0.hi, z.ph.hi, z.lm.hi, z.le.hi, z.lb.hi};
  slice_warm_start(d32, z32);
  SliceH<float> e32;
  slice_eval_h(d32, z32, e32);
  if (isfinite(e32.res)) {
    float scale = fmaxf(fmaxf(fabsf(d32.mx), fabsf(d32.mn)), fmaxf(fabsf(d32.uh0), fabsf(d32.uhh)));
    scale = fmaxf(scale, fmaxf(fabsf(d32.M), sqrtf(fabsf(d32.E) + fabsf(d32.C))));
    const float tol32 = fmaxf(fmaxf(1e-5f * e32.res, 1e-6f * scale), sf.tol);
    const int budget32 = o.max_iter > 16 ? o.max_iter - 8 : o.max_iter / 2;
    slice_newton_h<float>(d32, d32, z32, e32, tol32, c1x2, wk1, sf.cap,
                          o.max_backtracks < 8 ? o.max_backtracks : 8, budget32, R);
    if (R.status != SNAP_SAMPLE_NONFINITE) {
      z.lm = df_from_float(z32.lm); z.le = df_from_float(z32.le); z.lb = df_from_float(z32.lb);
    }
  }
  R.status = SNAP_SAMPLE_OK;
  slice_stationary(dd, z);
  SliceH<df64> eh;
  slice_eval_h(dd, z, eh);
  slice_newton_h<df64>(dd, d32, z, eh, sf.tol, c1x2, wk1, sf.cap, o.max_backtracks,
                       o.max_iter - R.iters, R);
  if (R.status == SNAP_SAMPLE_OK) slice_polish(dd, d32, z, eh);
  // the full residual (grad_u L included) at the returned point
  slice_eval_from_h(dd, z, eh, e);
  if (R.status == SNAP_SAMPLE_OK && !(e.res <= sd.tol)) R.status = SNAP_SAMPLE_MAXITER;
  if (R.status == SNAP_SAMPLE_OK && !(e.alpha > df64(0.0f, 0.0f) && e.beta > df64(0.0f, 0.0f))) {
    // W not positive definite: second-order check by the inertia of K
    SliceZ<float> zf{z.a.hi, z.c.hi, z.p0.hi, z.ph.hi, z.lm.hi, z.le.hi, z.lb.hi};
    SliceEval<float> ef;
    slice_eval(d32, zf, ef);
    if (!slice_sosc(d32, zf, ef)) R.status = SNAP_SAMPLE_NOT_MINIMUM;
  }
  return R;
}
