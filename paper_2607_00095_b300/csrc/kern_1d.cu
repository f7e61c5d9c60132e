// 1-D families A/B: forward projection, per-sample statistics, constraint residual and the
// implicit-function adjoint.  All arithmetic FP64.
//
// Work decomposition.  Every (sample b, slice k) pair is an independent block of the
// projection (the constraint graph splits by time slice: each row touches one slice,
// "Jacobian Structure"); slice k = 0 carries the IC rows, slices k >= 1 the mass / energy /
// boundary rows.  Slices are numbered s = b * nt + k, so a run of consecutive slices is one
// contiguous stretch of u_hat in HBM.
//
// Moment path (u0 = u_hat): a warp owns a tile of 32 consecutive slices.  Loads are done by
// groups of 8 lanes per slice (4 slices per warp instruction, 16-byte loads, 128 contiguous
// bytes per group), the interior moments are reduced inside each group with three
// butterfly steps, and then every lane owns one slice of the tile and runs that slice's
// Newton-KKT iteration in registers (slice_newton.cuh).  The write-back re-reads u_hat
// (an L2 hit: the tile was read microseconds earlier) and stores u = a u_hat + c.
//
// General path (any u0): one warp per slice, NPL values per lane in registers, warp-wide
// reductions for every sum of the Newton-KKT step.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>


#include "sample_1d.cuh"
#include "slice_newton.cuh"
#include "snap_internal.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

__device__ __forceinline__ double nan_max(double a, double b) {
  // max that propagates NaN
  return (a < b || b != b) ? b : a;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nan_max(v, __shfl_xor_sync(FULL, v, o));
  return v;
}

__device__ __forceinline__ double energy_target(const Geom1D &g, const SampleDerived &sd,
                                                double r, int k) {
  const double t = (double)k / (double)(g.nt - 1);
  const double e = sd.E0 * exp(-r * t);
  const double fl = sd.M * sd.M + g.energy_floor;
  return e >= fl ? e : fl;
}

// ---------------------------------------------------------------------------------------
// A1: per-sample derived parameters M = dx sum g, E0 = dx sum g^2 and the residual of the
// t = 0 rows that the IC rows imply (left out of the solve).  One warp per sample.
// ---------------------------------------------------------------------------------------
__global__ void k1d_params(Geom1D g, int B, const double *__restrict__ params,
                           SampleDerived *__restrict__ sd, const double *__restrict__ ic_uh,
                           double *__restrict__ ic_u, double *__restrict__ ic_lam,
                           BlockStat *__restrict__ ic_bst, double tol_kkt,
                           double *__restrict__ bwd_gh, BwdContrib *__restrict__ bwd_contrib,
                           double *__restrict__ bwd_gp, const snap_stats *__restrict__ bwd_st) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  // launched as a programmatic dependent of the stream's previous kernel: wait for it to
  // complete before touching memory; only then may this kernel's own dependent start (it
  // reads its inputs before its own wait, so every kernel before this one must be complete)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (warp >= B) return;
  const double *pg = params + (size_t)warp * g.n_params;
  const SampleDerived d = s1_derive(g, pg, lane);
  if (lane == 0) sd[warp] = d;
  if (ic_u)
    s1_ic_forward(g, pg, ic_uh + (size_t)warp * g.n_vars, ic_u + (size_t)warp * g.n_vars,
                  ic_lam + (size_t)warp * g.n_rows, ic_bst + (size_t)warp * g.nt, d.h0_inf,
                  tol_kkt, lane);
  if (bwd_gh) {
    // adjoint on the IC block: K = [I I; I 0] -> a = 0 (b_IC = gbar enters dL/dg later)
    const bool bad = bwd_st && bwd_st[warp].status != SNAP_SAMPLE_OK;
    double *out = bwd_gh + (size_t)warp * g.n_vars;
    for (int i = lane; i < g.nx; i += 32) out[i] = bad ? NAN : 0.0;
    if (lane == 0) {
      bwd_contrib[(size_t)warp * g.nt] = BwdContrib{0.0, 0.0, 0.0, 0.0};
      if (bwd_gp && (g.rows & SL_BOUND)) bwd_gp[(size_t)warp * g.n_params + g.p_c] = bad ? NAN : 0.0;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Per-sample reduction of the per-slice statistics (fixed order: deterministic).
// ---------------------------------------------------------------------------------------
__global__ void k_finalize_stats(int B, int nblk, const BlockStat *__restrict__ bs,
                                 const double *__restrict__ tol_h_ptr, double tol_h,
                                 snap_stats *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  // launched as a programmatic dependent of the tile kernel: wait for its statistics; the
  // next kernel (a programmatic dependent that waits before it touches memory) may then launch
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (warp >= B) return;
  (void)tol_h_ptr;
  s1_finalize<false>(bs + (size_t)warp * nblk, nblk, tol_h, out + warp, lane);
}

}  // namespace

namespace {

// Result kinds the owner lane passes to the write-back of its slice.
enum { KIND_MOMENT = 0, KIND_IC_G = 1, KIND_IC_KEEP = 2, KIND_NONE = 3 };

// ---------------------------------------------------------------------------------------
// Moment path.  Requires u0 = u_hat, nx even, u_hat / u 16-byte aligned.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
k1d_moment(Geom1D g, int B, const double *__restrict__ uh, const double *__restrict__ params,
           const SampleDerived *__restrict__ sd, double *__restrict__ u,
           double *__restrict__ lam, BlockStat *__restrict__ bst,
           SolverOpts o) {
  const int lane = threadIdx.x & 31;
  const int q = lane >> 3;        // group: slice 4*rho + q of a round
  const int r = lane & 7;         // lane within the group
  const long long total = (long long)B * g.nt;
  const long long ntiles = (total + 31) >> 5;
  const int wpb = blockDim.x >> 5;
  const int nx = g.nx, ih = g.ih;
  for (long long tile = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); tile < ntiles;
       tile += (long long)gridDim.x * wpb) {
    const long long sbase = tile << 5;
    // ---------------- phase 1: interior moments, 8 lanes per slice ----------------
    double m1 = 0.0, m2 = 0.0, mmx = -INFINITY, mmn = INFINITY;
#pragma unroll 1
    for (int rho = 0; rho < 8; ++rho) {
      const long long s = sbase + 4 * rho + q;
      double p1 = 0.0, p2 = 0.0, pmx = -INFINITY, pmn = INFINITY;
      if (s < total) {
        const int k = (int)(s % g.nt);
        const double *row = uh + (size_t)s * nx;
        if (k == 0) {
          // IC slice: max |u_hat - g| and sum (u_hat - g)^2
          const double *pg = params + (size_t)(s / g.nt) * g.n_params;
          for (int i = 2 * r; i < nx; i += 16) {
            const double2 v = *reinterpret_cast<const double2 *>(row + i);
            const double d0 = v.x - pg[i], d1 = v.y - pg[i + 1];
            p2 = fma(d0, d0, p2);
            p2 = fma(d1, d1, p2);
            pmx = nan_max(pmx, nan_max(fabs(d0), fabs(d1)));
          }
        } else {
          for (int i = 2 * r; i < nx; i += 16) {
            const double2 v = *reinterpret_cast<const double2 *>(row + i);
            const bool x0 = (i != 0) && (i != ih);
            const bool x1 = (i + 1 != ih);
            if (x0) {
              p1 += v.x;
              p2 = fma(v.x, v.x, p2);
              pmx = fmax(pmx, v.x);
              pmn = fmin(pmn, v.x);
              if (v.x != v.x) pmx = v.x;
            }
            if (x1) {
              p1 += v.y;
              p2 = fma(v.y, v.y, p2);
              pmx = fmax(pmx, v.y);
              pmn = fmin(pmn, v.y);
              if (v.y != v.y) pmx = v.y;
            }
          }
        }
      }
#pragma unroll
      for (int off = 1; off < 8; off <<= 1) {
        p1 += __shfl_xor_sync(FULL, p1, off);
        p2 += __shfl_xor_sync(FULL, p2, off);
        pmx = nan_max(pmx, __shfl_xor_sync(FULL, pmx, off));
        pmn = fmin(pmn, __shfl_xor_sync(FULL, pmn, off));
      }
      if (r == rho) { m1 = p1; m2 = p2; mmx = pmx; mmn = pmn; }
    }
    // ---------------- phase 2: one slice per lane, Newton-KKT in moment form ----------------
    const long long s = sbase + 4 * r + q;
    int kind = KIND_NONE;
    SliceZ<double> z{1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (s < total) {
      const int b = (int)(s / g.nt);
      const int k = (int)(s % g.nt);
      const double *pg = params + (size_t)b * g.n_params;
      double *lb = lam + (size_t)b * g.n_rows;
      const SampleDerived dv = sd[b];
      BlockStat st;
      if (k == 0) {
        const double res0 = mmx;   // ||F||_inf at (u_hat, 0) = max |u_hat - g|
        const bool take = !(res0 <= o.tol_kkt);
        kind = take ? KIND_IC_G : KIND_IC_KEEP;
        st.iters = take ? 1 : 0;
        st.backtracks = 0;
        st.corrections = 0;
        st.status = (res0 == res0 && !isinf(res0)) ? SNAP_SAMPLE_OK : SNAP_SAMPLE_NONFINITE;
        st.kkt_inf = take ? 0.0 : res0;
        st.h_inf = nan_max(take ? 0.0 : res0, dv.h0_inf);
        st.obj = take ? 0.5 * m2 : 0.0;
        if (g.off_mass >= 0) lb[g.off_mass] = 0.0;
        if (g.off_energy >= 0) lb[g.off_energy] = 0.0;
        if (g.off_bound >= 0) lb[g.off_bound] = 0.0;
      } else {
        kind = KIND_MOMENT;
        const double *row = uh + (size_t)s * nx;
        SliceIn<double> d;
        d.S1 = m1; d.S2 = m2; d.mx = mmx; d.mn = mmn;
        d.uh0 = row[0]; d.uhh = row[ih];
        d.n = (double)(nx - 2);
        d.nint = nx - 2;
        d.dx = g.dx;
        d.M = dv.M;
        d.E = (g.rows & SL_ENERGY) ? energy_target(g, dv, pg[g.p_rate], k) : 0.0;
        d.C = (g.rows & SL_BOUND) ? pg[g.p_c + k] : 0.0;
        d.rows = g.rows;
        z.p0 = d.uh0;
        z.ph = d.uhh;
        SliceEval<double> e;
        const bool infeasible = ((g.rows & SL_BOUND) && d.C < 0.0) ||
                                ((g.rows & SL_ENERGY) && d.E < ((g.rows & SL_MASS) ? d.M * d.M : 0.0));
        SliceResult R;
        if (infeasible) {
          slice_eval(d, z, e);
          R = SliceResult{0, 0, SNAP_SAMPLE_INFEASIBLE_PARAMS, 0};
        } else {
          R = slice_newton(d, z, e, o);
        }
        st.iters = R.iters;
        st.backtracks = R.backtracks;
        st.status = R.status;
        st.corrections = R.corrections;
        st.kkt_inf = e.res;
        st.h_inf = nan_max(nan_max(fabs(e.hm), fabs(e.he)), fabs(e.hb));
        const double am1 = z.a - 1.0;
        st.obj = 0.5 * (am1 * am1 * d.S2 + 2.0 * am1 * z.c * d.S1 + z.c * z.c * d.n +
                        (z.p0 - d.uh0) * (z.p0 - d.uh0) + (z.ph - d.uhh) * (z.ph - d.uhh));
        if (g.off_mass >= 0) lb[g.off_mass + k] = z.lm;
        if (g.off_energy >= 0) lb[g.off_energy + k] = z.le;
        if (g.off_bound >= 0) lb[g.off_bound + k] = z.lb;
      }
      bst[s] = st;
    }
    // ---------------- phase 3: write-back, 8 lanes per slice ----------------
#pragma unroll 1
    for (int rho = 0; rho < 8; ++rho) {
      const int src = 8 * q + rho;
      const double A = __shfl_sync(FULL, z.a, src);
      const double Cc = __shfl_sync(FULL, z.c, src);
      const double P0 = __shfl_sync(FULL, z.p0, src);
      const double PH = __shfl_sync(FULL, z.ph, src);
      const int kd = __shfl_sync(FULL, kind, src);
      const long long s2 = sbase + 4 * rho + q;
      if (s2 >= total || kd == KIND_NONE) continue;
      const double *row = uh + (size_t)s2 * nx;
      double *out = u + (size_t)s2 * nx;
      if (kd == KIND_MOMENT) {
        for (int i = 2 * r; i < nx; i += 16) {
          const double2 v = *reinterpret_cast<const double2 *>(row + i);
          double2 w;
          w.x = (i == 0) ? P0 : ((i == ih) ? PH : fma(A, v.x, Cc));
          w.y = (i + 1 == ih) ? PH : fma(A, v.y, Cc);
          *reinterpret_cast<double2 *>(out + i) = w;
        }
      } else {
        const int b = (int)(s2 / g.nt);
        const double *pg = params + (size_t)b * g.n_params;
        double *lb = lam + (size_t)b * g.n_rows;
        const bool take = kd == KIND_IC_G;
        for (int i = 2 * r; i < nx; i += 16) {
          const double2 v = *reinterpret_cast<const double2 *>(row + i);
          const double g0 = pg[i], g1 = pg[i + 1];
          double2 w;
          w.x = take ? g0 : v.x;
          w.y = take ? g1 : v.y;
          *reinterpret_cast<double2 *>(out + i) = w;
          lb[i] = take ? v.x - g0 : 0.0;
          lb[i + 1] = take ? v.y - g1 : 0.0;
        }
      }
    }
  }
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------------------
// General path: one warp per slice, element i = lane + 32 j held by lane in registers.
// ---------------------------------------------------------------------------------------
template <int NPL>
struct GenEval {
  double alpha, beta, su, su2, p0, ph, g0, gh, hm, he, hb, phi, res;
};

template <int NPL>
__device__ __forceinline__ double bcast_elem(const double (&X)[NPL], int idx, int lane) {
  double v = 0.0;
#pragma unroll
  for (int j = 0; j < NPL; ++j)
    if (j == (idx >> 5)) v = X[j];
  return __shfl_sync(FULL, v, idx & 31);
  (void)lane;
}

template <int NPL>
__device__ __forceinline__ void gen_eval(const Geom1D &g, const SliceIn<double> &d,
                                         const double (&U)[NPL], const double (&H)[NPL],
                                         double lm, double le, double lb, double (&G)[NPL],
                                         GenEval<NPL> &e, int lane) {
  e.alpha = 1.0 + 2.0 * g.dx * le;
  e.beta = e.alpha + 2.0 * lb;
  double su = 0.0, su2 = 0.0, g2 = 0.0, ginf = 0.0;
#pragma unroll
  for (int j = 0; j < NPL; ++j) {
    const int i = lane + 32 * j;
    G[j] = 0.0;
    if (i < g.nx) {
      const double w = (i == 0 || i == g.ih) ? e.beta : e.alpha;
      G[j] = w * U[j] - H[j] + g.dx * lm;
      su += U[j];
      su2 = fma(U[j], U[j], su2);
      g2 = fma(G[j], G[j], g2);
      ginf = nan_max(ginf, fabs(G[j]));
    }
  }
  e.su = warp_sum(su);
  e.su2 = warp_sum(su2);
  g2 = warp_sum(g2);
  ginf = warp_max(ginf);
  e.p0 = bcast_elem<NPL>(U, 0, lane);
  e.ph = bcast_elem<NPL>(U, g.ih, lane);
  e.g0 = bcast_elem<NPL>(G, 0, lane);
  e.gh = bcast_elem<NPL>(G, g.ih, lane);
  const double pp = e.p0 * e.p0 + e.ph * e.ph;
  e.hm = (d.rows & SL_MASS) ? g.dx * e.su - d.M : 0.0;
  e.he = (d.rows & SL_ENERGY) ? g.dx * e.su2 - d.E : 0.0;
  e.hb = (d.rows & SL_BOUND) ? pp - d.C : 0.0;
  e.phi = 0.5 * (g2 + e.hm * e.hm + e.he * e.he + e.hb * e.hb);
  double r = ginf;
  r = nan_max(r, fabs(e.hm));
  r = nan_max(r, fabs(e.he));
  r = nan_max(r, fabs(e.hb));
  if (e.phi != e.phi) r = e.phi;
  e.res = r;
}

// Schur complement and rhs of the general path at (U, G) with diagonal shifts w / wb.
template <int NPL>
__device__ __forceinline__ void gen_schur(const Geom1D &g, const SliceIn<double> &d,
                                          const double (&U)[NPL], const double (&G)[NPL],
                                          const GenEval<NPL> &e, double w, double wb,
                                          double &s00, double &s01, double &s02, double &s11,
                                          double &s12, double &s22, double &v0, double &v1,
                                          double &v2, int lane) {
  double suw = 0.0, su2w = 0.0, sgw = 0.0, sugw = 0.0;
  const double iw = 1.0 / w, iwb = 1.0 / wb;
#pragma unroll
  for (int j = 0; j < NPL; ++j) {
    const int i = lane + 32 * j;
    if (i < g.nx) {
      const double iwi = (i == 0 || i == g.ih) ? iwb : iw;
      suw = fma(U[j], iwi, suw);
      su2w = fma(U[j] * U[j], iwi, su2w);
      sgw = fma(G[j], iwi, sgw);
      sugw = fma(U[j] * G[j], iwi, sugw);
    }
  }
  suw = warp_sum(suw);
  su2w = warp_sum(su2w);
  sgw = warp_sum(sgw);
  sugw = warp_sum(sugw);
  const double s1w = (double)(g.nx - 2) * iw + 2.0 * iwb;
  const double pp = e.p0 * e.p0 + e.ph * e.ph, ps = e.p0 + e.ph;
  const bool hm = d.rows & SL_MASS, he = d.rows & SL_ENERGY, hb = d.rows & SL_BOUND;
  s00 = hm ? g.dx * g.dx * s1w : 1.0;
  s01 = (hm && he) ? 2.0 * g.dx * g.dx * suw : 0.0;
  s02 = (hm && hb) ? 2.0 * g.dx * ps * iwb : 0.0;
  s11 = he ? 4.0 * g.dx * g.dx * su2w : 1.0;
  s12 = (he && hb) ? 4.0 * g.dx * pp * iwb : 0.0;
  s22 = hb ? 4.0 * pp * iwb : 1.0;
  v0 = hm ? g.dx * sgw : 0.0;
  v1 = he ? 2.0 * g.dx * sugw : 0.0;
  v2 = hb ? 2.0 * (e.p0 * e.g0 + e.ph * e.gh) * iwb : 0.0;
}

template <int NPL>
__global__ void __launch_bounds__(128)
k1d_general(Geom1D g, int B, const double *__restrict__ uh, const double *__restrict__ params,
            const double *__restrict__ u0, const SampleDerived *__restrict__ sd,
            double *__restrict__ u, double *__restrict__ lam, BlockStat *__restrict__ bst,
            SolverOpts o) {
  const int lane = threadIdx.x & 31;
  const long long total = (long long)B * g.nt;
  const int wpb = blockDim.x >> 5;
  const int nx = g.nx;
  for (long long s = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); s < total;
       s += (long long)gridDim.x * wpb) {
    const int b = (int)(s / g.nt);
    const int k = (int)(s % g.nt);
    const double *row = uh + (size_t)s * nx;
    const double *row0 = (u0 ? u0 : uh) + (size_t)s * nx;
    const double *pg = params + (size_t)b * g.n_params;
    double *lb = lam + (size_t)b * g.n_rows;
    double *out = u + (size_t)s * nx;
    const SampleDerived dv = sd[b];
    double H[NPL], U[NPL];
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
      const int i = lane + 32 * j;
      H[j] = (i < nx) ? row[i] : 0.0;
      U[j] = (i < nx) ? row0[i] : 0.0;
    }
    BlockStat st;
    if (k == 0) {
      // IC block: rows u_i - g_i are linear and independent per variable; one Newton step
      // from (u0, 0) lands on u = g, lambda = u_hat - g.
      double res0 = 0.0;
#pragma unroll
      for (int j = 0; j < NPL; ++j) {
        const int i = lane + 32 * j;
        if (i < nx) res0 = nan_max(res0, nan_max(fabs(U[j] - H[j]), fabs(U[j] - pg[i])));
      }
      res0 = warp_max(res0);
      const bool take = !(res0 <= o.tol_kkt);
      double obj = 0.0, hic = 0.0;
#pragma unroll
      for (int j = 0; j < NPL; ++j) {
        const int i = lane + 32 * j;
        if (i < nx) {
          const double gi = pg[i];
          const double ui = take ? gi : U[j];
          out[i] = ui;
          lb[i] = take ? H[j] - gi : 0.0;
          obj = fma(ui - H[j], ui - H[j], obj);
          hic = nan_max(hic, fabs(ui - gi));
        }
      }
      obj = warp_sum(obj);
      hic = warp_max(hic);
      st.iters = take ? 1 : 0;
      st.backtracks = 0;
      st.corrections = 0;
      st.status = (res0 == res0 && !isinf(res0)) ? SNAP_SAMPLE_OK : SNAP_SAMPLE_NONFINITE;
      st.kkt_inf = take ? 0.0 : res0;
      st.h_inf = nan_max(hic, dv.h0_inf);
      st.obj = 0.5 * obj;
      if (lane == 0) {
        if (g.off_mass >= 0) lb[g.off_mass] = 0.0;
        if (g.off_energy >= 0) lb[g.off_energy] = 0.0;
        if (g.off_bound >= 0) lb[g.off_bound] = 0.0;
        bst[s] = st;
      }
      continue;
    }
    SliceIn<double> d;
    d.dx = g.dx;
    d.n = (double)(nx - 2);
    d.nint = nx - 2;
    d.M = dv.M;
    d.E = (g.rows & SL_ENERGY) ? energy_target(g, dv, pg[g.p_rate], k) : 0.0;
    d.C = (g.rows & SL_BOUND) ? pg[g.p_c + k] : 0.0;
    d.rows = g.rows;
    const int m_present = ((g.rows & SL_MASS) != 0) + ((g.rows & SL_ENERGY) != 0) +
                          ((g.rows & SL_BOUND) != 0);
    double lm = 0.0, le = 0.0, lbd = 0.0;
    // an explicit start point takes the primal-dual iteration; the start u_hat keeps the
    // iterates stationary in u (u = argmin L(., lambda)), as the moment paths do
    const bool restore = (u0 == nullptr);
    double G[NPL];
    GenEval<NPL> e;
    gen_eval<NPL>(g, d, U, H, lm, le, lbd, G, e, lane);
    int iters = 0, nbt = 0, ncorr = 0, status = SNAP_SAMPLE_OK;
    const bool infeasible = ((g.rows & SL_BOUND) && d.C < 0.0) ||
                            ((g.rows & SL_ENERGY) && d.E < ((g.rows & SL_MASS) ? d.M * d.M : 0.0));
    if (infeasible) status = SNAP_SAMPLE_INFEASIBLE_PARAMS;
    // polish: after the stopping test one more full Newton step, kept when ||F||_inf does not
    // increase (the multipliers of ill-conditioned slices to the rounding level)
    bool polish = false;
    for (int it = 0; !infeasible; ++it) {
      if (!(e.res == e.res) || isinf(e.res)) { status = SNAP_SAMPLE_NONFINITE; break; }
      if (e.res <= o.tol_kkt) {
        status = SNAP_SAMPLE_OK;
        if (polish) break;
        polish = true;
      } else if (polish) {
        break;
      }
      if (!polish && it >= o.max_iter) { status = SNAP_SAMPLE_MAXITER; break; }
      double delta = 0.0, w = e.alpha, wb = e.beta;
      double s00, s01, s02, s11, s12, s22, v0, v1, v2;
      Ldl3<double> f;
      bool ok = false;
      for (int corr = 0; corr <= o.max_corrections; ++corr) {
        w = e.alpha + delta;
        wb = e.beta + delta;
        gen_schur<NPL>(g, d, U, G, e, w, wb, s00, s01, s02, s11, s12, s22, v0, v1, v2, lane);
        if (w != 0.0 && wb != 0.0 && ldl3_factor(s00, s01, s02, s11, s12, s22, f) &&
            (o.max_corrections == 0 || slice_inertia_ok(f, w, wb, nx - 2, m_present, 3 - m_present))) {
          ok = true;
          break;
        }
        delta = (delta == 0.0) ? o.delta0 : delta * 10.0;
        ncorr++;
      }
      if (!ok) {
        if (!polish) status = SNAP_SAMPLE_SINGULAR;
        break;
      }
      double dlm, dle, dlb;
      ldl3_solve(f, (g.rows & SL_MASS) ? e.hm - v0 : 0.0, (g.rows & SL_ENERGY) ? e.he - v1 : 0.0,
                 (g.rows & SL_BOUND) ? e.hb - v2 : 0.0, dlm, dle, dlb);
      double dU[NPL];
#pragma unroll
      for (int j = 0; j < NPL; ++j) {
        const int i = lane + 32 * j;
        const bool bd = (i == 0 || i == g.ih);
        const double wi = bd ? wb : w;
        dU[j] = -(G[j] + g.dx * dlm + 2.0 * g.dx * U[j] * dle + (bd ? 2.0 * U[j] * dlb : 0.0)) / wi;
        if (i >= nx) dU[j] = 0.0;
      }
      double t = 1.0;
      if (o.w_keep > 0.0 && !polish) {
        const double da = (g.rows & SL_ENERGY) ? 2.0 * g.dx * dle : 0.0;
        const double db = da + 2.0 * dlb;
        if (e.alpha > 0.0 && da < 0.0) t = fmin(t, (1.0 - o.w_keep) * e.alpha / (-da));
        if (e.beta > 0.0 && db < 0.0) t = fmin(t, (1.0 - o.w_keep) * e.beta / (-db));
      }
      int nb = 0;
      bool accepted = false;
      double Ut[NPL], Gt[NPL];
      GenEval<NPL> et;
      for (;;) {
        if (restore) {
          // start at u_hat: trial points keep grad_u L = 0, u = (u_hat - dx lam_m 1) / W
          const double lmt = lm + t * dlm;
          const double alt = 1.0 + 2.0 * g.dx * (le + t * dle);
          const double bet = alt + 2.0 * (lbd + t * dlb);
#pragma unroll
          for (int j = 0; j < NPL; ++j) {
            const int i = lane + 32 * j;
            Ut[j] = (i < nx) ? (H[j] - g.dx * lmt) / ((i == 0 || i == g.ih) ? bet : alt) : 0.0;
          }
        } else {
#pragma unroll
          for (int j = 0; j < NPL; ++j) Ut[j] = U[j] + t * dU[j];
        }
        gen_eval<NPL>(g, d, Ut, H, lm + t * dlm, le + t * dle, lbd + t * dlb, Gt, et, lane);
        if (polish) {
          accepted = et.res <= e.res && et.alpha > 0.0 && et.beta > 0.0;
          break;
        }
        if (et.phi <= (1.0 - 2.0 * o.c1 * t) * e.phi) { accepted = true; break; }
        if (nb >= o.max_backtracks) break;
        nb++;
        t *= 0.5;
      }
      nbt += nb;
      if (!accepted) {
        if (!polish) status = SNAP_SAMPLE_LINESEARCH;
        break;
      }
#pragma unroll
      for (int j = 0; j < NPL; ++j) { U[j] = Ut[j]; G[j] = Gt[j]; }
      lm += t * dlm;
      le += t * dle;
      lbd += t * dlb;
      e = et;
      if (!polish) iters = it + 1;     // the polishing step is not counted
    }
    if (status == SNAP_SAMPLE_OK) {
      // second-order sufficient condition at the converged point
      double s00, s01, s02, s11, s12, s22, v0, v1, v2;
      gen_schur<NPL>(g, d, U, G, e, e.alpha, e.beta, s00, s01, s02, s11, s12, s22, v0, v1, v2, lane);
      Ldl3<double> f;
      if (!ldl3_factor(s00, s01, s02, s11, s12, s22, f) ||
          !slice_inertia_ok(f, e.alpha, e.beta, nx - 2, m_present, 3 - m_present))
        status = SNAP_SAMPLE_NOT_MINIMUM;
    }
    double obj = 0.0;
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
      const int i = lane + 32 * j;
      if (i < nx) {
        out[i] = U[j];
        obj = fma(U[j] - H[j], U[j] - H[j], obj);
      }
    }
    obj = warp_sum(obj);
    if (lane == 0) {
      st.iters = iters;
      st.backtracks = nbt;
      st.corrections = ncorr;
      st.status = status;
      st.kkt_inf = e.res;
      st.h_inf = nan_max(nan_max(fabs(e.hm), fabs(e.he)), fabs(e.hb));
      st.obj = 0.5 * obj;
      bst[s] = st;
      if (g.off_mass >= 0) lb[g.off_mass + k] = lm;
      if (g.off_energy >= 0) lb[g.off_energy + k] = le;
      if (g.off_bound >= 0) lb[g.off_bound + k] = lbd;
    }
  }
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------------------
// Constraint residual h(u) of every nominal row; one warp per slice.
// ---------------------------------------------------------------------------------------
template <int NPL>
__global__ void __launch_bounds__(128)
k1d_residual(Geom1D g, int B, const double *__restrict__ u, const double *__restrict__ params,
             const SampleDerived *__restrict__ sd, double *__restrict__ h,
             double *__restrict__ smax) {
  const int lane = threadIdx.x & 31;
  const long long total = (long long)B * g.nt;
  const int wpb = blockDim.x >> 5;
  for (long long s = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); s < total;
       s += (long long)gridDim.x * wpb) {
    const int b = (int)(s / g.nt);
    const int k = (int)(s % g.nt);
    const double *row = u + (size_t)s * g.nx;
    const double *pg = params + (size_t)b * g.n_params;
    double *hb = h ? h + (size_t)b * g.n_rows : nullptr;
    const SampleDerived dv = sd[b];
    double su = 0.0, su2 = 0.0, mx = 0.0, U[NPL];
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
      const int i = lane + 32 * j;
      U[j] = (i < g.nx) ? row[i] : 0.0;
      su += U[j];
      su2 = fma(U[j], U[j], su2);
      if (k == 0 && i < g.nx) {
        const double r = U[j] - pg[i];
        if (hb) hb[i] = r;
        mx = nan_max(mx, fabs(r));
      }
    }
    su = warp_sum(su);
    su2 = warp_sum(su2);
    mx = warp_max(mx);
    const double p0 = bcast_elem<NPL>(U, 0, lane);
    const double ph = bcast_elem<NPL>(U, g.ih, lane);
    if (lane == 0) {
      if (g.rows & SL_MASS) {
        const double r = g.dx * su - dv.M;
        if (hb) hb[g.off_mass + k] = r;
        mx = nan_max(mx, fabs(r));
      }
      if (g.rows & SL_ENERGY) {
        const double r = g.dx * su2 - energy_target(g, dv, pg[g.p_rate], k);
        if (hb) hb[g.off_energy + k] = r;
        mx = nan_max(mx, fabs(r));
      }
      if (g.rows & SL_BOUND) {
        const double r = p0 * p0 + ph * ph - pg[g.p_c + k];
        if (hb) hb[g.off_bound + k] = r;
        mx = nan_max(mx, fabs(r));
      }
      smax[s] = mx;
    }
  }
}

__global__ void k_rowmax(int B, int nblk, const double *__restrict__ smax,
                         double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= B) return;
  double m = 0.0;
  for (int k = lane; k < nblk; k += 32) m = nan_max(m, smax[(size_t)warp * nblk + k]);
  m = warp_max(m);
  if (lane == 0) out[warp] = m;
}

// Per-sample part of dL/dtheta: g (through the IC rows, M and E0) and r.
__global__ void k1d_backward_params(Geom1D g, int B, const double *__restrict__ gu,
                                    const double *__restrict__ params,
                                    const snap_stats *__restrict__ fst,
                                    const SampleDerived *__restrict__ sd,
                                    const BwdContrib *__restrict__ contrib,
                                    double *__restrict__ gp) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  // launched as a programmatic dependent of the adjoint tile kernel: wait for its output
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (warp >= B) return;
  const bool bad = fst && fst[warp].status != SNAP_SAMPLE_OK;
  s1_param_grad<false>(g, gu + (size_t)warp * g.n_vars, params + (size_t)warp * g.n_params,
                       sd[warp].M, contrib + (size_t)warp * g.nt, bad,
                       gp + (size_t)warp * g.n_params, lane);
}

template <int NPL>
void launch_general(const Geom1D &g, int B, const double *uh, const double *params,
                    const double *u0, const SampleDerived *sd, double *u, double *lam,
                    BlockStat *bst, const SolverOpts &o, cudaStream_t s) {
  const long long total = (long long)B * g.nt;
  const int threads = 128;
  long long blocks = (total + 3) / 4;
  if (blocks > 148LL * 64) blocks = 148LL * 64;
  k1d_general<NPL><<<(int)blocks, threads, 0, s>>>(g, B, uh, params, u0, sd, u, lam, bst, o);
}

template <int NPL>
void launch_residual(const Geom1D &g, int B, const double *u, const double *params,
                     const SampleDerived *sd, double *h, double *smax, cudaStream_t s) {
  const long long total = (long long)B * g.nt;
  long long blocks = (total + 3) / 4;
  if (blocks > 148LL * 64) blocks = 148LL * 64;
  k1d_residual<NPL><<<(int)blocks, 128, 0, s>>>(g, B, u, params, sd, h, smax);
}

#define SNAP_DISPATCH_NPL(nx, FN, ...)                      \
  do {                                                      \
    const int npl_ = ((nx) + 31) / 32;                      \
    if (npl_ <= 1) FN<1>(__VA_ARGS__);                      \
    else if (npl_ <= 2) FN<2>(__VA_ARGS__);                 \
    else if (npl_ <= 4) FN<4>(__VA_ARGS__);                 \
    else if (npl_ <= 8) FN<8>(__VA_ARGS__);                 \
    else FN<16>(__VA_ARGS__);                               \
  } while (0)

struct Ws1D {
  SampleDerived *sd;
  BlockStat *bst;
  BwdContrib *contrib;
  double *smax;
};

Ws1D carve_1d(const snap_problem *p, int B, void *ws) {
  char *c = (char *)ws;
  const size_t nblk = (size_t)B * p->g1.nt;
  Ws1D w;
  w.sd = (SampleDerived *)c;
  c += snap_align256(sizeof(SampleDerived) * (size_t)B);
  w.bst = (BlockStat *)c;
  c += snap_align256(sizeof(BlockStat) * nblk);
  w.contrib = (BwdContrib *)c;
  c += snap_align256(sizeof(BwdContrib) * nblk);
  w.smax = (double *)c;
  return w;
}

}  // namespace

size_t ws_bytes_1d(const snap_problem *p, int B) {
  const size_t nblk = (size_t)B * p->g1.nt;
  return snap_align256(sizeof(SampleDerived) * (size_t)B) + snap_align256(sizeof(BlockStat) * nblk) +
         snap_align256(sizeof(BwdContrib) * nblk) + snap_align256(sizeof(double) * nblk);
}

static int warps_blocks(int nwarps) { return (nwarps * 32 + 127) / 128; }

// k1d_params as a programmatic dependent of the stream's previous kernel: its launch overlaps
// that kernel's tail, and it waits for that kernel's completion before its first access
static void launch_params(const Geom1D &g, int B, const double *params, SampleDerived *sd,
                          const double *ic_uh, double *ic_u, double *ic_lam, BlockStat *ic_bst,
                          double tol_kkt, double *bwd_gh, BwdContrib *bwd_contrib,
                          double *bwd_gp, const snap_stats *bwd_st, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)warps_blocks(B));
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k1d_params, g, B, params, sd, ic_uh, ic_u, ic_lam, ic_bst, tol_kkt,
                     bwd_gh, bwd_contrib, bwd_gp, bwd_st);
}


cudaError_t launch_1d_forward(const snap_problem *p, int B, const double *u_hat,
                              const double *params, const double *u0, double *u, double *lambda,
                              snap_stats *stats, const SolverOpts &o, int path,
                              void *ws, cudaStream_t s) {
  const Geom1D &g = p->g1;
  Ws1D w = carve_1d(p, B, ws);
  int launches = 0;
  const bool mixed = path == SNAP_PATH_MIXED;
  launch_params(g, B, params, w.sd, u_hat, mixed ? u : nullptr, lambda, w.bst, o.tol_kkt,
                nullptr, nullptr, nullptr, nullptr, s);
  launches++;
  if (mixed) {
    const int pid = snap_prof_begin(s, "k1d_mixed");
    launch_1d_mixed(g, B, u_hat, params, w.sd, u, lambda, w.bst, o, 0, s);
    snap_prof_end(s, pid);
  } else if (path == SNAP_PATH_MOMENT) {
    const long long ntiles = ((long long)B * g.nt + 31) / 32;
    long long blocks = (ntiles + 3) / 4;
    if (blocks > 148LL * 64) blocks = 148LL * 64;
    const int pid = snap_prof_begin(s, "k1d_moment");
    k1d_moment<<<(int)blocks, 128, 0, s>>>(g, B, u_hat, params, w.sd, u, lambda, w.bst,
                                           o);
    snap_prof_end(s, pid);
  } else {
    const int pid = snap_prof_begin(s, "k1d_general");
    SNAP_DISPATCH_NPL(g.nx, launch_general, g, B, u_hat, params, u0, w.sd, u, lambda, w.bst,
                      o, s);
    snap_prof_end(s, pid);
  }
  launches++;
  if (stats) {
    launch_finalize_stats(B, g.nt, w.bst, o.tol_h, stats, s);
    launches++;
  }
  snap_note_launch(launches);
  return cudaGetLastError();
}

cudaError_t launch_1d_residual(const snap_problem *p, int B, const double *u,
                               const double *params, double *h, double *h_inf, void *ws,
                               cudaStream_t s) {
  const Geom1D &g = p->g1;
  Ws1D w = carve_1d(p, B, ws);
  launch_params(g, B, params, w.sd, nullptr, nullptr, nullptr, nullptr, 0.0, nullptr, nullptr,
                nullptr, nullptr, s);
  SNAP_DISPATCH_NPL(g.nx, launch_residual, g, B, u, params, w.sd, h, w.smax, s);
  int launches = 2;
  if (h_inf) {
    k_rowmax<<<warps_blocks(B), 128, 0, s>>>(B, g.nt, w.smax, h_inf);
    launches++;
  }
  snap_note_launch(launches);
  return cudaGetLastError();
}

cudaError_t launch_1d_backward(const snap_problem *p, int B, const double *grad_u,
                               const double *u, const double *lambda, const double *params,
                               const snap_stats *stats, double *grad_u_hat,
                               double *grad_params, void *ws, cudaStream_t s) {
  const Geom1D &g = p->g1;
  Ws1D w = carve_1d(p, B, ws);
  launch_params(g, B, params, w.sd, nullptr, nullptr, nullptr, nullptr, 0.0, grad_u_hat,
                w.contrib, grad_params, stats, s);
  const int pid = snap_prof_begin(s, "k1d_bwd_mixed");
  launch_1d_bwd_mixed(g, B, grad_u, u, lambda, params, stats, w.sd,
                      grad_u_hat, grad_params, w.contrib, s);
  snap_prof_end(s, pid);
  int launches = 2;
  if (grad_params) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)warps_blocks(B));
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k1d_backward_params, g, B, grad_u, params, stats,
                       (const SampleDerived *)w.sd, (const BwdContrib *)w.contrib, grad_params);
    launches++;
  }
  snap_note_launch(launches);
  return cudaGetLastError();
}

void launch_finalize_stats(int B, int nblk, const BlockStat *bst, double tol_h, snap_stats *stats,
                           cudaStream_t s) {
  // programmatic dependent of the kernel before it (k_finalize_stats waits for its completion)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)warps_blocks(B));
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_finalize_stats, B, nblk, bst, (const double *)nullptr, tol_h, stats);
}
