// 1-D families A/B, moment path with the arithmetic spread over the SM's pipes.
//
// On B300 the FP64 pipe retires ~0.46 T FMA/s against ~34 T FP32 FMA/s, so one FP64
// instruction per element already costs as much time as streaming the element through HBM.
// This kernel therefore keeps FP64 for the one operation per element that needs it (the
// write-back u_i = a u_hat_i + c) and moves everything else to the FP32 / integer pipes:
//
//   phase 1  (4 lanes per slice, 8 slices per warp instruction, 16-byte loads): every
//            u_hat_i is split into a float pair hi + lo with integer operations and one
//            conversion (|u_hat - hi - lo| <= 2^-48 |u_hat|), and the interior moments
//            S1 = sum u_hat_i, S2 = sum u_hat_i^2 are accumulated in double-float
//            (error-free TwoSum / TwoProd), reduced across the 4 lanes with two butterfly
//            steps;
//   phase 2  (one slice per lane): the slice's Newton-KKT iteration in moment form,
//            first in float, then in double-float to the FP64 stopping tolerance
//            (slice_solve_mixed); E_k = E0 q^k with q = exp(-r dt) by binary powering in
//            double-float;
//   phase 3  (4 lanes per slice): u = fma(a, u_hat, c) in FP64, 16-byte stores.
//
// The IC slices (k = 0) are solved by the per-sample prepare kernel (k1d_params), a full
// warp per slice, and skipped here.
//
// Launch overlap: the kernel is launched as a programmatic dependent of k1d_params.  Phase 1
// reads only u_hat, so it runs while k1d_params is still working; the first read of the
// per-sample values (phase 2) waits for k1d_params to complete (griddepcontrol.wait).  The
// kernel in turn lets the statistics kernel launch early (it waits the same way).
//
// A slice whose values leave the range of the float-pair representation (|u_hat| outside
// [2^-74, 2^57], or non-finite) falls back to FP64 moments and the FP64 iteration.
//
// The uneven-batch kernel runs the same three phases from tile_1d.cuh (slices located through
// a per-instance pointer table).  This kernel keeps its own copy of the tile inside its
// grid-stride loop: the same code moved into an inlined function measured 6-7 % slower here
// (95 against 89 us per B=512 Burgers launch on B300), so the hot path stays as written.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "slice_newton.cuh"
#include "snap_internal.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;

enum { KIND_MOMENT = 0, KIND_NONE = 3 };

__device__ __forceinline__ double nan_max(double a, double b) { return (a < b || b != b) ? b : a; }

// x^k for k >= 0 by binary powering in double-float
__device__ __forceinline__ df64 df_pow(df64 x, int k) {
  df64 r(1.0f, 0.0f);
  while (k > 0) {
    if (k & 1) r = r * x;
    x = x * x;
    k >>= 1;
  }
  return r;
}

__device__ __forceinline__ df64 shfl_df(df64 v, int off) {
  return df64(__shfl_xor_sync(FULL, v.hi, off), __shfl_xor_sync(FULL, v.lo, off));
}

__global__ void __launch_bounds__(64, 8)
k1d_mixed(Geom1D g, int B, const double *__restrict__ uh, const double *__restrict__ params,
          const SampleDerived *__restrict__ sd, double *__restrict__ u,
          double *__restrict__ lam, BlockStat *__restrict__ bst,
          SliceFactor *__restrict__ cache, SolverOpts o) {
  const int lane = threadIdx.x & 31;
  const int q = lane >> 2;        // group: slice 8*rho + q of round rho
  const int r = lane & 3;         // lane within the group
  const long long total = (long long)B * g.nt;
  const long long ntiles = (total + 31) >> 5;
  const int wpb = blockDim.x >> 5;
  const int nx = g.nx, ih = g.ih;
  const SliceOptsT<float> so_f = slice_opts<float>(o, o.tol_kkt);
  const SliceOptsT<df64> so_d = slice_opts<df64>(o, o.tol_kkt);
  const df64 dxd(g.dx);
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  for (long long tile = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); tile < ntiles;
       tile += (long long)gridDim.x * wpb) {
    const long long sbase = tile << 5;
    // ---------------- phase 1 ----------------
    {
      // pull the tile (32 consecutive slices, contiguous in HBM) into L2 ahead of the loads
      const long long s_end = (sbase + 32 < total) ? sbase + 32 : total;
      const char *t0 = reinterpret_cast<const char *>(uh + (size_t)sbase * nx);
      const size_t bytes = (size_t)(s_end - sbase) * nx * sizeof(double);
      for (size_t off = (size_t)lane * 128; off < bytes; off += 32 * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(t0 + off));
    }
    df64 m1(0.0f, 0.0f), m2(0.0f, 0.0f);
    float mmx = -INFINITY, mmn = INFINITY;
    int mok = 1;
#pragma unroll 1
    for (int rho = 0; rho < 4; ++rho) {
      const long long s = sbase + 8 * rho + q;
      float s1h = 0.0f, s1e = 0.0f, s2h = 0.0f, s2e = 0.0f;
      float pmx = -INFINITY, pmn = INFINITY;
      int ok = 1;
      if (s < total) {
        const int k = (int)(s % g.nt);
        const double *row = uh + (size_t)s * nx;
        if (k == 0) {
          // the IC slice is handled by the per-sample prepare kernel
        } else {
          // CH independent 16-byte loads in flight per lane, then the accumulation
          constexpr int CH = 16;
          for (int i0 = 2 * r; i0 < nx; i0 += 8 * CH) {
            double2 v[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
              const int i = i0 + 8 * c;
              v[c] = (i < nx) ? __ldg(reinterpret_cast<const double2 *>(row + i)) : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
              const int i = i0 + 8 * c;
              if (i >= nx) break;
              float h0, l0, h1, l1;
              ok &= df_split(v[c].x, h0, l0);
              ok &= df_split(v[c].y, h1, l1);
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
      for (int off = 1; off < 4; off <<= 1) {
        a1 = a1 + shfl_df(a1, off);
        a2 = a2 + shfl_df(a2, off);
        pmx = fmaxf(pmx, __shfl_xor_sync(FULL, pmx, off));
        pmn = fminf(pmn, __shfl_xor_sync(FULL, pmn, off));
        ok &= __shfl_xor_sync(FULL, ok, off);
      }
      if (r == rho) {
        m1 = a1; m2 = a2; mmx = pmx; mmn = pmn; mok = ok;
      }
    }
    // ---------------- phase 2: one slice per lane ----------------
    // the per-sample values come from k1d_params (programmatic dependency)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const long long s = sbase + 8 * r + q;
    int kind = KIND_NONE;
    double A = 1.0, Cc = 0.0, P0 = 0.0, PH = 0.0;
    if (s < total) {
      const int b = (int)(s / g.nt);
      const int k = (int)(s % g.nt);
      const double *pg = params + (size_t)b * g.n_params;
      double *lb = lam + (size_t)b * g.n_rows;
      const double *row = uh + (size_t)s * nx;
      const SampleDerived dv = sd[b];
      BlockStat st;
      if (k == 0) {
        // IC slice: written by the prepare kernel
      } else {
        kind = KIND_MOMENT;
        const double uh0 = row[0], uhh = row[ih];
        const double C = (g.rows & SL_BOUND) ? pg[g.p_c + k] : 0.0;
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
            const df64 e = df64(dv.E0h, dv.E0l) * df_pow(df64(dv.qh, dv.ql), k);
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
          if (cache) {
            const double al = (double)e.alpha, be = (double)e.beta;
            S1d = (double)m1; S2d = (double)m2;
            SliceIn<double> d64 = slice_in_cast<double>(d);
            SliceZ<double> z64{A, Cc, P0, PH, lmd, led, lbd};
            double s00, s01, s02, s11, s12, s22;
            slice_schur(d64, z64, A * S1d + Cc * (double)(nx - 2),
                        A * A * S2d + 2.0 * A * Cc * S1d + Cc * Cc * (double)(nx - 2), 1.0 / al,
                        1.0 / be, s00, s01, s02, s11, s12, s22);
            Ldl3<double> f;
            if (!ldl3_factor(s00, s01, s02, s11, s12, s22, f)) {
              f.d0 = f.d1 = f.d2 = 0.0;
              f.l10 = f.l20 = f.l21 = 0.0;
            }
            SliceFactor sf{al, be, f.d0, f.d1, f.d2, f.l10, f.l20, f.l21};
            cache[s] = sf;
          }
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
            const double e = dv.E0 * exp(-pg[g.p_rate] * ((double)k / (double)(g.nt - 1)));
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
          if (cache) {
            double s00, s01, s02, s11, s12, s22;
            slice_schur(d, z, e.su, e.su2, 1.0 / e.alpha, 1.0 / e.beta, s00, s01, s02, s11, s12, s22);
            Ldl3<double> f;
            if (!ldl3_factor(s00, s01, s02, s11, s12, s22, f)) {
              f.d0 = f.d1 = f.d2 = 0.0;
              f.l10 = f.l20 = f.l21 = 0.0;
            }
            SliceFactor sf{e.alpha, e.beta, f.d0, f.d1, f.d2, f.l10, f.l20, f.l21};
            cache[s] = sf;
          }
        }
        if (!range_ok) {
          st.iters = R.iters;
          st.backtracks = R.backtracks;
          st.status = R.status;
          st.corrections = R.corrections;
          st.kkt_inf = res;
          st.h_inf = nan_max(nan_max(fabs(hm), fabs(he)), fabs(hb));
          const double am1 = A - 1.0;
          st.obj = 0.5 * (am1 * am1 * S2d + 2.0 * am1 * Cc * S1d + Cc * Cc * (double)(nx - 2) +
                          (P0 - uh0) * (P0 - uh0) + (PH - uhh) * (PH - uhh));
        }
        if (g.off_mass >= 0) lb[g.off_mass + k] = lmd;
        if (g.off_energy >= 0) lb[g.off_energy + k] = led;
        if (g.off_bound >= 0) lb[g.off_bound + k] = lbd;
        bst[s] = st;
      }
    }
    // ---------------- phase 3: write-back, 4 lanes per slice ----------------
#pragma unroll 1
    for (int rho = 0; rho < 4; ++rho) {
      const int src = 4 * q + rho;
      const double a = __shfl_sync(FULL, A, src);
      const double c0 = __shfl_sync(FULL, Cc, src);
      const double p0 = __shfl_sync(FULL, P0, src);
      const double ph = __shfl_sync(FULL, PH, src);
      const int kd = __shfl_sync(FULL, kind, src);
      const long long s2 = sbase + 8 * rho + q;
      if (s2 >= total || kd == KIND_NONE) continue;
      const double *row = uh + (size_t)s2 * nx;
      double *out = u + (size_t)s2 * nx;
      if (kd == KIND_MOMENT) {
        constexpr int CH = 16;
        for (int i0 = 2 * r; i0 < nx; i0 += 8 * CH) {
          double2 v[CH];
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const int i = i0 + 8 * c;
            v[c] = (i < nx) ? __ldg(reinterpret_cast<const double2 *>(row + i)) : make_double2(0.0, 0.0);
          }
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const int i = i0 + 8 * c;
            if (i >= nx) break;
            double2 w;
            w.x = (i == 0) ? p0 : ((i == ih) ? ph : fma(a, v[c].x, c0));
            w.y = (i + 1 == ih) ? ph : fma(a, v[c].y, c0);
            *reinterpret_cast<double2 *>(out + i) = w;
          }
        }
      }
    }
  }
}

}  // namespace

void launch_1d_mixed(const Geom1D &g, int B, const double *u_hat, const double *params,
                     const SampleDerived *sd, double *u, double *lambda, BlockStat *bst,
                     SliceFactor *cache, const SolverOpts &o, int blocks_per_sm, cudaStream_t s) {
  const long long ntiles = ((long long)B * g.nt + 31) / 32;
  long long blocks = (ntiles + 1) / 2;
  if (blocks_per_sm > 0 && blocks > 148LL * blocks_per_sm) blocks = 148LL * blocks_per_sm;
  if (blocks > 148LL * 128) blocks = 148LL * 128;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(64);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k1d_mixed, g, B, u_hat, params, sd, u, lambda, bst, cache, o);
}
