// 1-D families A/B, moment path with the arithmetic spread over the SM's pipes.
//
// On B300 the FP64 pipe retires ~0.46 T FMA/s against ~34 T FP32 FMA/s, so one FP64
// instruction per element already costs as much time as streaming the element through HBM.
// This kernel therefore keeps FP64 for the one operation per element that needs it (the
// write-back u_i = a u_hat_i + c) and moves everything else to the FP32 / integer pipes:
//
//   phase 1  (4 lanes per slice, 8 slices per warp instruction, 16-byte loads): every
//            u_hat_i is split into a float pair hi + lo with integer operations only
//            (df_split_trunc_fast: nothing on the FP64 pipe; |u_hat - hi - lo| < 2^-46
//            |u_hat|), and the interior moments
//            S1 = sum u_hat_i, S2 = sum u_hat_i^2 are accumulated in double-float
//            (error-free TwoSum / TwoProd), reduced across the 4 lanes with two butterfly
//            steps;
//   phase 2  (one slice per lane): the slice's Newton-KKT iteration in moment form,
//            first in float, then in double-float to the FP64 stopping tolerance
//            (t1_solve_slice / slice_solve_mixed, warm-started inside W > 0); E_k = E0 q^k
//            with q = exp(-r dt) by binary powering in double-float;
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
// [2^-74, 2^57], exactly zero, or non-finite) falls back to FP64 moments and the FP64
// iteration.
//
// Phase 2 is t1_solve_slice (tile_1d.cuh), the same device code as the uneven-batch kernel's
// tile; phases 1 and 3 stay inline here (the batch kernel locates its slices through a
// per-instance pointer table instead).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "snap_bounds.cuh"
#include "tile_1d.cuh"
#include "snap_internal.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;

enum { KIND_MOMENT = 0, KIND_NONE = 3 };

__device__ __forceinline__ df64 shfl_df(df64 v, int off) {
  return df64(__shfl_xor_sync(FULL, v.hi, off), __shfl_xor_sync(FULL, v.lo, off));
}

__global__ void __launch_bounds__(64, 8)
k1d_mixed(Geom1D g, int B, const double *__restrict__ uh, const double *__restrict__ params,
          const SampleDerived *__restrict__ sd, double *__restrict__ u,
          double *__restrict__ lam, BlockStat *__restrict__ bst, SolverOpts o,
          SliceOptsT<float> so_f, SliceOptsT<df64> so_d, df64 dxd) {
  const int lane = threadIdx.x & 31;
  const int q = lane >> 2;        // group: slice 8*rho + q of round rho
  const int r = lane & 3;         // lane within the group
  const long long total = (long long)B * g.nt;
  const long long ntiles = (total + 31) >> 5;
  const int wpb = blockDim.x >> 5;
  const int nx = g.nx, ih = g.ih;
  // so_f, so_d, dxd: the options and dx in float and double-float, converted once on the host
  // (the same conversion functions): each FP64 conversion here would hold the SM's narrow
  // FP64 pipe for every thread of the launch before the first loads
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
              v[c] = (i < nx && snap_in_bounds(SNAP_SITE_MOMENT_ROW, s * nx + i + 1, total * nx))
                         ? *reinterpret_cast<const double2 *>(row + i) : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
              const int i = i0 + 8 * c;
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
    if (s < total && (s % g.nt) != 0 && snap_in_bounds(SNAP_SITE_MIXED_ROW, s, total)) {
      // the IC slice (k = 0) is written by the prepare kernel
      const int b = (int)(s / g.nt);
      const int k = (int)(s % g.nt);
      const double *row = uh + (size_t)s * nx;
      kind = KIND_MOMENT;
      t1_solve_slice(g, k, m1, m2, mmx, mmn, mok, __ldg(row), __ldg(row + ih), row,
                     params + (size_t)b * g.n_params, sd[b], lam + (size_t)b * g.n_rows, bst + s,
                     o, so_f, so_d, dxd, A, Cc, P0, PH);
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
            v[c] = (i < nx) ? *reinterpret_cast<const double2 *>(row + i) : make_double2(0.0, 0.0);
          }
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const int i = i0 + 8 * c;
            if (i >= nx) break;
            double2 w;
            w.x = (i == 0) ? p0 : ((i == ih) ? ph : fma(a, v[c].x, c0));
            w.y = (i + 1 == ih) ? ph : fma(a, v[c].y, c0);
            if (snap_in_bounds(SNAP_SITE_MIXED_ROW, s2 * nx + i + 1, total * nx))
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
                     const SolverOpts &o, int blocks_per_sm, cudaStream_t s) {
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
  const SliceOptsT<float> so_f = slice_opts<float>(o, o.tol_kkt);
  const SliceOptsT<df64> so_d = slice_opts<df64>(o, o.tol_kkt);
  const df64 dxd(g.dx);
  cudaLaunchKernelEx(&cfg, k1d_mixed, g, B, u_hat, params, sd, u, lambda, bst, o, so_f, so_d,
                     dxd);
}
