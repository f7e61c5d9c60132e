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
// The three phases are the warp tile mixed_tile (tile_1d.cuh), the device code of the
// uneven-batch kernel too, instantiated here with 4 lanes per slice and 16 loads in flight per
// lane and an address policy over the rows of one batch (the batch kernel locates its slices
// through a per-instance pointer table instead).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "snap_bounds.cuh"
#include "tile_1d.cuh"
#include "snap_internal.h"

namespace {

// Slices of the per-problem batch: slice s = b nt + k is row s of u_hat / u, its sample's
// parameters, multipliers and derived values are at b.
struct DirectTiles {
  const double *uh, *params;
  const SampleDerived *sd;
  double *u, *lam;
  BlockStat *bst;
  long long total;
  int nt, nx, n_params, n_rows;
  __device__ __forceinline__ int slice_k(long long s) const { return (int)(s % nt); }
  __device__ __forceinline__ long long sample(long long s) const { return s / nt; }
  __device__ __forceinline__ const double *row_in(long long s) const { return uh + (size_t)s * nx; }
  __device__ __forceinline__ double *row_out(long long s) const { return u + (size_t)s * nx; }
  __device__ __forceinline__ const double *par(long long s) const {
    return params + (size_t)sample(s) * n_params;
  }
  __device__ __forceinline__ double *lam_of(long long s) const {
    return lam + (size_t)sample(s) * n_rows;
  }
  __device__ __forceinline__ SampleDerived derived(long long s) const { return sd[sample(s)]; }
  __device__ __forceinline__ BlockStat *stat(long long s) const { return bst + s; }
  // pull the tile (consecutive slices, contiguous in HBM) into L2 ahead of the loads
  __device__ __forceinline__ void prefetch(long long s0, long long s1, int lane) const {
    const char *t0 = reinterpret_cast<const char *>(uh + (size_t)s0 * nx);
    const size_t bytes = (size_t)(s1 - s0) * nx * sizeof(double);
    for (size_t off = (size_t)lane * 128; off < bytes; off += 32 * 128)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(t0 + off));
  }
  // the per-sample values come from k1d_params (programmatic dependency)
  __device__ __forceinline__ void before_solve(long long, long long, int) const {
    asm volatile("griddepcontrol.wait;" ::: "memory");
  }
  __device__ __forceinline__ bool row_ok(int site, long long s, int i) const {
    return snap_in_bounds(site, s * nx + i + 1, total * nx);
  }
  __device__ __forceinline__ bool slice_ok(long long s) const {
    return snap_in_bounds(SNAP_SITE_MIXED_ROW, s, total);
  }
};

// One warp per tile of 32 consecutive slices (the shared warp tile mixed_tile of tile_1d.cuh
// with 4 lanes per slice and 16 loads in flight per lane); a grid-stride loop over the tiles.
__global__ void __launch_bounds__(64, 8)
k1d_mixed(Geom1D g, int B, const double *__restrict__ uh, const double *__restrict__ params,
          const SampleDerived *__restrict__ sd, double *__restrict__ u,
          double *__restrict__ lam, BlockStat *__restrict__ bst, SolverOpts o,
          SliceOptsT<float> so_f, SliceOptsT<df64> so_d, df64 dxd) {
  // so_f, so_d, dxd: the options and dx in float and double-float, converted once on the host
  // (the same conversion functions): each FP64 conversion here would hold the SM's narrow
  // FP64 pipe for every thread of the launch before the first loads
  const long long total = (long long)B * g.nt;
  const long long ntiles = (total + 31) >> 5;
  const int wpb = blockDim.x >> 5;
  const DirectTiles ad{uh, params, sd, u, lam, bst, total, g.nt, g.nx, g.n_params, g.n_rows};
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  for (long long tile = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); tile < ntiles;
       tile += (long long)gridDim.x * wpb) {
    const long long sbase = tile << 5;
    const long long send = (sbase + 32 < total) ? sbase + 32 : total;
    mixed_tile<DirectTiles, 2, 16>(g, ad, sbase, send, o, so_f, so_d, dxd, 2);
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
