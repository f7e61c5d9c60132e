// 1-D families A/B: the per-problem implicit-function adjoint kernel, one warp per tile of 32
// consecutive slices (bwd_tile, tile_1d_bwd.cuh, which also documents the three phases).  The
// IC slices (a = 0) are written by the per-sample prepare kernel.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "slice_newton.cuh"
#include "snap_internal.h"
#include "tile_1d_bwd.cuh"

namespace {

// Slices of one per-problem batch: slice s is slice s % nt of sample s / nt.
struct DirectBwd {
  long long total;
  int nt, nx, n_rows, n_params;
  const double *gu, *u, *lam;
  const snap_stats *fst;
  const SampleDerived *sd;
  double *gh, *gp;
  BwdContrib *contrib;
  __device__ __forceinline__ int sample(long long s) const { return (int)(s / nt); }
  __device__ __forceinline__ bool live(long long s) const { return s < total && (s % nt) != 0; }
  __device__ __forceinline__ int slice_k(long long s) const { return (int)(s % nt); }
  __device__ __forceinline__ const double *row_u(long long s) const { return u + (size_t)s * nx; }
  __device__ __forceinline__ const double *row_g(long long s) const { return gu + (size_t)s * nx; }
  __device__ __forceinline__ double *row_out(long long s) const { return gh + (size_t)s * nx; }
  __device__ __forceinline__ const double *lam_of(long long s) const {
    return lam + (size_t)sample(s) * n_rows;
  }
  __device__ __forceinline__ bool bad(long long s) const {
    return fst && fst[sample(s)].status != SNAP_SAMPLE_OK;
  }
  __device__ __forceinline__ SampleDerived derived(long long s) const { return sd[sample(s)]; }
  __device__ __forceinline__ BwdContrib *contrib_at(long long s) const { return contrib + s; }
  __device__ __forceinline__ double *gp_of(long long s) const {
    return gp ? gp + (size_t)sample(s) * n_params : nullptr;
  }
  // launched as a programmatic dependent of k1d_params: phase 1 overlaps it, the per-sample
  // values and everything written after this point wait for its completion
  __device__ __forceinline__ void before_solve(int) const {
    asm volatile("griddepcontrol.wait;" ::: "memory");
  }
};

__global__ void __launch_bounds__(128, 4)
k1d_bwd_mixed(Geom1D g, int B, const double *__restrict__ gu, const double *__restrict__ u,
              const double *__restrict__ lam, const snap_stats *__restrict__ fst,
              const SampleDerived *__restrict__ sd, double *__restrict__ gh,
              double *__restrict__ gp, BwdContrib *__restrict__ contrib, df64 dxd) {
  const long long total = (long long)B * g.nt;
  const long long ntiles = (total + 31) >> 5;
  const int wpb = blockDim.x >> 5;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const DirectBwd ad{total, g.nt, g.nx, g.n_rows, g.n_params, gu, u, lam, fst, sd, gh, gp,
                     contrib};
  for (long long tile = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); tile < ntiles;
       tile += (long long)gridDim.x * wpb)
    bwd_tile(g, ad, tile << 5, dxd);
}

}  // namespace

void launch_1d_bwd_mixed(const Geom1D &g, int B, const double *grad_u, const double *u,
                         const double *lambda, const double *params, const snap_stats *stats,
                         const SampleDerived *sd, double *grad_u_hat, double *grad_params,
                         BwdContrib *contrib, cudaStream_t s) {
  (void)params;
  const long long ntiles = ((long long)B * g.nt + 31) / 32;
  long long blocks = (ntiles + 3) / 4;
  if (blocks > 148LL * 64) blocks = 148LL * 64;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const df64 dxd(g.dx);
  cudaLaunchKernelEx(&cfg, k1d_bwd_mixed, g, B, grad_u, u, lambda, stats, sd, grad_u_hat,
                     grad_params, contrib, dxd);
}
