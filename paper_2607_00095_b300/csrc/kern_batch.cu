// Uneven batches: instances of different grid sizes and constraint families (1-D families A/B,
// 2-D family C) projected in one persistent kernel launch.
//
// Work units.  A 1-D group (all instances of one 1-D problem) is a virtual batch of
// n_inst * nt time slices; its unit is a tile of up to 32 consecutive slices, solved by one
// warp with the three phases of the per-problem kernel k1d_mixed (tile_1d.cuh).  With pack_1d a tile
// may run across the boundary of two instances of the group, which keeps all 32 lanes busy in
// the per-slice solve when nt is not a multiple of 32.  A 2-D group's unit is one frame of one
// instance, solved by a whole block with the per-problem frame code (frame_2d.cuh).
//
// Scheduling.  The host lays out two queues in the schedule's order; blocks pull 2-D frames
// (one atomic per frame, whole block) and warps pull 1-D tiles (one atomic per tile).  No unit
// waits for another: the per-sample parameters a tile needs (M, E0, q, Appendix-B IC block) are
// derived by the tile's warp itself, and the last unit of an instance to finish -- seen from
// an arrival counter -- reduces that instance's per-slice statistics in fixed order.  Writers
// fence before they count; the reducer fences after and reads through L2.
//
// Workspace: header (queue counters), per-instance arrival counters and first-start stamps
// (zeroed by one memset per call), then the per-slice / per-frame statistics.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "frame_2d.cuh"
#include "sample_1d.cuh"
#include "snap_internal.h"
#include "tile_1d.cuh"
#include "tile_1d_bwd.cuh"

namespace {

constexpr int kThreads = 256;            // block size of the persistent kernel (= T2D)
constexpr int kWarps = kThreads / 32;
constexpr int kMaxTileInst = 17;         // instances one 32-slice tile can touch (nt >= 2)

static_assert(kThreads == T2D, "2-D frames need the whole block");

struct InstRec {
  const double *uh, *params;
  double *u, *lam;
  snap_stats *stats;
};

struct GroupRec {
  Geom1D g;                 // 1-D geometry (family A/B)
  const float *Q, *I;       // 2-D factor (family C)
  long long bst_off;        // first statistics record of the group in the workspace
  int kind;                 // 0: 1-D, 1: 2-D
  int n_inst, list_off, nt, M;
  int lps;                  // 1-D: lanes per slice in the load / write-back passes (2, 4, 8)
  df64 dxd;                 // 1-D: dx in double-float (converted on the host)
};

struct Item1D { int group, s0, s1; };     // slices [s0, s1) of the group's virtual batch
struct Item2D { int group, unit; };       // unit = instance-in-group * nt + frame

struct Hdr {
  unsigned int q1d, q2d;
  unsigned int pad[62];
};

struct BatchArgs {
  const InstRec *inst;
  const GroupRec *groups;
  const int *list;                       // group-ordered instance ids
  const Item1D *items1d;
  const Item2D *items2d;
  int n1d, n2d, order;
  Hdr *hdr;
  unsigned int *done;                    // [n_inst] finished slices / frames
  unsigned long long *negstart;          // [n_inst] max of ~start stamp
  BlockStat *bst;
  unsigned long long *t_ns;
  SolverOpts o;
  // the options in float and double-float, converted once on the host (the same conversion
  // functions as on the device): conversions here would load the narrow FP64 pipe per tile
  SliceOptsT<float> so_f;
  SliceOptsT<df64> so_d;
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Per-warp context of the tile in flight, in shared memory: the compiler reads the geometry
// and offsets from there instead of keeping them in registers through the slice solve.
struct TileCtx {
  Geom1D g;
  BlockStat *bst;                        // the group's first statistics record
  int nt, nx, list_off, first_inst;      // first_inst: instance (in group) of the tile's slice 0
};

// Address policy of a 1-D tile of a group: slice s of the group's virtual batch is slice
// s % nt of the group's instance s / nt (32-bit: n_inst nt < 2^31 is checked at create); the
// derived values of the tile's instances sit in the warp's shared table (filled by
// before_solve).
struct BatchTiles {
  const InstRec *inst;
  const int *list;
  SampleDerived *sdw;                    // this warp's table
  const TileCtx *c;
  double tol_kkt;
  __device__ __forceinline__ int nt() const { return c->nt; }
  __device__ __forceinline__ int inst_of(long long s) const { return (int)s / nt(); }
  __device__ __forceinline__ const InstRec &rec(long long s) const {
    return inst[list[c->list_off + inst_of(s)]];
  }
  __device__ __forceinline__ int slice_k(long long s) const { return (int)s % nt(); }
  __device__ __forceinline__ const double *row_in(long long s) const {
    return rec(s).uh + (size_t)slice_k(s) * c->nx;
  }
  __device__ __forceinline__ double *row_out(long long s) const {
    return rec(s).u + (size_t)slice_k(s) * c->nx;
  }
  __device__ __forceinline__ const double *par(long long s) const { return rec(s).params; }
  __device__ __forceinline__ double *lam_of(long long s) const { return rec(s).lam; }
  __device__ __forceinline__ SampleDerived derived(long long s) const {
    return sdw[inst_of(s) - c->first_inst];
  }
  __device__ __forceinline__ BlockStat *stat(long long s) const { return c->bst + (int)s; }
  // the bounds-checked build checks the per-problem kernels; the batch's slices are located
  // through the instance table
  __device__ __forceinline__ bool row_ok(int, long long, int) const { return true; }
  __device__ __forceinline__ bool slice_ok(long long) const { return true; }
  __device__ __forceinline__ void prefetch(long long s0l, long long s1l, int lane) const {
    const int s0 = (int)s0l, s1 = (int)s1l, n = nt();
    for (int i = s0 / n; i * n < s1; ++i) {
      const int a = (i * n > s0) ? i * n : s0;
      const int b = ((i + 1) * n < s1) ? (i + 1) * n : s1;
      const char *t0 = reinterpret_cast<const char *>(row_in(a));
      const int bytes = (b - a) * c->nx * (int)sizeof(double);
      for (int off = lane * 128; off < bytes; off += 32 * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(t0 + off));
    }
  }
  __device__ __forceinline__ void before_solve(long long s0l, long long s1l, int lane) const {
    const int s0 = (int)s0l, s1 = (int)s1l, n = nt();
    for (int i = s0 / n; i * n < s1; ++i) {
      const InstRec &R = inst[list[c->list_off + i]];
      const SampleDerived d = s1_derive(c->g, R.params, lane);
      if (lane == 0) sdw[i - c->first_inst] = d;
      if (i * n >= s0)                   // slice 0 of this instance is in the tile
        s1_ic_forward(c->g, R.params, R.uh, R.u, R.lam, c->bst + i * n, d.h0_inf, tol_kkt, lane);
    }
    __syncwarp();
  }
};

template <int M>
__device__ __forceinline__ void run_frame(unsigned char *smem, const GroupRec &G, const InstRec &R,
                                          int f, BlockStat *out, const SolverOpts &o) {
  constexpr int NN = 4 * M * M;
  View2D<M> v(smem);
  frame2d_forward<M>(v, R.uh + (size_t)f * 2 * NN, R.params, f, G.nt, G.Q, G.I,
                     R.u + (size_t)f * 2 * NN, R.lam, out, o);
}

__device__ __forceinline__ void batch_2d(const BatchArgs &a, unsigned char *smem) {
  __shared__ int s_item, s_last;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(&a.hdr->q2d, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= a.n2d) break;
    const Item2D w = a.items2d[it];
    const GroupRec &G = a.groups[w.group];
    const int il = w.unit / G.nt, f = w.unit % G.nt;
    const int id = a.list[G.list_off + il];
    const InstRec &R = a.inst[id];
    if (threadIdx.x == 0 && a.t_ns) atomicMax(&a.negstart[id], ~gtimer());
    BlockStat *bs = a.bst + G.bst_off + w.unit;
    switch (G.M) {
      case 2: run_frame<2>(smem, G, R, f, bs, a.o); break;
      case 4: run_frame<4>(smem, G, R, f, bs, a.o); break;
      case 8: run_frame<8>(smem, G, R, f, bs, a.o); break;
      case 16: run_frame<16>(smem, G, R, f, bs, a.o); break;
      default: run_frame<32>(smem, G, R, f, bs, a.o); break;
    }
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned old = atomicAdd(&a.done[id], 1u);
      s_last = (old + 1u == (unsigned)G.nt);
    }
    __syncthreads();
    if (s_last && threadIdx.x < 32) {
      __threadfence();
      s1_finalize<true>(a.bst + G.bst_off + (long long)il * G.nt, G.nt, a.o.tol_h, R.stats,
                        threadIdx.x);
      if (threadIdx.x == 0 && a.t_ns) {
        a.t_ns[2 * (size_t)id] = ~atomicOr(&a.negstart[id], 0ull);
        a.t_ns[2 * (size_t)id + 1] = gtimer();
      }
    }
    __syncthreads();
  }
}

// Arrival of 1-D tile `it`: count its slices per instance; the last arrival reduces.
__device__ __noinline__ void finish_tile(const BatchArgs &a, unsigned it, int lane) {
  const Item1D w = a.items1d[it];
  const GroupRec &G = a.groups[w.group];
  const int nt = G.nt;
  const int s0 = w.s0, s1 = w.s1;
  for (int i = s0 / nt; i * nt < s1; ++i) {
    const int a0 = (i * nt > s0) ? i * nt : s0;
    const int b0 = ((i + 1) * nt < s1) ? (i + 1) * nt : s1;
    const int id = a.list[G.list_off + i];
    unsigned last = 0;
    if (lane == 0) {
      const unsigned cnt = (unsigned)(b0 - a0);
      last = (atomicAdd(&a.done[id], cnt) + cnt == (unsigned)nt) ? 1u : 0u;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      __threadfence();
      s1_finalize<true>(a.bst + G.bst_off + (long long)i * nt, nt, a.o.tol_h, a.inst[id].stats,
                        lane);
      if (lane == 0 && a.t_ns) {
        a.t_ns[2 * (size_t)id] = ~atomicOr(&a.negstart[id], 0ull);
        a.t_ns[2 * (size_t)id + 1] = gtimer();
      }
    }
  }
}

// One 32-slice (or shorter) tile [t0, t1) of an item: the warp's context, then the tile with
// the group's lanes per slice.
__device__ __forceinline__ void run_subtile_1d(const BatchArgs &a, const GroupRec &G, int t0,
                                               int t1, SampleDerived *sdw, TileCtx *cx) {
  const int lane = threadIdx.x & 31;
  const int nt = G.nt;
  const int i0 = t0 / nt, i1 = (t1 - 1) / nt;
  if (a.t_ns && lane <= i1 - i0) atomicMax(&a.negstart[a.list[G.list_off + i0 + lane]], ~gtimer());
  {
    const int *src = reinterpret_cast<const int *>(&G.g);
    int *dst = reinterpret_cast<int *>(&cx->g);
    if (lane < (int)(sizeof(Geom1D) / sizeof(int))) dst[lane] = src[lane];
  }
  if (lane == 0) {
    cx->bst = a.bst + G.bst_off;
    cx->nt = nt;
    cx->nx = G.g.nx;
    cx->list_off = G.list_off;
    cx->first_inst = i0;
  }
  __syncwarp();
  BatchTiles ad;
  ad.inst = a.inst;
  ad.list = a.list;
  ad.sdw = sdw;
  ad.c = cx;
  ad.tol_kkt = a.o.tol_kkt;
  mixed_tile(cx->g, ad, t0, t1, a.o, a.so_f, a.so_d, G.dxd,
             G.lps == 2 ? 1 : (G.lps == 8 ? 3 : 2));
  __syncwarp();                          // the context is rewritten by the next tile
}

__device__ __forceinline__ void batch_1d(const BatchArgs &a, SampleDerived *sdw, TileCtx *cx) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned it = 0;
    if (lane == 0) it = atomicAdd(&a.hdr->q1d, 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= (unsigned)a.n1d) break;
    const Item1D w = a.items1d[it];
    const GroupRec &G = a.groups[w.group];
    // an item of up to 64 slices runs as tiles of at most 32
    for (int t0 = w.s0; t0 < w.s1; t0 += 32) {
      const int t1 = (t0 + 32 < w.s1) ? t0 + 32 : w.s1;
      run_subtile_1d(a, G, t0, t1, sdw, cx);
    }
    // arrival: every lane's statistics and outputs are fenced before lane 0 counts
    __threadfence();
    __syncwarp();
    finish_tile(a, it, lane);
    __syncwarp();
  }
}

__global__ void __launch_bounds__(kThreads, 2) k_batch(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_batch[];
  __shared__ SampleDerived sdtab[kWarps][kMaxTileInst];
  __shared__ TileCtx ctx[kWarps];
  SampleDerived *sdw = sdtab[threadIdx.x >> 5];
  TileCtx *cx = &ctx[threadIdx.x >> 5];
  if (a.order == 0) {
    if (a.n2d > 0) batch_2d(a, smem_batch);
    if (a.n1d > 0) batch_1d(a, sdw, cx);
  } else {
    if (a.n1d > 0) batch_1d(a, sdw, cx);
    if (a.n2d > 0) {
      __syncthreads();
      batch_2d(a, smem_batch);
    }
  }
}

// ---------------------------------------------------------------------------------------
// Adjoint of an uneven batch: the same work lists and queues as the forward, the per-family
// adjoint device code (bwd_tile for 1-D tiles, frame2d_backward for 2-D frames), per-slice /
// per-frame contributions to dL/dparams in the statistics area of the workspace, and the
// per-instance parameter gradient formed by the last unit of the instance to finish.
// ---------------------------------------------------------------------------------------
struct BwdRec {
  const double *gu;        // dL/du (input)
  double *gh, *gp;         // dL/du_hat, dL/dparams (outputs; gp may be null)
};

struct BwdArgs {
  const InstRec *inst;
  const BwdRec *bwd;
  const GroupRec *groups;
  const int *list;
  const Item1D *items1d;
  const Item2D *items2d;
  int n1d, n2d, order;
  Hdr *hdr;
  unsigned int *done;
  BwdContrib *contrib;
};

// Address policy of a 1-D adjoint tile of a group (the slices of instance i of the group are
// i nt .. i nt + nt - 1 of the group's virtual batch; the tile is [s0, s1)).
struct BatchBwdTiles {
  const InstRec *inst;
  const BwdRec *bwd;
  const int *list;
  BwdContrib *contrib;                   // the group's first contribution
  SampleDerived *sdw;                    // this warp's table
  const TileCtx *c;
  long long s0, s1;
  __device__ __forceinline__ int nt() const { return c->nt; }
  __device__ __forceinline__ int inst_of(long long s) const { return (int)s / nt(); }
  __device__ __forceinline__ int id_of(long long s) const { return list[c->list_off + inst_of(s)]; }
  __device__ __forceinline__ bool live(long long s) const {
    return s < s1 && ((int)s % nt()) != 0;
  }
  __device__ __forceinline__ int slice_k(long long s) const { return (int)s % nt(); }
  __device__ __forceinline__ const double *row_u(long long s) const {
    return inst[id_of(s)].u + (size_t)slice_k(s) * c->nx;
  }
  __device__ __forceinline__ const double *row_g(long long s) const {
    return bwd[id_of(s)].gu + (size_t)slice_k(s) * c->nx;
  }
  __device__ __forceinline__ double *row_out(long long s) const {
    return bwd[id_of(s)].gh + (size_t)slice_k(s) * c->nx;
  }
  __device__ __forceinline__ const double *lam_of(long long s) const { return inst[id_of(s)].lam; }
  __device__ __forceinline__ bool bad(long long s) const {
    return inst[id_of(s)].stats->status != SNAP_SAMPLE_OK;
  }
  __device__ __forceinline__ SampleDerived derived(long long s) const {
    return sdw[inst_of(s) - c->first_inst];
  }
  __device__ __forceinline__ BwdContrib *contrib_at(long long s) const { return contrib + (int)s; }
  __device__ __forceinline__ double *gp_of(long long s) const { return bwd[id_of(s)].gp; }
  // the tile's instances: derived values into the warp's table; the IC block of an instance
  // whose slice 0 is in the tile (a = 0 there, and the boundary parameter of slice 0)
  __device__ __forceinline__ void before_solve(int lane) const {
    const int n = nt(), a0 = (int)s0, a1 = (int)s1;
    for (int i = a0 / n; i * n < a1; ++i) {
      const int id = list[c->list_off + i];
      const InstRec &R = inst[id];
      const SampleDerived d = s1_derive(c->g, R.params, lane);
      if (lane == 0) sdw[i - c->first_inst] = d;
      if (i * n >= a0) {
        const BwdRec &W = bwd[id];
        const bool bd = R.stats->status != SNAP_SAMPLE_OK;
        for (int x = lane; x < c->nx; x += 32) W.gh[x] = bd ? NAN : 0.0;
        if (lane == 0 && W.gp && (c->g.rows & SL_BOUND)) W.gp[c->g.p_c] = bd ? NAN : 0.0;
      }
    }
    __syncwarp();
  }
};

template <int M>
__device__ __forceinline__ void run_frame_bwd(unsigned char *smem, const GroupRec &G,
                                              const InstRec &R, const BwdRec &W, int f,
                                              BwdContrib *out) {
  constexpr int NN = 4 * M * M;
  View2D<M> v(smem);
  const bool bd = R.stats->status != SNAP_SAMPLE_OK;
  frame2d_backward<M>(v, W.gu + (size_t)f * 2 * NN, R.u + (size_t)f * 2 * NN,
                      R.lam[(size_t)G.nt * NN + f], R.params, f, G.nt, bd, G.Q, G.I,
                      W.gh + (size_t)f * 2 * NN, out);
}

__device__ __forceinline__ void batch_2d_bwd(const BwdArgs &a, unsigned char *smem) {
  __shared__ int s_item, s_last;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(&a.hdr->q2d, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= a.n2d) break;
    const Item2D w = a.items2d[it];
    const GroupRec &G = a.groups[w.group];
    const int il = w.unit / G.nt, f = w.unit % G.nt;
    const int id = a.list[G.list_off + il];
    const InstRec &R = a.inst[id];
    const BwdRec &W = a.bwd[id];
    BwdContrib *cs = a.contrib + G.bst_off + w.unit;
    switch (G.M) {
      case 2: run_frame_bwd<2>(smem, G, R, W, f, cs); break;
      case 4: run_frame_bwd<4>(smem, G, R, W, f, cs); break;
      case 8: run_frame_bwd<8>(smem, G, R, W, f, cs); break;
      case 16: run_frame_bwd<16>(smem, G, R, W, f, cs); break;
      default: run_frame_bwd<32>(smem, G, R, W, f, cs); break;
    }
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned old = atomicAdd(&a.done[id], 1u);
      s_last = (old + 1u == (unsigned)G.nt);
    }
    __syncthreads();
    if (s_last && threadIdx.x < 32 && W.gp) {
      __threadfence();
      frame2d_param_grad<true>(a.contrib + G.bst_off + (long long)il * G.nt, G.nt,
                               R.stats->status != SNAP_SAMPLE_OK, W.gp, threadIdx.x);
    }
    __syncthreads();
  }
}

// Arrival of adjoint tile `it`: count its slices per instance; the last arrival forms the
// instance's dL/dparams.
__device__ __noinline__ void finish_tile_bwd(const BwdArgs &a, unsigned it, int lane) {
  const Item1D w = a.items1d[it];
  const GroupRec &G = a.groups[w.group];
  const int nt = G.nt;
  const int s0 = w.s0, s1 = w.s1;
  for (int i = s0 / nt; i * nt < s1; ++i) {
    const int a0 = (i * nt > s0) ? i * nt : s0;
    const int b0 = ((i + 1) * nt < s1) ? (i + 1) * nt : s1;
    const int id = a.list[G.list_off + i];
    unsigned last = 0;
    if (lane == 0) {
      const unsigned cnt = (unsigned)(b0 - a0);
      last = (atomicAdd(&a.done[id], cnt) + cnt == (unsigned)nt) ? 1u : 0u;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    const BwdRec &W = a.bwd[id];
    if (last && W.gp) {
      __threadfence();
      const InstRec &R = a.inst[id];
      const double M = s1_derive(G.g, R.params, lane).M;
      s1_param_grad<true>(G.g, W.gu, R.params, M,
                          a.contrib + G.bst_off + (long long)i * nt,
                          R.stats->status != SNAP_SAMPLE_OK, W.gp, lane);
    }
  }
}

__device__ __forceinline__ void batch_1d_bwd(const BwdArgs &a, SampleDerived *sdw, TileCtx *cx) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned it = 0;
    if (lane == 0) it = atomicAdd(&a.hdr->q1d, 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= (unsigned)a.n1d) break;
    const Item1D w = a.items1d[it];
    const GroupRec &G = a.groups[w.group];
    const int nt = G.nt;
    // an item of up to 64 slices runs as tiles of at most 32
    for (int t0 = w.s0; t0 < w.s1; t0 += 32) {
      const int t1 = (t0 + 32 < w.s1) ? t0 + 32 : w.s1;
      const int first = t0 / nt;
      {
        const int *src = reinterpret_cast<const int *>(&G.g);
        int *dst = reinterpret_cast<int *>(&cx->g);
        if (lane < (int)(sizeof(Geom1D) / sizeof(int))) dst[lane] = src[lane];
      }
      if (lane == 0) {
        cx->nt = nt;
        cx->nx = G.g.nx;
        cx->list_off = G.list_off;
        cx->first_inst = first;
      }
      __syncwarp();
      BatchBwdTiles ad;
      ad.inst = a.inst;
      ad.bwd = a.bwd;
      ad.list = a.list;
      ad.contrib = a.contrib + G.bst_off;
      ad.sdw = sdw;
      ad.c = cx;
      ad.s0 = t0;
      ad.s1 = t1;
      bwd_tile(cx->g, ad, t0, G.dxd);
      __syncwarp();
    }
    // arrival: every lane's contributions and outputs are fenced before lane 0 counts
    __threadfence();
    __syncwarp();
    finish_tile_bwd(a, it, lane);
    __syncwarp();                        // the context is rewritten by the next item
  }
}

__global__ void __launch_bounds__(kThreads, 2) k_batch_bwd(BwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem_batch_bwd[];
  __shared__ SampleDerived sdtab[kWarps][kMaxTileInst];
  __shared__ TileCtx ctx[kWarps];
  SampleDerived *sdw = sdtab[threadIdx.x >> 5];
  TileCtx *cx = &ctx[threadIdx.x >> 5];
  if (a.order == 0) {
    if (a.n2d > 0) batch_2d_bwd(a, smem_batch_bwd);
    if (a.n1d > 0) batch_1d_bwd(a, sdw, cx);
  } else {
    if (a.n1d > 0) batch_1d_bwd(a, sdw, cx);
    if (a.n2d > 0) {
      __syncthreads();
      batch_2d_bwd(a, smem_batch_bwd);
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------------------

struct snap_batch {
  int n_inst = 0;
  std::vector<const snap_problem *> probs;
  std::vector<int> inst_problem;
  // groups: one per problem with instances, in problem order
  std::vector<int> group_problem;
  std::vector<std::vector<int>> group_inst;
  std::vector<GroupRec> groups;          // host copy (bst_off, list_off set at create)
  std::vector<int> list;
  long long n_blocks = 0;                // statistics records
  int max_m = 0;                         // largest 2-D class size in the batch
  size_t smem_bytes = 0;
  size_t grouped_ws = 0;
  bool bound = false;
  std::vector<InstRec> h_inst;
  std::vector<char> group_contig;        // bound buffers contiguous per group
  snap_batch_schedule sched{2, 0, 1, 1, 32, 4};
  int n1d = 0, n2d = 0;
  int device = 0;
  int grid = 0;                          // persistent grid of the current schedule
  // device tables
  InstRec *d_inst = nullptr;
  GroupRec *d_groups = nullptr;
  int *d_list = nullptr;
  Item1D *d_items1d = nullptr;
  Item2D *d_items2d = nullptr;
  size_t cap1d = 0, cap2d = 0;
  cudaGraphExec_t graph = nullptr;
  // adjoint
  BwdRec *d_bwd = nullptr;
  std::vector<BwdRec> h_bwd;
  std::vector<char> group_contig_bwd;
  bool bound_bwd = false;
  int grid_bwd = 0;                      // persistent grid of the adjoint kernel
  cudaGraphExec_t graph_bwd = nullptr;
};

namespace {

size_t hdr_bytes(const snap_batch *b) {
  return snap_align256(sizeof(Hdr) + sizeof(unsigned int) * (size_t)b->n_inst) +
         snap_align256(sizeof(unsigned long long) * (size_t)b->n_inst);
}

size_t batch_ws_bytes(const snap_batch *b) {
  const size_t own = hdr_bytes(b) + snap_align256(sizeof(BlockStat) * (size_t)b->n_blocks);
  return own > b->grouped_ws ? own : b->grouped_ws;
}

void build_items(const snap_batch *b, const snap_batch_schedule &s, std::vector<Item1D> &i1,
                 std::vector<Item2D> &i2) {
  i1.clear();
  i2.clear();
  std::vector<int> order;
  for (int gi = 0; gi < (int)b->groups.size(); ++gi) order.push_back(gi);
  if (s.sort_1d == 1)
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      const GroupRec &a = b->groups[x], &c = b->groups[y];
      const int wa = a.kind == 0 ? a.g.nx : 0, wc = c.kind == 0 ? c.g.nx : 0;
      return wa > wc;
    });
  for (int gi : order) {
    const GroupRec &G = b->groups[gi];
    if (G.kind == 0) {
      const int total = G.n_inst * G.nt;
      const int tile = s.tile_1d;
      if (s.pack_1d) {
        for (int s0 = 0; s0 < total; s0 += tile) i1.push_back(Item1D{gi, s0, std::min(s0 + tile, total)});
      } else {
        for (int i = 0; i < G.n_inst; ++i)
          for (int k = 0; k < G.nt; k += tile)
            i1.push_back(Item1D{gi, i * G.nt + k, i * G.nt + std::min(k + tile, G.nt)});
      }
    }
  }
  // 2-D: larger frames first, frames of one instance together
  std::vector<int> o2;
  for (int gi = 0; gi < (int)b->groups.size(); ++gi)
    if (b->groups[gi].kind == 1) o2.push_back(gi);
  std::stable_sort(o2.begin(), o2.end(),
                   [&](int x, int y) { return b->groups[x].M > b->groups[y].M; });
  for (int gi : o2) {
    const GroupRec &G = b->groups[gi];
    for (int u = 0; u < G.n_inst * G.nt; ++u) i2.push_back(Item2D{gi, u});
  }
}

template <class K>
int grid_blocks_of(const snap_batch *b, int ctas_per_sm, K kernel) {
  int sms = 148, occ = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, b->smem_bytes) !=
          cudaSuccess ||
      occ < 1)
    occ = 1;
  int per = ctas_per_sm < 1 ? 1 : ctas_per_sm;
  if (per > occ) per = occ;
  return sms * per;
}

int grid_blocks(const snap_batch *b, int ctas_per_sm) { return grid_blocks_of(b, ctas_per_sm, k_batch); }

snap_status upload_items(snap_batch *b) {
  std::vector<Item1D> i1;
  std::vector<Item2D> i2;
  build_items(b, b->sched, i1, i2);
  if (i1.size() > b->cap1d || i2.size() > b->cap2d)
    return snap_fail_msg(SNAP_ERR_INVALID_ARG, "batch work list larger than its allocation");
  if (!i1.empty() && cudaMemcpy(b->d_items1d, i1.data(), sizeof(Item1D) * i1.size(),
                                cudaMemcpyHostToDevice) != cudaSuccess)
    return snap_fail_msg(SNAP_ERR_CUDA, "upload of the 1-D work list failed");
  if (!i2.empty() && cudaMemcpy(b->d_items2d, i2.data(), sizeof(Item2D) * i2.size(),
                                cudaMemcpyHostToDevice) != cudaSuccess)
    return snap_fail_msg(SNAP_ERR_CUDA, "upload of the 2-D work list failed");
  b->n1d = (int)i1.size();
  b->n2d = (int)i2.size();
  b->grid = grid_blocks(b, b->sched.ctas_per_sm);
  b->grid_bwd = grid_blocks_of(b, b->sched.ctas_per_sm, k_batch_bwd);
  return SNAP_OK;
}

void free_batch(snap_batch *b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->graph_bwd) cudaGraphExecDestroy(b->graph_bwd);
  cudaFree(b->d_bwd);
  cudaFree(b->d_inst);
  cudaFree(b->d_groups);
  cudaFree(b->d_list);
  cudaFree(b->d_items1d);
  cudaFree(b->d_items2d);
  delete b;
}

bool aligned(const void *p, unsigned a) { return ((uintptr_t)p & (a - 1)) == 0; }

SolverOpts solver_opts(const snap_options &o) {
  SolverOpts so;
  so.tol_kkt = o.tol_kkt;
  so.tol_h = o.tol_h;
  so.c1 = o.armijo_c1;
  so.delta0 = o.delta0;
  so.w_keep = o.w_keep;
  so.max_iter = o.max_iter;
  so.max_backtracks = o.max_backtracks;
  so.max_corrections = o.max_corrections;
  so.pad = 0;
  return so;
}

snap_status get_opts(const snap_options *opt, snap_options &o) {
  snap_options_default(&o);
  if (opt) o = *opt;
  if (snap_check_options(o) != SNAP_OK) return SNAP_ERR_INVALID_ARG;
  return SNAP_OK;
}

// Lanes per slice of every 1-D group (2, 4 or 8; entries of 2-D groups ignored); uploads the
// group table.
snap_status set_group_lanes(snap_batch *b, const int *lanes) {
  for (size_t k = 0; k < b->groups.size(); ++k)
    if (b->groups[k].kind == 0 && lanes[k] != 2 && lanes[k] != 4 && lanes[k] != 8)
      return snap_fail_msg(SNAP_ERR_INVALID_ARG, "lanes per slice must be 2, 4 or 8");
  for (size_t k = 0; k < b->groups.size(); ++k)
    if (b->groups[k].kind == 0) b->groups[k].lps = lanes[k];
  if (!b->groups.empty() && cudaMemcpy(b->d_groups, b->groups.data(),
                                       sizeof(GroupRec) * b->groups.size(),
                                       cudaMemcpyHostToDevice) != cudaSuccess)
    return snap_fail_msg(SNAP_ERR_CUDA, "upload of the group table failed");
  return SNAP_OK;
}

snap_status launch_batch(snap_batch *b, const snap_options &o, unsigned long long *t_ns,
                         void *ws, size_t bytes, cudaStream_t s) {
  if (!b->bound) return snap_fail_msg(SNAP_ERR_NOT_READY, "batch used before snap_batch_bind");
  if (b->n_inst == 0) return SNAP_OK;
  if (!ws || bytes < batch_ws_bytes(b) || !aligned(ws, 256))
    return snap_fail_msg(SNAP_ERR_WORKSPACE, "batch workspace missing, unaligned or too small");
  char *c = (char *)ws;
  BatchArgs a;
  a.inst = b->d_inst;
  a.groups = b->d_groups;
  a.list = b->d_list;
  a.items1d = b->d_items1d;
  a.items2d = b->d_items2d;
  a.n1d = b->n1d;
  a.n2d = b->n2d;
  a.order = b->sched.order;
  a.hdr = (Hdr *)c;
  a.done = (unsigned int *)(c + sizeof(Hdr));
  a.negstart = (unsigned long long *)(c + snap_align256(sizeof(Hdr) + sizeof(unsigned) * (size_t)b->n_inst));
  a.bst = (BlockStat *)(c + hdr_bytes(b));
  a.t_ns = t_ns;
  a.o = solver_opts(o);
  a.so_f = slice_opts<float>(a.o, a.o.tol_kkt);
  a.so_d = slice_opts<df64>(a.o, a.o.tol_kkt);
  cudaError_t e = cudaMemsetAsync(ws, 0, hdr_bytes(b), s);
  if (e != cudaSuccess) return snap_fail_msg(SNAP_ERR_CUDA, cudaGetErrorString(e));
  k_batch<<<b->grid, kThreads, b->smem_bytes, s>>>(a);
  snap_note_launch(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return snap_fail_msg(SNAP_ERR_CUDA, cudaGetErrorString(e));
  return SNAP_OK;
}

snap_status launch_batch_bwd(snap_batch *b, void *ws, size_t bytes, cudaStream_t s) {
  if (!b->bound || !b->bound_bwd)
    return snap_fail_msg(SNAP_ERR_NOT_READY, "batch adjoint used before snap_batch_bind(_backward)");
  if (b->n_inst == 0) return SNAP_OK;
  if (!ws || bytes < batch_ws_bytes(b) || !aligned(ws, 256))
    return snap_fail_msg(SNAP_ERR_WORKSPACE, "batch workspace missing, unaligned or too small");
  char *c = (char *)ws;
  BwdArgs a;
  a.inst = b->d_inst;
  a.bwd = b->d_bwd;
  a.groups = b->d_groups;
  a.list = b->d_list;
  a.items1d = b->d_items1d;
  a.items2d = b->d_items2d;
  a.n1d = b->n1d;
  a.n2d = b->n2d;
  a.order = b->sched.order;
  a.hdr = (Hdr *)c;
  a.done = (unsigned int *)(c + sizeof(Hdr));
  // per-slice / per-frame contributions in the statistics area (32 of its 40 bytes a record)
  a.contrib = (BwdContrib *)(c + hdr_bytes(b));
  static_assert(sizeof(BwdContrib) <= sizeof(BlockStat), "contributions fit the statistics area");
  cudaError_t e = cudaMemsetAsync(ws, 0, hdr_bytes(b), s);
  if (e != cudaSuccess) return snap_fail_msg(SNAP_ERR_CUDA, cudaGetErrorString(e));
  k_batch_bwd<<<b->grid_bwd, kThreads, b->smem_bytes, s>>>(a);
  snap_note_launch(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return snap_fail_msg(SNAP_ERR_CUDA, cudaGetErrorString(e));
  return SNAP_OK;
}

}  // namespace

extern "C" {

SNAP_API snap_status snap_batch_create(int n_problems, const snap_problem_t *probs, int n_inst,
                                       const int *inst_problem, snap_batch_t *out) {
  if (!out || n_problems < 1 || !probs || n_inst < 0 || (n_inst > 0 && !inst_problem))
    return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null arrays or bad counts");
  *out = nullptr;
  for (int i = 0; i < n_problems; ++i) {
    if (!probs[i]) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null problem in the list");
    const int f = probs[i]->desc.family;
    if (f != SNAP_FAMILY_A_MASS_ENERGY && f != SNAP_FAMILY_B_BURGERS_BOUNDARY &&
        f != SNAP_FAMILY_C_DIV_ENERGY)
      return snap_fail_msg(SNAP_ERR_UNSUPPORTED, "uneven batches take families A, B and C");
  }
  for (int i = 0; i < n_inst; ++i)
    if (inst_problem[i] < 0 || inst_problem[i] >= n_problems)
      return snap_fail_msg(SNAP_ERR_INVALID_ARG, "instance problem index out of range");
  snap_batch *b = new snap_batch;
  cudaGetDevice(&b->device);
  b->n_inst = n_inst;
  b->probs.assign(probs, probs + n_problems);
  b->inst_problem.assign(inst_problem, inst_problem + n_inst);
  std::vector<int> gid(n_problems, -1);
  for (int i = 0; i < n_inst; ++i) {
    const int pi = inst_problem[i];
    if (gid[pi] < 0) {
      gid[pi] = (int)b->group_problem.size();
      b->group_problem.push_back(pi);
      b->group_inst.emplace_back();
    }
    b->group_inst[gid[pi]].push_back(i);
  }
  // groups in problem order (stable, independent of instance order)
  std::vector<int> perm(b->group_problem.size());
  for (size_t i = 0; i < perm.size(); ++i) perm[i] = (int)i;
  std::sort(perm.begin(), perm.end(),
            [&](int x, int y) { return b->group_problem[x] < b->group_problem[y]; });
  std::vector<int> gp;
  std::vector<std::vector<int>> gi;
  for (int x : perm) { gp.push_back(b->group_problem[x]); gi.push_back(b->group_inst[x]); }
  b->group_problem = gp;
  b->group_inst = gi;
  size_t cap1_packed = 0, cap1_split = 0, cap2 = 0;
  for (size_t k = 0; k < gp.size(); ++k) {
    const snap_problem *p = probs[gp[k]];
    GroupRec G;
    memset(&G, 0, sizeof(G));
    G.n_inst = (int)gi[k].size();
    G.nt = p->desc.nt;
    G.list_off = (int)b->list.size();
    G.bst_off = b->n_blocks;
    for (int id : gi[k]) b->list.push_back(id);
    if ((long long)G.n_inst * G.nt >= (1LL << 31)) {
      delete b;
      return snap_fail_msg(SNAP_ERR_INVALID_ARG, "a group holds 2^31 or more slices / frames");
    }
    b->n_blocks += (long long)G.n_inst * G.nt;
    if (p->desc.family == SNAP_FAMILY_C_DIV_ENERGY) {
      // the batch kernel holds the frame code for the power-of-two sides only
      const int side = p->desc.nx;
      if (side != 4 && side != 8 && side != 16 && side != 32 && side != 64) {
        delete b;
        return snap_fail_msg(SNAP_ERR_UNSUPPORTED,
                             "uneven batches take 2-D grid sides 4, 8, 16, 32 and 64 only");
      }
      G.kind = 1;
      G.M = p->desc.nx / 2;
      if (ensure_2d_factor(p) != cudaSuccess) {
        delete b;
        return snap_fail_msg(SNAP_ERR_CUDA, "upload of a 2-D factor failed");
      }
      G.Q = (const float *)p->dev_const;
      G.I = G.Q + (size_t)G.M * G.M;
      b->max_m = std::max(b->max_m, G.M);
      cap2 += (size_t)G.n_inst * G.nt;
    } else {
      G.kind = 0;
      G.g = p->g1;
      G.dxd = df64(p->g1.dx);
      // the smallest item size (16 slices) gives the most items
      cap1_packed += ((size_t)G.n_inst * G.nt + 15) / 16;
      cap1_split += (size_t)G.n_inst * ((G.nt + 15) / 16);
      G.lps = 4;
    }
    const size_t wsg = (p->desc.family == SNAP_FAMILY_C_DIV_ENERGY) ? ws_bytes_2d(p, G.n_inst)
                                                                     : ws_bytes_1d(p, G.n_inst);
    b->grouped_ws = std::max(b->grouped_ws, wsg);
    b->groups.push_back(G);
  }
  switch (b->max_m) {
    case 0: b->smem_bytes = 0; break;
    case 2: b->smem_bytes = Smem2D<2>::bytes; break;
    case 4: b->smem_bytes = Smem2D<4>::bytes; break;
    case 8: b->smem_bytes = Smem2D<8>::bytes; break;
    case 16: b->smem_bytes = Smem2D<16>::bytes; break;
    default: b->smem_bytes = Smem2D<32>::bytes; break;
  }
  b->cap1d = std::max(cap1_packed, cap1_split);
  b->cap2d = cap2;
  bool ok = cudaMalloc(&b->d_inst, sizeof(InstRec) * std::max(n_inst, 1)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_groups, sizeof(GroupRec) * std::max<size_t>(b->groups.size(), 1)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_list, sizeof(int) * std::max<size_t>(b->list.size(), 1)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_items1d, sizeof(Item1D) * std::max<size_t>(b->cap1d, 1)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_items2d, sizeof(Item2D) * std::max<size_t>(b->cap2d, 1)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_bwd, sizeof(BwdRec) * std::max(n_inst, 1)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_batch(b);
    return snap_fail_msg(SNAP_ERR_NO_MEMORY, "device allocation of the batch tables failed");
  }
  if ((!b->groups.empty() && cudaMemcpy(b->d_groups, b->groups.data(), sizeof(GroupRec) * b->groups.size(),
                                        cudaMemcpyHostToDevice) != cudaSuccess) ||
      (!b->list.empty() && cudaMemcpy(b->d_list, b->list.data(), sizeof(int) * b->list.size(),
                                      cudaMemcpyHostToDevice) != cudaSuccess)) {
    free_batch(b);
    return snap_fail_msg(SNAP_ERR_CUDA, "upload of the batch tables failed");
  }
  if (b->smem_bytes > 0 &&
      (cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)b->smem_bytes) != cudaSuccess ||
       cudaFuncSetAttribute(k_batch_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)b->smem_bytes) != cudaSuccess)) {
    free_batch(b);
    return snap_fail_msg(SNAP_ERR_CUDA, "shared-memory size of the batch kernel refused");
  }
  const snap_status st = upload_items(b);
  if (st != SNAP_OK) {
    free_batch(b);
    return st;
  }
  *out = b;
  return SNAP_OK;
}

SNAP_API void snap_batch_destroy(snap_batch_t b) {
  if (b) free_batch(b);
}

SNAP_API snap_status snap_batch_bind(snap_batch_t b, const double *const *u_hat,
                                     const double *const *params, double *const *u,
                                     double *const *lambda, snap_stats *const *stats) {
  if (!b) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null batch");
  if (b->n_inst > 0 && (!u_hat || !params || !u || !lambda || !stats))
    return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null pointer table");
  std::vector<InstRec> rec(b->n_inst);
  char msg[128];
  for (int i = 0; i < b->n_inst; ++i) {
    const snap_problem *p = b->probs[b->inst_problem[i]];
    const bool one_d = p->desc.family != SNAP_FAMILY_C_DIV_ENERGY;
    const unsigned va = one_d ? 16u : 8u;
    if (!u_hat[i] || !params[i] || !u[i] || !lambda[i] || !stats[i] || !aligned(u_hat[i], va) ||
        !aligned(u[i], va) || !aligned(params[i], 8) || !aligned(lambda[i], 8) ||
        !aligned(stats[i], 8)) {
      snprintf(msg, sizeof(msg), "instance %d: null or misaligned buffer", i);
      return snap_fail_msg(SNAP_ERR_INVALID_ARG, msg);
    }
    rec[i] = InstRec{u_hat[i], params[i], u[i], lambda[i], stats[i]};
  }
  if (b->n_inst > 0 &&
      cudaMemcpy(b->d_inst, rec.data(), sizeof(InstRec) * rec.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return snap_fail_msg(SNAP_ERR_CUDA, "upload of the pointer table failed");
  // contiguity per group (the grouped baseline launches snap_project on the group's block)
  b->group_contig.assign(b->groups.size(), 1);
  for (size_t k = 0; k < b->groups.size(); ++k) {
    const snap_problem *p = b->probs[b->group_problem[k]];
    const auto &ids = b->group_inst[k];
    for (size_t j = 1; j < ids.size(); ++j) {
      const InstRec &x = rec[ids[j - 1]], &y = rec[ids[j]];
      if (y.uh != x.uh + p->info.n_vars || y.u != x.u + p->info.n_vars ||
          y.params != x.params + p->info.n_params || y.lam != x.lam + p->info.n_rows_nominal ||
          y.stats != x.stats + 1)
        b->group_contig[k] = 0;
    }
  }
  b->h_inst = rec;
  b->bound = true;
  return SNAP_OK;
}

SNAP_API snap_status snap_batch_workspace_size(snap_batch_t b, size_t *bytes) {
  if (!b || !bytes) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null argument");
  *bytes = batch_ws_bytes(b);
  return SNAP_OK;
}

SNAP_API snap_status snap_batch_project(snap_batch_t b, const snap_options *opt,
                                        unsigned long long *t_ns, void *workspace,
                                        size_t workspace_bytes, snap_stream_t stream) {
  if (!b) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null batch");
  snap_options o;
  if (get_opts(opt, o) != SNAP_OK) return SNAP_ERR_INVALID_ARG;
  return launch_batch(b, o, t_ns, workspace, workspace_bytes, (cudaStream_t)stream);
}

SNAP_API snap_status snap_batch_project_grouped(snap_batch_t b, const snap_options *opt,
                                                void *workspace, size_t workspace_bytes,
                                                snap_stream_t stream) {
  if (!b) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null batch");
  if (!b->bound) return snap_fail_msg(SNAP_ERR_NOT_READY, "batch used before snap_batch_bind");
  snap_options o;
  if (get_opts(opt, o) != SNAP_OK) return SNAP_ERR_INVALID_ARG;
  if (b->n_inst == 0) return SNAP_OK;
  if (!workspace || workspace_bytes < batch_ws_bytes(b) || !aligned(workspace, 256))
    return snap_fail_msg(SNAP_ERR_WORKSPACE, "batch workspace missing, unaligned or too small");
  for (size_t k = 0; k < b->groups.size(); ++k)
    if (!b->group_contig[k])
      return snap_fail_msg(SNAP_ERR_UNSUPPORTED,
                           "grouped launches need each group's buffers contiguous");
  const SolverOpts so = solver_opts(o);
  for (size_t k = 0; k < b->groups.size(); ++k) {
    const snap_problem *p = b->probs[b->group_problem[k]];
    const InstRec &r = b->h_inst[b->group_inst[k][0]];
    const int n = (int)b->group_inst[k].size();
    cudaError_t e;
    if (p->desc.family == SNAP_FAMILY_C_DIV_ENERGY)
      e = launch_2d_forward(p, n, r.uh, r.params, nullptr, r.u, r.lam, r.stats, so,
                            SNAP_PATH_MIXED, workspace, (cudaStream_t)stream);
    else
      e = launch_1d_forward(p, n, r.uh, r.params, nullptr, r.u, r.lam, r.stats, so,
                            SNAP_PATH_MIXED, workspace, (cudaStream_t)stream);
    if (e != cudaSuccess) return snap_fail_msg(SNAP_ERR_CUDA, cudaGetErrorString(e));
  }
  return SNAP_OK;
}

SNAP_API snap_status snap_batch_get_schedule(snap_batch_t b, snap_batch_schedule *s) {
  if (!b || !s) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null argument");
  *s = b->sched;
  return SNAP_OK;
}

SNAP_API snap_status snap_batch_set_schedule(snap_batch_t b, const snap_batch_schedule *s) {
  if (!b || !s) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null argument");
  if (s->ctas_per_sm < 1 || s->ctas_per_sm > 2 || s->order < 0 || s->order > 1 ||
      s->pack_1d < 0 || s->pack_1d > 1 || s->sort_1d < 0 || s->sort_1d > 1 ||
      (s->tile_1d != 16 && s->tile_1d != 32 && s->tile_1d != 64) ||
      (s->lanes_1d != 0 && s->lanes_1d != 2 && s->lanes_1d != 4 && s->lanes_1d != 8))
    return snap_fail_msg(SNAP_ERR_INVALID_ARG, "schedule field out of range");
  if (s->lanes_1d != 0) {
    std::vector<int> lanes(b->groups.size());
    for (size_t k = 0; k < lanes.size(); ++k) lanes[k] = b->groups[k].kind == 0 ? s->lanes_1d : 0;
    const snap_status st = set_group_lanes(b, lanes.data());
    if (st != SNAP_OK) return st;
  }
  const snap_batch_schedule old = b->sched;
  b->sched = *s;
  const snap_status st = upload_items(b);
  if (st != SNAP_OK) b->sched = old;
  return st;
}

SNAP_API snap_status snap_batch_get_group_lanes(snap_batch_t b, int *lanes) {
  if (!b || !lanes) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null argument");
  for (size_t k = 0; k < b->groups.size(); ++k)
    lanes[k] = b->groups[k].kind == 0 ? b->groups[k].lps : 0;
  return SNAP_OK;
}

SNAP_API snap_status snap_batch_set_group_lanes(snap_batch_t b, const int *lanes) {
  if (!b || !lanes) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null argument");
  return set_group_lanes(b, lanes);
}

SNAP_API snap_status snap_batch_autotune(snap_batch_t b, const snap_options *opt, void *workspace,
                                         size_t workspace_bytes, snap_stream_t stream, int reps,
                                         snap_batch_schedule *best, double *best_ms) {
  if (!b) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null batch");
  if (reps < 1 || reps > 1000) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "reps must be in [1, 1000]");
  snap_options o;
  if (get_opts(opt, o) != SNAP_OK) return SNAP_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return snap_fail_msg(SNAP_ERR_CUDA, "event create");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return snap_fail_msg(SNAP_ERR_CUDA, "event create");
  }
  // best of `reps` timed launches of the batch as it is now set up (after one warm-up)
  auto time_now = [&](double &t) -> snap_status {
    snap_status st = launch_batch(b, o, nullptr, workspace, workspace_bytes, s);
    t = 1e300;
    for (int r = 0; r < reps && st == SNAP_OK; ++r) {
      cudaEventRecord(e0, s);
      st = launch_batch(b, o, nullptr, workspace, workspace_bytes, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess)
        return snap_fail_msg(SNAP_ERR_CUDA, "autotune timing failed");
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      t = std::min(t, (double)ms);
    }
    return st;
  };
  const size_t ng = b->groups.size();
  std::vector<int> lanes(ng), best_lanes(ng);
  for (size_t k = 0; k < ng; ++k) lanes[k] = b->groups[k].kind == 0 ? 4 : 0;
  snap_status st = set_group_lanes(b, lanes.data());
  best_lanes = lanes;
  snap_batch_schedule bestS = b->sched;
  double bestT = 1e300;
  // stage 1: queue order and occupancy (32-slice items, 4 lanes per slice)
  for (int cps = 1; cps <= 2 && st == SNAP_OK; ++cps)
    for (int order = 0; order <= 1 && st == SNAP_OK; ++order)
      for (int pack = 0; pack <= 1 && st == SNAP_OK; ++pack)
        for (int sort = 0; sort <= 1 && st == SNAP_OK; ++sort) {
          const snap_batch_schedule cand{cps, order, pack, sort, 32, 0};
          st = snap_batch_set_schedule(b, &cand);
          double t = 1e300;
          if (st == SNAP_OK) st = time_now(t);
          if (st == SNAP_OK && t < bestT) {
            bestT = t;
            bestS = cand;
          }
        }
  // stage 2: slices per 1-D item
  for (int tile : {16, 64}) {
    if (st != SNAP_OK) break;
    snap_batch_schedule cand = bestS;
    cand.tile_1d = tile;
    st = snap_batch_set_schedule(b, &cand);
    double t = 1e300;
    if (st == SNAP_OK) st = time_now(t);
    if (st == SNAP_OK && t < bestT) {
      bestT = t;
      bestS = cand;
    }
  }
  if (st == SNAP_OK) st = snap_batch_set_schedule(b, &bestS);
  // stage 3: lanes per slice, one 1-D group at a time (coordinate descent from 4)
  for (size_t k = 0; k < ng && st == SNAP_OK; ++k) {
    if (b->groups[k].kind != 0) continue;
    for (int l : {2, 8}) {
      lanes = best_lanes;
      lanes[k] = l;
      st = set_group_lanes(b, lanes.data());
      double t = 1e300;
      if (st == SNAP_OK) st = time_now(t);
      if (st != SNAP_OK) break;
      if (t < bestT) {
        bestT = t;
        best_lanes = lanes;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SNAP_OK) return st;
  st = snap_batch_set_schedule(b, &bestS);
  if (st == SNAP_OK) st = set_group_lanes(b, best_lanes.data());
  if (st != SNAP_OK) return st;
  if (best) *best = bestS;
  if (best_ms) *best_ms = bestT;
  return SNAP_OK;
}

SNAP_API snap_status snap_batch_capture_graph(snap_batch_t b, const snap_options *opt,
                                              unsigned long long *t_ns, void *workspace,
                                              size_t workspace_bytes) {
  if (!b) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null batch");
  snap_options o;
  if (get_opts(opt, o) != SNAP_OK) return SNAP_ERR_INVALID_ARG;
  if (!b->bound) return snap_fail_msg(SNAP_ERR_NOT_READY, "batch used before snap_batch_bind");
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    return snap_fail_msg(SNAP_ERR_CUDA, "stream create");
  cudaGraph_t g = nullptr;
  snap_status st = SNAP_OK;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    st = snap_fail_msg(SNAP_ERR_CUDA, "begin capture");
  } else {
    st = launch_batch(b, o, t_ns, workspace, workspace_bytes, s);
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st == SNAP_OK && e != cudaSuccess) st = snap_fail_msg(SNAP_ERR_CUDA, "end capture");
  }
  cudaGraphExec_t x = nullptr;
  if (st == SNAP_OK && g && cudaGraphInstantiate(&x, g, 0) != cudaSuccess)
    st = snap_fail_msg(SNAP_ERR_CUDA, "graph instantiate");
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(s);
  if (st != SNAP_OK) return st;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = x;
  return SNAP_OK;
}

SNAP_API snap_status snap_batch_launch_graph(snap_batch_t b, snap_stream_t stream) {
  if (!b) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null batch");
  if (b->n_inst == 0) return SNAP_OK;
  if (!b->graph) return snap_fail_msg(SNAP_ERR_NOT_READY, "no graph captured");
  const cudaError_t e = cudaGraphLaunch(b->graph, (cudaStream_t)stream);
  if (e != cudaSuccess) return snap_fail_msg(SNAP_ERR_CUDA, cudaGetErrorString(e));
  snap_note_launch(1);
  return SNAP_OK;
}

SNAP_API snap_status snap_batch_bind_backward(snap_batch_t b, const double *const *grad_u,
                                              double *const *grad_u_hat,
                                              double *const *grad_params) {
  if (!b) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null batch");
  if (b->n_inst > 0 && (!grad_u || !grad_u_hat))
    return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null pointer table");
  std::vector<BwdRec> rec(b->n_inst);
  char msg[128];
  for (int i = 0; i < b->n_inst; ++i) {
    const snap_problem *p = b->probs[b->inst_problem[i]];
    const unsigned va = p->desc.family != SNAP_FAMILY_C_DIV_ENERGY ? 16u : 8u;
    double *gp = grad_params ? grad_params[i] : nullptr;
    if (!grad_u[i] || !grad_u_hat[i] || !aligned(grad_u[i], va) || !aligned(grad_u_hat[i], va) ||
        (gp && !aligned(gp, 8))) {
      snprintf(msg, sizeof(msg), "instance %d: null or misaligned adjoint buffer", i);
      return snap_fail_msg(SNAP_ERR_INVALID_ARG, msg);
    }
    rec[i] = BwdRec{grad_u[i], grad_u_hat[i], gp};
  }
  if (b->n_inst > 0 &&
      cudaMemcpy(b->d_bwd, rec.data(), sizeof(BwdRec) * rec.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return snap_fail_msg(SNAP_ERR_CUDA, "upload of the adjoint pointer table failed");
  b->group_contig_bwd.assign(b->groups.size(), 1);
  for (size_t k = 0; k < b->groups.size(); ++k) {
    const snap_problem *p = b->probs[b->group_problem[k]];
    const auto &ids = b->group_inst[k];
    for (size_t j = 1; j < ids.size(); ++j) {
      const BwdRec &x = rec[ids[j - 1]], &y = rec[ids[j]];
      if (y.gu != x.gu + p->info.n_vars || y.gh != x.gh + p->info.n_vars ||
          (x.gp == nullptr) != (y.gp == nullptr) || (x.gp && y.gp != x.gp + p->info.n_params))
        b->group_contig_bwd[k] = 0;
    }
  }
  b->h_bwd = rec;
  b->bound_bwd = true;
  return SNAP_OK;
}

SNAP_API snap_status snap_batch_project_backward(snap_batch_t b, void *workspace,
                                                 size_t workspace_bytes, snap_stream_t stream) {
  if (!b) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null batch");
  return launch_batch_bwd(b, workspace, workspace_bytes, (cudaStream_t)stream);
}

SNAP_API snap_status snap_batch_project_backward_grouped(snap_batch_t b, void *workspace,
                                                         size_t workspace_bytes,
                                                         snap_stream_t stream) {
  if (!b) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null batch");
  if (!b->bound || !b->bound_bwd)
    return snap_fail_msg(SNAP_ERR_NOT_READY, "batch adjoint used before snap_batch_bind(_backward)");
  if (b->n_inst == 0) return SNAP_OK;
  if (!workspace || workspace_bytes < batch_ws_bytes(b) || !aligned(workspace, 256))
    return snap_fail_msg(SNAP_ERR_WORKSPACE, "batch workspace missing, unaligned or too small");
  for (size_t k = 0; k < b->groups.size(); ++k)
    if (!b->group_contig[k] || !b->group_contig_bwd[k])
      return snap_fail_msg(SNAP_ERR_UNSUPPORTED,
                           "grouped launches need each group's buffers contiguous");
  for (size_t k = 0; k < b->groups.size(); ++k) {
    const snap_problem *p = b->probs[b->group_problem[k]];
    const int id0 = b->group_inst[k][0];
    const InstRec &r = b->h_inst[id0];
    const BwdRec &w = b->h_bwd[id0];
    const int n = (int)b->group_inst[k].size();
    cudaError_t e;
    if (p->desc.family == SNAP_FAMILY_C_DIV_ENERGY)
      e = launch_2d_backward(p, n, w.gu, r.u, r.lam, r.params, r.stats, w.gh, w.gp, workspace,
                             (cudaStream_t)stream);
    else
      e = launch_1d_backward(p, n, w.gu, r.u, r.lam, r.params, r.stats, w.gh, w.gp, workspace,
                             (cudaStream_t)stream);
    if (e != cudaSuccess) return snap_fail_msg(SNAP_ERR_CUDA, cudaGetErrorString(e));
  }
  return SNAP_OK;
}

SNAP_API snap_status snap_batch_capture_graph_backward(snap_batch_t b, void *workspace,
                                                       size_t workspace_bytes) {
  if (!b) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null batch");
  if (!b->bound || !b->bound_bwd)
    return snap_fail_msg(SNAP_ERR_NOT_READY, "batch adjoint used before snap_batch_bind(_backward)");
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    return snap_fail_msg(SNAP_ERR_CUDA, "stream create");
  cudaGraph_t g = nullptr;
  snap_status st = SNAP_OK;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    st = snap_fail_msg(SNAP_ERR_CUDA, "begin capture");
  } else {
    st = launch_batch_bwd(b, workspace, workspace_bytes, s);
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st == SNAP_OK && e != cudaSuccess) st = snap_fail_msg(SNAP_ERR_CUDA, "end capture");
  }
  cudaGraphExec_t x = nullptr;
  if (st == SNAP_OK && g && cudaGraphInstantiate(&x, g, 0) != cudaSuccess)
    st = snap_fail_msg(SNAP_ERR_CUDA, "graph instantiate");
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(s);
  if (st != SNAP_OK) return st;
  if (b->graph_bwd) cudaGraphExecDestroy(b->graph_bwd);
  b->graph_bwd = x;
  return SNAP_OK;
}

SNAP_API snap_status snap_batch_launch_graph_backward(snap_batch_t b, snap_stream_t stream) {
  if (!b) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null batch");
  if (b->n_inst == 0) return SNAP_OK;
  if (!b->graph_bwd) return snap_fail_msg(SNAP_ERR_NOT_READY, "no adjoint graph captured");
  const cudaError_t e = cudaGraphLaunch(b->graph_bwd, (cudaStream_t)stream);
  if (e != cudaSuccess) return snap_fail_msg(SNAP_ERR_CUDA, cudaGetErrorString(e));
  snap_note_launch(1);
  return SNAP_OK;
}

SNAP_API snap_status snap_batch_info(snap_batch_t b, int *n_groups, int *n_tiles_1d,
                                     int *n_frames_2d) {
  if (!b) return snap_fail_msg(SNAP_ERR_INVALID_ARG, "null batch");
  if (n_groups) *n_groups = (int)b->groups.size();
  if (n_tiles_1d) *n_tiles_1d = b->n1d;
  if (n_frames_2d) *n_frames_2d = b->n2d;
  return SNAP_OK;
}

}  // extern "C"
