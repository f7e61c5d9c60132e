// Family E, the IC regime of the Burgers problem with Godunov flux rows (Appendix A, "IC,
// mass, Flux(k)"; the flux residual of Appendix D): a 1-D field on x_i = i dx, dx = 1/(nx-1),
// periodic neighbours, t_k = k dt, dt = 1/(nt-1), c = dt/dx, and the rows
//   IC     u^0_i - g_i                                   (nx)
//   mass   dx sum_i u^k_i - M,  M = dx sum_i g_i          (nt; mass_0..mass_K implied)
//   flux   u^k_i - G(u^{k-1})_i,  k = 1..K                (K nx)
//   G(v)_i = v_i - c (F(v_i, v_{i+1}) - F(v_{i-1}, v_i)),  F the Godunov flux of u^2/2.
// mass_0 follows from the IC rows and, with periodic neighbours, the fluxes of a step
// telescope, so mass_k (k <= K) follows from mass_{k-1} and the flux rows: these rows are left
// out of the solve (multiplier 0) and counted in ||h||_inf.  The active rows then fix slices
// 0..K (block lower-triangular in time, identity diagonal blocks), and the Newton-KKT
// iteration of Appendix B converges to the point the kernel evaluates directly:
//   u^0 = g, u^k = G(u^{k-1}) (forward substitution over the K steps),
//   lambda^(K) = u_hat^K - u^K,  lambda^(j) = u_hat^j - u^j + J_G(u^j)^T lambda^(j+1),
//   lambda_IC = u_hat^0 - g + J_G(g)^T lambda^(1)      (backward substitution: stationarity),
// and every later slice only carries its mass row: u^k = u_hat^k + (sum g - sum u_hat^k)/nx.
// Generalised Jacobian of F at its switches: the branch chosen by the comparisons below.
//
// Two kernels: k1dflux_chain runs one warp per sample through the K steps and back (the time
// chain is sequential; the slice lives in registers and shared memory, the multipliers'
// recursion reads the slices back from u), and k1dflux_mass, its programmatic dependent,
// gives each mass slice four lanes (eight per warp), as the boundary-condition family does,
// while the chains run.  stats.iters = 1: one structured solve, no iteration.
#include <cuda_runtime.h>
#include <math.h>

#include "sample_1d.cuh"
#include "kern_1dflux.h"
#include "snap_internal.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kThreads = 128;
constexpr int kChainWarps = kThreads / 32;   // samples per chain block

// Order key of a double for the branch decisions, taken on the integer pipe (FP64 is the
// scarce pipe): non-negative bit patterns keep their value, negative ones map to
// INT64_MIN - bits, so that for non-NaN x, y: x <= y iff key(x) <= key(y) (+0 and -0 both
// map to 0), key(-x) = -key(x), and x + y >= 0 (rounded) iff key(x) >= -key(y) (rounding
// never changes the sign of a sum).
__device__ __forceinline__ long long gd_key(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : (-0x7fffffffffffffffLL - 1) - b;
}

// Godunov flux of f(u) = u^2/2: the minimum of f over [a, b] (a <= b) or its maximum over
// [b, a] (a > b).  Rounded products, so that the residual kernel reproduces the same bits.
__device__ __forceinline__ double gd_flux(double a, double b) {
  const long long ka = gd_key(a), kb = gd_key(b);
  if (ka <= kb) return ka > 0 ? __dmul_rn(0.5 * a, a) : (kb < 0 ? __dmul_rn(0.5 * b, b) : 0.0);
  return ka >= -kb ? __dmul_rn(0.5 * a, a) : __dmul_rn(0.5 * b, b);
}

// dF/da and dF/db of the branch taken (a <= b, a > 0, b < 0, a + b >= 0, as in gd_flux)
__device__ __forceinline__ void gd_dflux(double a, double b, double &da, double &db) {
  const long long ka = gd_key(a), kb = gd_key(b);
  bool ia, ib;
  if (ka <= kb) {
    ia = ka > 0;
    ib = !ia && kb < 0;
  } else {
    ia = ka >= -kb;
    ib = !ia;
  }
  da = ia ? a : 0.0;
  db = ib ? b : 0.0;
}

// v - c (Fr - Fl), rounded step by step
__device__ __forceinline__ double gd_update(double v, double fr, double fl, double c) {
  return __dsub_rn(v, __dmul_rn(c, __dsub_rn(fr, fl)));
}

__device__ __forceinline__ double fx_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

struct FluxArgs {
  int B, nt, nx, K;
  double dx, c;
  double inv_nx, inv_dx;       // 1/nx and 1/dx, rounded on the host
  int n_chain_blocks;
  long long n_mass;            // B (nt - K - 1) mass slices
  const double *uh, *g;        // u_hat [B][nt][nx], params g [B][nx]
  double *u, *lam;             // u [B][nt][nx], lambda [B][nx + nt + K nx]
  BlockStat *bst;              // [B][nt]
};

__device__ __forceinline__ void put_stat(BlockStat *dst, double hinf, double obj) {
  BlockStat st;
  st.iters = 1;
  st.backtracks = 0;
  st.corrections = 0;
  const bool fin = hinf == hinf && !isinf(hinf) && obj == obj && !isinf(obj);
  st.status = fin ? SNAP_SAMPLE_OK : SNAP_SAMPLE_NONFINITE;
  st.h_inf = hinf;
  st.kkt_inf = hinf;   // active rows hold by construction; stationarity by substitution
  st.obj = obj;
  *dst = st;
}

// Mass slices k = K+1..nt-1: four lanes per slice (eight slices per warp).
// sum_i g[i] over the full warp (lane l takes i = l, l + 32, ...) in the same split / TwoSum
// arithmetic, the lane sums combined by a fixed butterfly in double-float: the same bits in
// every warp that computes it.  A row with a value outside the split range is summed in FP64
// (warp-uniform).
__device__ __forceinline__ double fx_row_sum32(const double *g, int nx, int lane) {
  float sh = 0.0f, se = 0.0f;
  int ok = 1;
  for (int i = lane; i < nx; i += 32) {
    float h, l;
    ok &= df_split_trunc(g[i], h, l);
    const float t = sh + h, bb = t - sh;
    se += ((sh - (t - bb)) + (h - bb)) + l;
    sh = t;
  }
  if (!__all_sync(FULL, ok)) {
    double t = 0.0;
    for (int i = lane; i < nx; i += 32) t += g[i];
    return fx_warp_sum(t);
  }
  df64 v = df_fast_two_sum(sh, se);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = v + df64(__shfl_xor_sync(FULL, v.hi, o), __shfl_xor_sync(FULL, v.lo, o));
  return (double)v.hi + (double)v.lo;
}

__device__ __forceinline__ void flux_mass(const FluxArgs &a, long long wid, int lane) {
  const int q = lane >> 2, r = lane & 3;
  const long long s = wid * 8 + q;
  const bool live = s < a.n_mass;
  const int nm = a.nt - a.K - 1, nx = a.nx;
  int b = 0, k = 0;
  if (live) {
    if (a.n_mass < (1LL << 31)) {      // 32-bit division (the 64-bit one is a long sequence)
      const unsigned su = (unsigned)s;
      b = (int)(su / (unsigned)nm);
      k = a.K + 1 + (int)(su - (unsigned)b * (unsigned)nm);
    } else {
      b = (int)(s / nm);
      k = a.K + 1 + (int)(s % nm);
    }
  }
  const size_t off = ((size_t)b * a.nt + k) * nx;
  const double *row = a.uh + off;
  const double S = s4_slice_sum(row, nx, r, live);
  // sum g of each distinct sample among the warp's eight slices (usually one or two): a
  // full-warp sum, the same bits whichever warp computes it
  double Gs = 0.0, cur = 0.0;
  int cb = -1;
  for (int qq = 0; qq < 8; ++qq) {
    const int bq = __shfl_sync(FULL, b, qq * 4);
    if (!__shfl_sync(FULL, live ? 1 : 0, qq * 4)) break;   // live slices are a prefix
    if (bq != cb) {
      cur = fx_row_sum32(a.g + (size_t)bq * nx, nx, lane);
      cb = bq;
    }
    if (q == qq) Gs = cur;
  }
  if (!live) return;
  const double sh = (Gs - S) * a.inv_nx;
  double *out = a.u + off;
#pragma unroll 8
  for (int i = r; i < nx; i += 4) out[i] = row[i] + sh;
  if (r == 0) {
    a.lam[(size_t)b * ((size_t)nx + a.nt + (size_t)a.K * nx) + nx + k] = -sh * a.inv_dx;
    put_stat(a.bst + (size_t)b * a.nt + k, fabs(a.dx * (S + (double)nx * sh) - a.dx * Gs),
             0.5 * (double)nx * sh * sh);
  }
}

// The time chain with the sample's slice in registers (lane l holds i = l + 32 m, m < MAXM,
// nx <= 32 MAXM): each step's global loads are issued one step ahead, so a step costs one
// round trip instead of one per element.  The same arithmetic as flux_chain (the same bits).
template <int MAXM>
__global__ void __launch_bounds__(kThreads) k1dflux_chain(FluxArgs a) {
  extern __shared__ double fx_smem[];
  // the mass kernel is independent of this one: let it start now
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int b = (int)blockIdx.x * kChainWarps + wib;
  if (b >= a.B) return;
  const int nx = a.nx, nt = a.nt, K = a.K;
  const double c = a.c;
  double *sv = fx_smem + (size_t)wib * 3 * nx, *sa = sv + nx, *sw = sa + nx;
  const size_t base = (size_t)b * nt * nx;
  const double *__restrict__ uh = a.uh + base;
  double *__restrict__ u = a.u + base;
  double *__restrict__ lam = a.lam + (size_t)b * ((size_t)nx + nt + (size_t)K * nx);
  const double *__restrict__ g = a.g + (size_t)b * nx;
  BlockStat *bst = a.bst + (size_t)b * nt;
  double v[MAXM], uc[MAXM], un[MAXM];
#pragma unroll
  for (int m = 0; m < MAXM; ++m) {
    const int i = lane + 32 * m;
    v[m] = i < nx ? g[i] : 0.0;
    uc[m] = i < nx ? uh[i] : 0.0;
    un[m] = i < nx ? uh[nx + i] : 0.0;
  }
  double sg = 0.0, ob = 0.0;
#pragma unroll
  for (int m = 0; m < MAXM; ++m) {
    const int i = lane + 32 * m;
    if (i < nx) {
      sv[i] = v[m];
      u[i] = v[m];
      sg += v[m];
      const double d = v[m] - uc[m];
      ob = fma(d, d, ob);
    }
  }
  sg = fx_warp_sum(sg);
  ob = fx_warp_sum(ob);
  const double M = a.dx * sg;
  if (lane == 0) put_stat(bst, fabs(a.dx * sg - M), 0.5 * ob);
  for (int k = lane; k <= K; k += 32) lam[nx + k] = 0.0;   // implied mass rows
  // forward substitution: u^k = G(u^{k-1})
  for (int k = 1; k <= K; ++k) {
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      const int i = lane + 32 * m;
      uc[m] = un[m];
      un[m] = (k < K && i < nx) ? uh[(size_t)(k + 1) * nx + i] : 0.0;
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      const int i = lane + 32 * m;
      if (i < nx) sa[i] = gd_flux(v[m], sv[i + 1 == nx ? 0 : i + 1]);
    }
    __syncwarp();
    double *uk = u + (size_t)k * nx;
    double sm = 0.0, o = 0.0;
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      const int i = lane + 32 * m;
      if (i < nx) {
        const double w = gd_update(v[m], sa[i], sa[i == 0 ? nx - 1 : i - 1], c);
        v[m] = w;
        sv[i] = w;
        uk[i] = w;
        sm += w;
        const double d = w - uc[m];
        o = fma(d, d, o);
      }
    }
    sm = fx_warp_sum(sm);
    o = fx_warp_sum(o);
    if (lane == 0) put_stat(bst + k, fabs(a.dx * sm - M), 0.5 * o);
  }
  // backward substitution: w = lambda^(j+1) in registers (and in sw for the neighbours)
  double w[MAXM], uj[MAXM];
  {
    double *lk = lam + nx + nt + (size_t)(K - 1) * nx;
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      const int i = lane + 32 * m;
      w[m] = uc[m] - v[m];
      if (i < nx) {
        sw[i] = w[m];
        lk[i] = w[m];
      }
      // slice K-1 (u and u_hat) for the first backward step
      uj[m] = i < nx ? u[(size_t)(K - 1) * nx + i] : 0.0;
      un[m] = i < nx ? uh[(size_t)(K - 1) * nx + i] : 0.0;
    }
  }
  for (int j = K - 1; j >= 0; --j) {
    double ujc[MAXM], pa[MAXM];
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      const int i = lane + 32 * m;
      ujc[m] = uj[m];
      uc[m] = un[m];
      uj[m] = (j > 0 && i < nx) ? u[(size_t)(j - 1) * nx + i] : 0.0;
      un[m] = (j > 0 && i < nx) ? uh[(size_t)(j - 1) * nx + i] : 0.0;
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      const int i = lane + 32 * m;
      if (i < nx) sv[i] = ujc[m];
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      const int i = lane + 32 * m;
      if (i < nx) {
        const int ip = i + 1 == nx ? 0 : i + 1;
        double da, db;
        gd_dflux(ujc[m], sv[ip], da, db);
        const double d = sw[ip] - w[m];
        pa[m] = da * d;      // used by this lane only
        sa[i] = db * d;      // used by the right neighbour
      }
    }
    __syncwarp();
    double *lj = j > 0 ? lam + nx + nt + (size_t)(j - 1) * nx : lam;
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      const int i = lane + 32 * m;
      if (i < nx) {
        const double jt = w[m] + c * (pa[m] + sa[i == 0 ? nx - 1 : i - 1]);
        w[m] = (uc[m] - ujc[m]) + jt;
        sw[i] = w[m];
        lj[i] = w[m];
      }
    }
  }
}

// Mass slices, the programmatic dependent of the chain kernel: it streams while the chains
// run.  Block 0 ends by waiting for the chain grid, so that this grid completes after it (the
// statistics kernel waits for this one); the other blocks exit when done and free their
// slots for the next wave.
__global__ void __launch_bounds__(kThreads) k1dflux_mass(FluxArgs a) {
  const long long wid = ((long long)blockIdx.x * kThreads + threadIdx.x) >> 5;
  flux_mass(a, wid, threadIdx.x & 31);
  if (blockIdx.x == 0) asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Adjoint (implicit-function theorem, Appendix B's K at the solution): K [a; b] = [gbar; 0].
// On slices 0..K the active rows are square and invertible, so a = 0 there and J^T b = gbar:
// the multipliers' backward substitution with u_hat - u replaced by gbar; dL/dg = b_IC plus
// dx times the mass multipliers of the later slices (dM/dg_i = dx).  On a mass slice
// a = gbar - mean(gbar) and dx b = sum(gbar) / nx, which goes to msum for the params kernel.
struct FluxBwdArgs {
  int B, nt, nx, K;
  double c;
  int n_chain_blocks;
  long long n_mass;
  const double *gu, *u;        // dL/du, u
  const snap_stats *fst;       // forward statistics or NULL
  double *gh, *gp;             // dL/du_hat [B][nt][nx], dL/dg [B][nx] or NULL
  double *msum;                // [B][nt]
};

__device__ __forceinline__ void flux_chain_bwd(const FluxBwdArgs &a, int b, int lane, double *w,
                                               double *sa, double *sb) {
  const int nx = a.nx, nt = a.nt, K = a.K;
  const size_t base = (size_t)b * nt * nx;
  const bool bad = a.fst && a.fst[b].status != SNAP_SAMPLE_OK;
  double *gh = a.gh + base;
  for (int i = lane; i < (K + 1) * nx; i += 32) gh[i] = bad ? NAN : 0.0;
  if (!a.gp) return;
  double *gp = a.gp + (size_t)b * nx;
  if (bad) {
    for (int i = lane; i < nx; i += 32) gp[i] = NAN;
    return;
  }
  const double *gu = a.gu + base, *u = a.u + base;
  for (int i = lane; i < nx; i += 32) w[i] = gu[(size_t)K * nx + i];
  for (int j = K - 1; j >= 0; --j) {
    __syncwarp();
    const double *uj = u + (size_t)j * nx;
    for (int i = lane; i < nx; i += 32) {
      const int ip = i + 1 == nx ? 0 : i + 1;
      double da, db;
      gd_dflux(uj[i], uj[ip], da, db);
      const double d = w[ip] - w[i];
      sa[i] = da * d;
      sb[i] = db * d;
    }
    __syncwarp();
    const double *gj = gu + (size_t)j * nx;
    for (int i = lane; i < nx; i += 32)
      w[i] = gj[i] + (w[i] + a.c * (sa[i] + sb[i == 0 ? nx - 1 : i - 1]));
  }
  __syncwarp();
  for (int i = lane; i < nx; i += 32) gp[i] = w[i];
}

__device__ __forceinline__ void flux_mass_bwd(const FluxBwdArgs &a, long long wid, int lane) {
  const int q = lane >> 2, r = lane & 3;
  const long long s = wid * 8 + q;
  const bool live = s < a.n_mass;
  const int nm = a.nt - a.K - 1, nx = a.nx;
  const int b = live ? (int)(s / nm) : 0, k = live ? a.K + 1 + (int)(s % nm) : 0;
  const size_t off = ((size_t)b * a.nt + k) * nx;
  const double *row = a.gu + off;
  const double S = s4_slice_sum(row, nx, r, live);
  if (!live) return;
  const bool bad = a.fst && a.fst[b].status != SNAP_SAMPLE_OK;
  const double mean = S / (double)nx;
  double *out = a.gh + off;
  for (int i = r; i < nx; i += 4) out[i] = bad ? NAN : row[i] - mean;
  if (r == 0) a.msum[(size_t)b * a.nt + k] = bad ? NAN : mean;
}

__global__ void __launch_bounds__(kThreads) k1dflux_backward(FluxBwdArgs a) {
  extern __shared__ double fx_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if ((int)blockIdx.x < a.n_chain_blocks) {
    const int b = (int)blockIdx.x * kChainWarps + wib;
    if (b >= a.B) return;
    double *w = fx_smem + (size_t)wib * 3 * a.nx;
    flux_chain_bwd(a, b, lane, w, w + a.nx, w + 2 * a.nx);
    return;
  }
  const long long wid = ((long long)(blockIdx.x - a.n_chain_blocks) * kThreads + threadIdx.x) >> 5;
  flux_mass_bwd(a, wid, lane);
}

// dL/dg_i += sum over the mass slices of mean(gbar^k) (fixed order), one warp per sample.
__global__ void k1dflux_backward_params(int B, int nt, int nx, int K,
                                        const double *__restrict__ msum, double *__restrict__ gp) {
  const int lane = threadIdx.x & 31;
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= B) return;
  double t = 0.0;
  for (int k = K + 1 + lane; k < nt; k += 32) t += msum[(size_t)b * nt + k];
  t = fx_warp_sum(t);
  for (int i = lane; i < nx; i += 32) gp[(size_t)b * nx + i] += t;
}

// Every nominal row at u: one warp per slice (the slice's mass row, its IC rows at k = 0, its
// flux rows at 1 <= k <= K); smax[b][k] = max |h| over them.
__global__ void __launch_bounds__(256)
k1dflux_residual(int B, int nt, int nx, int K, double dx, double c,
                 const double *__restrict__ u, const double *__restrict__ g,
                 double *__restrict__ h, double *__restrict__ smax) {
  const int lane = threadIdx.x & 31;
  const long long s = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (s >= (long long)B * nt) return;
  const int b = (int)(s / nt), k = (int)(s % nt);
  const double *row = u + (size_t)s * nx;
  const double *gb = g + (size_t)b * nx;
  double *hb = h ? h + (size_t)b * ((size_t)nx + nt + (size_t)K * nx) : nullptr;
  double su = 0.0, sg = 0.0, mx = 0.0;
  for (int i = lane; i < nx; i += 32) {
    su += row[i];
    sg += gb[i];
  }
  su = fx_warp_sum(su);
  sg = fx_warp_sum(sg);
  const double hm = dx * su - dx * sg;
  if (k == 0) {
    for (int i = lane; i < nx; i += 32) {
      const double v = row[i] - gb[i];
      if (hb) hb[i] = v;
      mx = s1_nan_max(mx, fabs(v));
    }
  } else if (k <= K) {
    const double *pv = row - nx;
    for (int i = lane; i < nx; i += 32) {
      const int ip = i + 1 == nx ? 0 : i + 1, im = i == 0 ? nx - 1 : i - 1;
      const double fr = gd_flux(pv[i], pv[ip]), fl = gd_flux(pv[im], pv[i]);
      const double v = row[i] - gd_update(pv[i], fr, fl, c);
      if (hb) hb[nx + nt + (size_t)(k - 1) * nx + i] = v;
      mx = s1_nan_max(mx, fabs(v));
    }
  }
  mx = s1_warp_max(mx);
  if (lane == 0) {
    if (hb) hb[nx + k] = hm;
    smax[s] = s1_nan_max(mx, fabs(hm));
  }
}

__global__ void k1dflux_rowmax(int B, int nt, const double *__restrict__ smax,
                               double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= B) return;
  double m = 0.0;
  for (int k = lane; k < nt; k += 32) m = s1_nan_max(m, smax[(size_t)b * nt + k]);
  m = s1_warp_max(m);
  if (lane == 0) out[b] = m;
}

unsigned blocks_for_warps(long long nwarps, int threads) {
  return (unsigned)((nwarps * 32 + threads - 1) / threads);
}

// c = dt / dx with dt = 1/(nt-1) and dx = 1/(nx-1), each rounded (the grid's definition)
double courant(int nx, int nt) { return (1.0 / (nt - 1)) / (1.0 / (nx - 1)); }

struct Grid {
  int n_chain_blocks;
  long long n_mass;
  unsigned mass_blocks;
  unsigned blocks;             // chain blocks + mass blocks (the combined adjoint kernel)
  size_t smem;
};

Grid flux_grid(const snap_problem *p, int B) {
  Grid G;
  const int nt = p->desc.nt, K = p->desc.n_flux;
  G.n_chain_blocks = (B + kChainWarps - 1) / kChainWarps;
  G.n_mass = (long long)B * (nt - K - 1);
  G.mass_blocks = blocks_for_warps((G.n_mass + 7) / 8, kThreads);
  G.blocks = (unsigned)G.n_chain_blocks + G.mass_blocks;
  G.smem = sizeof(double) * 3 * (size_t)p->desc.nx * kChainWarps;
  return G;
}

}  // namespace

size_t ws_bytes_1dflux(const snap_problem *p, int B) {
  const size_t nblk = (size_t)B * p->desc.nt;
  return snap_align256(sizeof(BlockStat) * nblk) + snap_align256(sizeof(double) * nblk);
}

cudaError_t launch_1dflux_forward(const snap_problem *p, int B, const double *u_hat,
                                  const double *params, double *u, double *lambda,
                                  snap_stats *stats, const SolverOpts &o, void *ws,
                                  cudaStream_t s) {
  const int nx = p->desc.nx, nt = p->desc.nt;
  const Grid G = flux_grid(p, B);
  FluxArgs a;
  a.B = B;
  a.nt = nt;
  a.nx = nx;
  a.K = p->desc.n_flux;
  a.dx = 1.0 / (nx - 1);
  a.c = courant(nx, nt);
  a.inv_nx = 1.0 / nx;
  a.inv_dx = (double)(nx - 1);
  a.n_chain_blocks = G.n_chain_blocks;
  a.n_mass = G.n_mass;
  a.uh = u_hat;
  a.g = params;
  a.u = u;
  a.lam = lambda;
  a.bst = (BlockStat *)ws;
  const int pid = snap_prof_begin(s, "k1dflux_forward");
  if (nx <= 128)
    k1dflux_chain<4><<<G.n_chain_blocks, kThreads, G.smem, s>>>(a);
  else if (nx <= 256)
    k1dflux_chain<8><<<G.n_chain_blocks, kThreads, G.smem, s>>>(a);
  else
    k1dflux_chain<16><<<G.n_chain_blocks, kThreads, G.smem, s>>>(a);
  int launches = 1;
  if (G.n_mass > 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G.mass_blocks);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k1dflux_mass, a);
    launches++;
  }
  snap_prof_end(s, pid);
  if (stats) {
    launch_finalize_stats(B, nt, a.bst, o.tol_h, stats, s);
    launches++;
  }
  snap_note_launch(launches);
  return cudaGetLastError();
}

cudaError_t launch_1dflux_backward(const snap_problem *p, int B, const double *grad_u,
                                   const double *u, const snap_stats *stats, double *grad_u_hat,
                                   double *grad_params, void *ws, cudaStream_t s) {
  const int nx = p->desc.nx, nt = p->desc.nt, K = p->desc.n_flux;
  const Grid G = flux_grid(p, B);
  FluxBwdArgs a;
  a.B = B;
  a.nt = nt;
  a.nx = nx;
  a.K = K;
  a.c = courant(nx, nt);
  a.n_chain_blocks = G.n_chain_blocks;
  a.n_mass = G.n_mass;
  a.gu = grad_u;
  a.u = u;
  a.fst = stats;
  a.gh = grad_u_hat;
  a.gp = grad_params;
  a.msum = (double *)ws;    // one double per slice, inside the statistics area
  const int pid = snap_prof_begin(s, "k1dflux_backward");
  k1dflux_backward<<<G.blocks, kThreads, G.smem, s>>>(a);
  snap_prof_end(s, pid);
  int launches = 1;
  if (grad_params && G.n_mass > 0) {
    k1dflux_backward_params<<<blocks_for_warps(B, 256), 256, 0, s>>>(B, nt, nx, K, a.msum,
                                                                    grad_params);
    launches++;
  }
  snap_note_launch(launches);
  return cudaGetLastError();
}

cudaError_t launch_1dflux_residual(const snap_problem *p, int B, const double *u,
                                   const double *params, double *h, double *h_inf, void *ws,
                                   cudaStream_t s) {
  const int nx = p->desc.nx, nt = p->desc.nt, K = p->desc.n_flux;
  double *smax = (double *)((char *)ws + snap_align256(sizeof(BlockStat) * (size_t)B * nt));
  k1dflux_residual<<<blocks_for_warps((long long)B * nt, 256), 256, 0, s>>>(
      B, nt, nx, K, 1.0 / (nx - 1), courant(nx, nt), u, params, h, smax);
  int launches = 1;
  if (h_inf) {
    k1dflux_rowmax<<<blocks_for_warps(B, 256), 256, 0, s>>>(B, nt, smax, h_inf);
    launches++;
  }
  snap_note_launch(launches);
  return cudaGetLastError();
}
