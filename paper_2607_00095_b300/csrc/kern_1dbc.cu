// Family D, the boundary-condition regime of the Burgers problem (Appendix A): per time slice
// k of a 1-D field on [0, 1] with nx grid points x_i = i dx, dx = 1 / (nx - 1) (both ends on
// the grid, no periodicity), the rows
//   Dirichlet  u_{k,0} - u_L = 0
//   mass       dx sum_i u_{k,i} - m0 = 0                       (Riemann sum, Appendix D)
//   Neumann    u_{k,nx-1} - u_{k,nx-2} = 0                      (Appendix D, right boundary)
// All three are linear, so the Newton-KKT iteration of Appendix B from (u_hat, 0) lands on the
// solution in one step: u = u_hat - A^T lambda with (A A^T) lambda = A u_hat - b.  With rows
// ordered (D, M, N) and nx >= 3, A A^T = [[1, dx, 0], [dx, nx dx^2, 0], [0, 0, 2]] (the
// Neumann row sums to zero and misses x_0), solved in closed form per slice.
//
// Four lanes per slice (eight slices per warp): the sum of u_hat on the FP32 and integer pipes
// (s4_slice_sum), the 3x3 solve on one lane of the slice, the write u_i = u_hat_i - dx
// lambda_M (- lambda_D at i = 0, -+ lambda_N at the right pair): one FP64 operation per element
// (FP64 is the scarce pipe on this GPU).  The
// statistics come from the step's closed form.
#include <cuda_runtime.h>
#include <math.h>

#include "sample_1d.cuh"
#include "snap_internal.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double bc_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// rows of slice k at u (every lane returns the same values)
struct BcRows {
  double hd, hm, hn;
};

__device__ __forceinline__ BcRows bc_rows(const double *__restrict__ row, int nx, double dx,
                                          double uL, double m0, int lane) {
  double s = 0.0;
  for (int i = lane; i < nx; i += 32) s += row[i];
  s = bc_warp_sum(s);
  return BcRows{row[0] - uL, dx * s - m0, row[nx - 1] - row[nx - 2]};
}

// Four lanes per slice, eight slices per warp: lane group q owns slice 8 w + q of warp w, lane
// r = 0..3 of the group reads elements r, r + 4, ... (32 contiguous bytes per group per load,
// eight rows per warp instruction), the group sums with two butterfly steps, lane r = 0 of
// the group solves the 3x3 system (eight slices in parallel) and broadcasts it.
__global__ void __launch_bounds__(256)
k1dbc_forward(int B, int nt, int nx, double dx, double inv_det, const double *__restrict__ uh,
              const double *__restrict__ params, double *__restrict__ u,
              double *__restrict__ lam, BlockStat *__restrict__ bst, double tol_kkt) {
  const int lane = threadIdx.x & 31;
  const int q = lane >> 2, r = lane & 3;
  const long long s = ((((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) << 3) + q;
  const long long nsl = (long long)B * nt;
  const bool live = s < nsl;
  int b = 0, k = 0;
  if (live) {
    if (nsl < (1LL << 31)) {           // 32-bit division (the 64-bit one is a long sequence)
      const unsigned su = (unsigned)s;
      b = (int)(su / (unsigned)nt);
      k = (int)(su - (unsigned)b * (unsigned)nt);
    } else {
      b = (int)(s / nt);
      k = (int)(s % nt);
    }
  }
  const double *row = uh + (size_t)(live ? s : 0) * nx;
  double *out = u + (size_t)(live ? s : 0) * nx;
  // F at (u_hat, 0): the rows (the Lagrangian gradient is zero there)
  const double S = s4_slice_sum(row, nx, r, live);
  double f0 = 0.0, lD = 0.0, lM = 0.0, lN = 0.0;
  double uL = 0.0, m0 = 0.0, u0v = 0.0, ua = 0.0, ub = 0.0;
  if (live && r == 0) {
    uL = params[2 * (size_t)b];
    m0 = params[2 * (size_t)b + 1];
    u0v = row[0]; ua = row[nx - 2]; ub = row[nx - 1];
    const double rd = u0v - uL, rm = dx * S - m0, rn = ub - ua;
    f0 = fmax(fabs(rd), fmax(fabs(rm), fabs(rn)));
    if (!(f0 <= tol_kkt) || f0 != f0) {
      lD = ((double)nx * dx * dx * rd - dx * rm) * inv_det;
      lM = (rm - dx * rd) * inv_det;
      lN = 0.5 * rn;
    }
  }
  const int src = lane & ~3;
  f0 = __shfl_sync(FULL, f0, src);
  lD = __shfl_sync(FULL, lD, src);
  lM = __shfl_sync(FULL, lM, src);
  lN = __shfl_sync(FULL, lN, src);
  if (!live) return;
  const bool take = !(f0 <= tol_kkt);
  const double c = dx * lM;
  if (take) {
    // one FP64 subtraction per element; the three special points are rewritten by the lanes
    // that own them (same thread: program order)
#pragma unroll 8
    for (int i = r; i < nx; i += 4) out[i] = row[i] - c;
    if (r == 0) out[0] = (row[0] - c) - lD;
    if (r == (nx - 2) % 4) out[nx - 2] = (row[nx - 2] - c) + lN;
    if (r == (nx - 1) % 4) out[nx - 1] = (row[nx - 1] - c) - lN;
  } else {
    for (int i = r; i < nx; i += 4) out[i] = row[i];
  }
  if (r == 0) {
    // the rows after the step, from the step's closed form (u_0, the right pair and the sum
    // sum u = S - nx dx lambda_M - lambda_D)
    const double w0 = (u0v - c) - lD;
    const double wa = (ua - c) + lN, wb = (ub - c) - lN;
    const double hd = w0 - uL, hn = wb - wa;
    const double hm = dx * (S - (double)nx * c - lD) - m0;
    double *lb = lam + (size_t)b * 3 * nt;
    lb[k] = lD;
    lb[nt + k] = lM;
    lb[2 * nt + k] = lN;
    BlockStat st;
    st.iters = take ? 1 : 0;
    st.backtracks = 0;
    st.corrections = 0;
    const double hinf = take ? fmax(fabs(hd), fmax(fabs(hm), fabs(hn))) : f0;
    st.status = (f0 == f0 && !isinf(f0) && hinf == hinf) ? SNAP_SAMPLE_OK : SNAP_SAMPLE_NONFINITE;
    st.h_inf = hinf;
    st.kkt_inf = hinf;     // grad L = u - u_hat + A^T lambda vanishes by construction
    // 1/2 ||u - u_hat||^2 = 1/2 lambda^T (A A^T) lambda
    st.obj = 0.5 * (lD * lD + 2.0 * dx * lD * lM + (double)nx * dx * dx * lM * lM + 2.0 * lN * lN);
    bst[s] = st;
  }
}

// Adjoint (implicit-function theorem on the linear KKT system; Appendix B's K at the solution
// does not depend on u for linear rows): K [a; b] = [gbar; 0] gives
// b = (A A^T)^-1 A gbar and a = dL/du_hat = gbar - A^T b, the same projector as the forward
// step applied to gbar with zero right-hand side.  dL/du_L = sum_k b_D,k and
// dL/dm0 = sum_k b_M,k (each right-hand side enters h with a minus sign).  The per-slice
// (b_D, b_M) go to the workspace; a sample whose forward status is not OK gets NaN.
__global__ void __launch_bounds__(256)
k1dbc_backward(int B, int nt, int nx, double dx, double inv_det, const double *__restrict__ gu,
               const snap_stats *__restrict__ fst, double *__restrict__ gh,
               double2 *__restrict__ bsum) {
  const int lane = threadIdx.x & 31;
  const int q = lane >> 2, r = lane & 3;
  const long long s = ((((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) << 3) + q;
  const long long nsl = (long long)B * nt;
  const bool live = s < nsl;
  const int b = !live ? 0 : nsl < (1LL << 31) ? (int)((unsigned)s / (unsigned)nt) : (int)(s / nt);
  const double *row = gu + (size_t)(live ? s : 0) * nx;
  double *out = gh + (size_t)(live ? s : 0) * nx;
  const double S = s4_slice_sum(row, nx, r, live);
  double lD = 0.0, lM = 0.0, lN = 0.0;
  const bool bad = live && fst && fst[b].status != SNAP_SAMPLE_OK;
  if (live && r == 0) {
    const double rd = row[0], rm = dx * S, rn = row[nx - 1] - row[nx - 2];
    lD = ((double)nx * dx * dx * rd - dx * rm) * inv_det;
    lM = (rm - dx * rd) * inv_det;
    lN = 0.5 * rn;
  }
  const int src = lane & ~3;
  lD = __shfl_sync(FULL, lD, src);
  lM = __shfl_sync(FULL, lM, src);
  lN = __shfl_sync(FULL, lN, src);
  if (!live) return;
  const double c = dx * lM;
  if (bad) {
    for (int i = r; i < nx; i += 4) out[i] = NAN;
  } else {
    for (int i = r; i < nx; i += 4) out[i] = row[i] - c;
    if (r == 0) out[0] = (row[0] - c) - lD;
    if (r == (nx - 2) % 4) out[nx - 2] = (row[nx - 2] - c) + lN;
    if (r == (nx - 1) % 4) out[nx - 1] = (row[nx - 1] - c) - lN;
  }
  if (r == 0) bsum[s] = bad ? make_double2(NAN, NAN) : make_double2(lD, lM);
}

// dL/d(u_L, m0) per sample: fixed-order sums of the slices' (b_D, b_M).
__global__ void k1dbc_backward_params(int B, int nt, const double2 *__restrict__ bsum,
                                      double *__restrict__ gp) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= B) return;
  double d = 0.0, m = 0.0;
  for (int k = lane; k < nt; k += 32) {
    const double2 v = bsum[(size_t)warp * nt + k];
    d += v.x;
    m += v.y;
  }
  d = bc_warp_sum(d);
  m = bc_warp_sum(m);
  if (lane == 0) {
    gp[2 * (size_t)warp] = d;
    gp[2 * (size_t)warp + 1] = m;
  }
}

__global__ void __launch_bounds__(256)
k1dbc_residual(int B, int nt, int nx, double dx, const double *__restrict__ u,
               const double *__restrict__ params, double *__restrict__ h,
               double *__restrict__ smax) {
  const int lane = threadIdx.x & 31;
  const long long s = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (s >= (long long)B * nt) return;
  const int b = (int)(s / nt), k = (int)(s % nt);
  const BcRows r = bc_rows(u + (size_t)s * nx, nx, dx, params[2 * (size_t)b],
                           params[2 * (size_t)b + 1], lane);
  if (lane == 0) {
    if (h) {
      double *hb = h + (size_t)b * 3 * nt;
      hb[k] = r.hd;
      hb[nt + k] = r.hm;
      hb[2 * nt + k] = r.hn;
    }
    smax[s] = s1_nan_max(s1_nan_max(fabs(r.hd), fabs(r.hm)), fabs(r.hn));
  }
}

__global__ void k1dbc_rowmax(int B, int nt, const double *__restrict__ smax,
                             double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= B) return;
  double m = 0.0;
  for (int k = lane; k < nt; k += 32) m = s1_nan_max(m, smax[(size_t)warp * nt + k]);
  m = s1_warp_max(m);
  if (lane == 0) out[warp] = m;
}

unsigned blocks_for_warps(long long nwarps) { return (unsigned)((nwarps * 32 + 255) / 256); }

}  // namespace

size_t ws_bytes_1dbc(const snap_problem *p, int B) {
  const size_t nblk = (size_t)B * p->desc.nt;
  return snap_align256(sizeof(BlockStat) * nblk) + snap_align256(sizeof(double) * nblk);
}

cudaError_t launch_1dbc_forward(const snap_problem *p, int B, const double *u_hat,
                                const double *params, double *u, double *lambda,
                                snap_stats *stats, const SolverOpts &o, void *ws,
                                cudaStream_t s) {
  const int nx = p->desc.nx, nt = p->desc.nt;
  BlockStat *bst = (BlockStat *)ws;
  const int pid = snap_prof_begin(s, "k1dbc_forward");
  const double dx = 1.0 / (nx - 1);
  const double inv_det = 1.0 / ((double)(nx - 1) * dx * dx);   // 1 / det of the (D, M) block
  k1dbc_forward<<<blocks_for_warps(((long long)B * nt + 7) / 8), 256, 0, s>>>(
      B, nt, nx, dx, inv_det, u_hat, params, u, lambda, bst, o.tol_kkt);
  snap_prof_end(s, pid);
  int launches = 1;
  if (stats) {
    launch_finalize_stats(B, nt, bst, o.tol_h, stats, s);
    launches++;
  }
  snap_note_launch(launches);
  return cudaGetLastError();
}

cudaError_t launch_1dbc_backward(const snap_problem *p, int B, const double *grad_u,
                                 const snap_stats *stats, double *grad_u_hat, double *grad_params,
                                 void *ws, cudaStream_t s) {
  const int nx = p->desc.nx, nt = p->desc.nt;
  // (b_D, b_M) per slice in the statistics area of the workspace (16 of its 40 bytes / slice)
  double2 *bsum = (double2 *)ws;
  const double dx = 1.0 / (nx - 1);
  const double inv_det = 1.0 / ((double)(nx - 1) * dx * dx);
  const int pid = snap_prof_begin(s, "k1dbc_backward");
  k1dbc_backward<<<blocks_for_warps(((long long)B * nt + 7) / 8), 256, 0, s>>>(
      B, nt, nx, dx, inv_det, grad_u, stats, grad_u_hat, bsum);
  snap_prof_end(s, pid);
  int launches = 1;
  if (grad_params) {
    k1dbc_backward_params<<<blocks_for_warps(B), 256, 0, s>>>(B, nt, bsum, grad_params);
    launches++;
  }
  snap_note_launch(launches);
  return cudaGetLastError();
}

cudaError_t launch_1dbc_residual(const snap_problem *p, int B, const double *u,
                                 const double *params, double *h, double *h_inf, void *ws,
                                 cudaStream_t s) {
  const int nx = p->desc.nx, nt = p->desc.nt;
  double *smax = (double *)((char *)ws + snap_align256(sizeof(BlockStat) * (size_t)B * nt));
  k1dbc_residual<<<blocks_for_warps((long long)B * nt), 256, 0, s>>>(B, nt, nx, 1.0 / (nx - 1), u,
                                                                    params, h, smax);
  int launches = 1;
  if (h_inf) {
    k1dbc_rowmax<<<blocks_for_warps(B), 256, 0, s>>>(B, nt, smax, h_inf);
    launches++;
  }
  snap_note_launch(launches);
  return cudaGetLastError();
}
