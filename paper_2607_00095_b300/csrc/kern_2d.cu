// 2-D family C: per frame f, w = (u, v) on a periodic N x N grid (dx = 1/N),
//   divergence rows  (D w)_{ij} = (u_{i+1,j} - u_{i-1,j} + v_{i,j+1} - v_{i,j-1}) / (2 dx)
//   kinetic energy   1/2 dx^2 ||w||^2 = K_f = K0 exp(-r2 t_f),
// projected with the Newton-KKT iteration of Appendix B.
//
// Structure used.  W = (1 + kappa dx^2) I =: alpha I is uniform (kappa = energy multiplier),
// and the divergence block of S = J W^-1 J^T is (1/alpha) D_a D_a^T with D_a the active
// divergence rows.  D D^T couples only cells of the same parity class (i mod 2, j mod 2):
//   (D D^T x)_{ij} = (4 x_{ij} - x_{i+-2,j} - x_{i,j+-2}) / (4 dx^2),
// i.e. on each class a periodic M x M 5-point Laplacian (M = N/2) -- the same matrix for all
// four classes -- singular with the class constant as null vector; the row of the class's
// first cell is left out of the solve (multiplier 0 there).  Its right-hand sides always sum
// to zero over a class (every divergence does), so the system with that row left out is
// solved by the zero-mean periodic solution shifted to vanish at the left-out cell.
//
// The divergence block is factored once per problem, at create, as the eigen-decomposition
// of the class Laplacian A = T (x) I + I (x) T (T = periodic second difference, eigenvectors
// Q = real Fourier basis, eigenvalues theta_p = 2 - 2 cos(2 pi p / M)): A^+ B = Q ((Q^T B Q) /
// (theta_p + theta_q)) Q^T.  The factor is shared by every sample, frame, class and Newton
// step; per right-hand side the solve is four M x M dense products on the FP32 pipe, refined
// against the exact stencil residual in double-float (mixed-precision iterative refinement).
//
// Moment form.  From w = w_hat, lambda = 0, every Newton iterate has the form
//   w = a P w_hat + s y,   lambda_div = mu z,   kappa,
// with z = (D_a D_a^T)^-1 D_a w_hat and y = D_a^T z = (I - P) w_hat (P = orthogonal projector
// on null(D_a)): the step of Appendix B maps this family into itself, so one Poisson solve
// per frame plus the moments A1 = ||P w_hat||^2, A2 = ||y||^2, d2 = ||D_a w_hat||^2 describe
// every iterate.  The step itself is closed form in (a, s, mu, kappa):
//   alpha da + dx^2 a dk = -p,  alpha ds + dmu + dx^2 s dk = -r,  ds = -s,
//   dx^2 (a A1 da + s A2 ds) = -h_K,
// with p = alpha a - 1, r = alpha s - 1 + mu (grad_w L = p P w_hat + r y), h_K the energy row.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "df64.cuh"
#include "slice_newton.cuh"
#include "snap_internal.h"

// ---------------------------------------------------------------------------------------
// host: the shared factor (Q and 1 / (theta_p + theta_q) in float)
// ---------------------------------------------------------------------------------------

struct Const2D {
  int M;
  float *Q;      // [M][M] column p = eigenvector p (row k = component k)
  float *inv;    // [M][M] 1 / (theta_p + theta_q), 0 for p = q = 0
};

static void class_eigen(int M, std::vector<double> &Q, std::vector<double> &theta) {
  // real orthonormal eigenvectors of the periodic second difference T (T_kk = 2,
  // T_{k,k+-1} = -1, periodic): cosines and sines of the Fourier modes
  Q.assign((size_t)M * M, 0.0);
  theta.assign(M, 0.0);
  const double pi = 3.14159265358979323846;
  int col = 0;
  auto set_col = [&](int c, int mode, bool sine, double norm) {
    for (int k = 0; k < M; ++k) {
      const double ang = 2.0 * pi * (double)mode * (double)k / (double)M;
      Q[(size_t)k * M + c] = norm * (sine ? sin(ang) : cos(ang));
    }
    theta[c] = 2.0 - 2.0 * cos(2.0 * pi * (double)mode / (double)M);
  };
  set_col(col++, 0, false, 1.0 / sqrt((double)M));
  for (int p = 1; 2 * p < M; ++p) {
    set_col(col++, p, false, sqrt(2.0 / M));
    set_col(col++, p, true, sqrt(2.0 / M));
  }
  if (M % 2 == 0 && M >= 2) set_col(col++, M / 2, false, 1.0 / sqrt((double)M));
}

// Host copy of the factor, uploaded on create (or on first use when the create call ran
// without a usable device, e.g. a host-only pattern query).
struct Host2D {
  std::vector<float> Qinv;   // [Q | inv], 2 M^2 floats
};

static cudaError_t upload_2d(snap_problem *p) {
  Host2D *h = (Host2D *)p->host_const;
  if (!h) return cudaErrorInvalidValue;
  const size_t bytes = sizeof(float) * h->Qinv.size();
  void *d = nullptr;
  cudaError_t e = cudaMalloc(&d, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  e = cudaMemcpy(d, h->Qinv.data(), bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return e;
  }
  p->dev_const = d;
  p->dev_const_bytes = bytes;
  return cudaSuccess;
}

cudaError_t setup_2d(snap_problem *p) {
  const int N = p->desc.nx;
  const int M = N / 2;
  std::vector<double> Q, th;
  class_eigen(M, Q, th);
  Host2D *h = new Host2D;
  h->Qinv.resize((size_t)2 * M * M);
  for (int i = 0; i < M * M; ++i) h->Qinv[i] = (float)Q[i];
  for (int a = 0; a < M; ++a)
    for (int b = 0; b < M; ++b) {
      const double e = th[a] + th[b];
      h->Qinv[(size_t)M * M + (size_t)a * M + b] = (a == 0 && b == 0) ? 0.0f : (float)(1.0 / e);
    }
  p->host_const = h;
  p->n2d_m = M;
  upload_2d(p);      // a failure here is reported by the first compute call
  return cudaSuccess;
}

// Device copy of the factor for a compute call (uploaded now if create could not).
static cudaError_t ensure_2d(const snap_problem *p) {
  if (p->dev_const) return cudaSuccess;
  return upload_2d(const_cast<snap_problem *>(p));
}

void teardown_2d(snap_problem *p) {
  if (p->dev_const) cudaFree(p->dev_const);
  p->dev_const = nullptr;
  delete (Host2D *)p->host_const;
  p->host_const = nullptr;
}

// ---------------------------------------------------------------------------------------
// device
// ---------------------------------------------------------------------------------------
namespace {

constexpr int T2D = 256;                 // threads per frame
constexpr int REFINE = 4;                // float solves per right-hand side (refinement)

__device__ __forceinline__ df64 dsplit(double x) {
  float h, l;
  if (df_split(x, h, l)) return df64(h, l);
  return df64(x);                        // out of the pair range: FP64 conversion
}

__device__ __forceinline__ float fabs_max(float a, float b) {
  const float x = fabsf(b);
  return (a < x || x != x) ? x : a;
}

// block reductions (T2D threads); every thread gets the result
__device__ float block_max(float v, float *red) {
  for (int o = 16; o > 0; o >>= 1) {
    const float w = __shfl_xor_sync(0xffffffffu, v, o);
    v = (v < w || w != w) ? w : v;
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  float r = red[0];
  for (int i = 1; i < T2D / 32; ++i) r = (r < red[i] || red[i] != red[i]) ? red[i] : r;
  __syncthreads();
  return r;
}

__device__ float block_sumf(float v, float *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  float r = 0.0f;
  for (int i = 0; i < T2D / 32; ++i) r += red[i];
  __syncthreads();
  return r;
}

__device__ df64 block_sumdf(df64 v, float *red) {
  for (int o = 16; o > 0; o >>= 1)
    v = v + df64(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) { red[2 * wid] = v.hi; red[2 * wid + 1] = v.lo; }
  __syncthreads();
  df64 r(0.0f, 0.0f);
  for (int i = 0; i < T2D / 32; ++i) r = r + df64(red[2 * i], red[2 * i + 1]);
  __syncthreads();
  return r;
}

// zero-mean solution of A x = r on the four classes (A = class Laplacian, r in rf, result in
// rf): x = Q ((Q^T r Q) .* inv) Q^T, four M x M products per class, all in float
template <int M>
__device__ void fd_solve(float *rf, float *tf, const float *Q, const float *inv) {
  constexpr int MM = M * M;
  // T = Q^T R   (tf)
  for (int o = threadIdx.x; o < 4 * MM; o += T2D) {
    const int c = o / MM, m = (o % MM) / M, pp = o % M;
    const float *R = rf + c * MM;
    float acc = 0.0f;
#pragma unroll 8
    for (int k = 0; k < M; ++k) acc = fmaf(Q[k * M + m], R[k * M + pp], acc);
    tf[o] = acc;
  }
  __syncthreads();
  // R = (T Q) .* inv
  for (int o = threadIdx.x; o < 4 * MM; o += T2D) {
    const int c = o / MM, m = (o % MM) / M, n = o % M;
    const float *T = tf + c * MM;
    float acc = 0.0f;
#pragma unroll 8
    for (int p = 0; p < M; ++p) acc = fmaf(T[m * M + p], Q[p * M + n], acc);
    rf[o] = acc * inv[m * M + n];
  }
  __syncthreads();
  // T = Q R
  for (int o = threadIdx.x; o < 4 * MM; o += T2D) {
    const int c = o / MM, k = (o % MM) / M, n = o % M;
    const float *R = rf + c * MM;
    float acc = 0.0f;
#pragma unroll 8
    for (int m = 0; m < M; ++m) acc = fmaf(Q[k * M + m], R[m * M + n], acc);
    tf[o] = acc;
  }
  __syncthreads();
  // R = T Q^T
  for (int o = threadIdx.x; o < 4 * MM; o += T2D) {
    const int c = o / MM, k = (o % MM) / M, j = o % M;
    const float *T = tf + c * MM;
    float acc = 0.0f;
#pragma unroll 8
    for (int n = 0; n < M; ++n) acc = fmaf(T[k * M + n], Q[j * M + n], acc);
    rf[o] = acc;
  }
  __syncthreads();
}

// class / class-local coordinates of cell (i, j) of an N = 2M grid
template <int M>
__device__ __forceinline__ int cell_slot(int i, int j) {
  constexpr int N = 2 * M;
  i = (i + N) % N;
  j = (j + N) % N;
  const int c = (i & 1) + 2 * (j & 1);
  return c * M * M + (j >> 1) * M + (i >> 1);
}

struct Frame2D {
  df64 A1, A2, K, dx;
  float d2, dinf, Pinf, yinf;
};

struct Z2D {
  df64 a, s, mu, kap;
};

struct E2D {
  df64 alpha, p, r, hK, phi, res;
};

__device__ __forceinline__ void eval2d(const Frame2D &F, const Z2D &z, E2D &e) {
  const df64 one(1.0f, 0.0f), half(0.5f, 0.0f);
  const df64 dx2 = F.dx * F.dx;
  e.alpha = one + z.kap * dx2;
  e.p = e.alpha * z.a - one;
  e.r = e.alpha * z.s - one + z.mu;
  e.hK = half * dx2 * (z.a * z.a * F.A1 + z.s * z.s * F.A2) - F.K;
  const float p = e.p.hi, r = e.r.hi, s = z.s.hi, hk = e.hK.hi;
  const float phi = 0.5f * (p * p * F.A1.hi + r * r * F.A2.hi + s * s * F.d2 + hk * hk);
  float res = fmaxf(fabsf(p) * F.Pinf + fabsf(r) * F.yinf, fmaxf(fabsf(s) * F.dinf, fabsf(hk)));
  if (phi != phi) res = phi;
  e.phi = df64(phi, 0.0f);
  e.res = df64(res, 0.0f);
}

// Newton-KKT of one frame in the moment coordinates (closed-form steps)
__device__ SliceResult newton2d(const Frame2D &F, Z2D &z, E2D &e, const SolverOpts &o) {
  SliceResult R{0, 0, SNAP_SAMPLE_OK, 0};
  const df64 zero(0.0f, 0.0f), one(1.0f, 0.0f), half(0.5f, 0.0f);
  const df64 dx2 = F.dx * F.dx;
  const df64 tol = df64(o.tol_kkt);
  const bool has_y = F.A2.hi > 0.0f && F.d2 > 0.0f;
  eval2d(F, z, e);
  for (int it = 0;; ++it) {
    if (!sl_finite(e.res)) { R.status = SNAP_SAMPLE_NONFINITE; break; }
    if (e.res <= tol) { R.status = SNAP_SAMPLE_OK; break; }
    if (it >= o.max_iter) { R.status = SNAP_SAMPLE_MAXITER; break; }
    // W = alpha I; inertia correction (max_corrections > 0) shifts alpha until positive
    df64 al = e.alpha;
    if (o.max_corrections > 0 && !(al > zero)) {
      df64 d = df64(o.delta0);
      int corr = 0;
      while (!(al + d > zero) && corr < o.max_corrections) { d = d * df64(10.0f, 0.0f); corr++; }
      R.corrections += corr + 1;
      al = al + d;
    }
    if (z.a == zero || F.A1 == zero || al == zero) { R.status = SNAP_SAMPLE_SINGULAR; break; }
    Z2D dz;
    dz.s = has_y ? -z.s : zero;
    dz.a = (-e.hK - dx2 * z.s * F.A2 * dz.s) / (dx2 * z.a * F.A1);
    dz.kap = (-e.p - al * dz.a) / (dx2 * z.a);
    dz.mu = has_y ? (-e.r - al * dz.s - dx2 * z.s * dz.kap) : zero;
    // W-positivity cap: alpha(t) = alpha + t dx^2 dkappa
    df64 t = one;
    if (o.w_keep > 0.0) {
      const df64 da = dx2 * dz.kap;
      if (e.alpha > zero && da < zero) {
        const df64 tm = df64(1.0 - o.w_keep) * e.alpha / (-da);
        if (tm < t) t = tm;
      }
    }
    int nb = 0;
    bool acc = false;
    Z2D zt;
    E2D et;
    for (;;) {
      zt.a = z.a + t * dz.a; zt.s = z.s + t * dz.s;
      zt.mu = z.mu + t * dz.mu; zt.kap = z.kap + t * dz.kap;
      eval2d(F, zt, et);
      if (et.phi <= (one - df64(2.0 * o.c1) * t) * e.phi) { acc = true; break; }
      if (nb >= o.max_backtracks) break;
      nb++;
      t = t * half;
    }
    R.backtracks += nb;
    if (!acc) { R.status = SNAP_SAMPLE_LINESEARCH; break; }
    z = zt;
    e = et;
    R.iters++;
  }
  if (R.status == SNAP_SAMPLE_OK && !(e.alpha > zero)) R.status = SNAP_SAMPLE_NOT_MINIMUM;
  return R;
}

}  // namespace

namespace {

// Dynamic shared memory of one frame (N = 2M): w [2 N^2] double, then float arrays
// b (hi, lo), z (hi, lo), r, t [4 M^2 = N^2 each], Q, inv [M^2 each], reduction scratch.
template <int M>
struct Smem2D {
  static constexpr int N = 2 * M, NN = N * N, MM = M * M;
  static constexpr size_t bytes = sizeof(double) * 2 * NN + sizeof(float) * (6 * NN + 2 * MM + 64);
};

template <int M>
struct View2D {
  double *W;
  float *Bh, *Bl, *Zh, *Zl, *Rf, *Tf, *Q, *I, *red;
  __device__ explicit View2D(unsigned char *base) {
    constexpr int NN = Smem2D<M>::NN, MM = Smem2D<M>::MM;
    W = reinterpret_cast<double *>(base);
    float *f = reinterpret_cast<float *>(base + sizeof(double) * 2 * NN);
    Bh = f; Bl = f + NN; Zh = f + 2 * NN; Zl = f + 3 * NN; Rf = f + 4 * NN; Tf = f + 5 * NN;
    Q = f + 6 * NN; I = Q + MM; red = I + MM;
  }
  __device__ df64 z(int slot) const { return df64(Zh[slot], Zl[slot]); }
};

// Solve (D D^T) z = b on the four classes of one frame (b already in Bh/Bl), result in
// Zh/Zl with z = 0 at each class's left-out cell.  REFINE float solves, the residual
// r = b - (D D^T) z formed in double-float between them.
template <int M>
__device__ void poisson_frame(View2D<M> &v, const df64 &scale) {
  constexpr int N = 2 * M, NN = N * N, MM = M * M;
  for (int s = threadIdx.x; s < NN; s += T2D) {
    v.Zh[s] = 0.0f;
    v.Zl[s] = 0.0f;
    v.Rf[s] = v.Bh[s];
  }
  __syncthreads();
  const df64 inv_scale = df64(1.0f, 0.0f) / scale;
  for (int round = 0; round < REFINE; ++round) {
    fd_solve<M>(v.Rf, v.Tf, v.Q, v.I);
    for (int s = threadIdx.x; s < NN; s += T2D) {
      const df64 zz = v.z(s) + scale * df64(v.Rf[s], 0.0f);
      v.Zh[s] = zz.hi;
      v.Zl[s] = zz.lo;
    }
    __syncthreads();
    if (round + 1 < REFINE) {
      for (int s = threadIdx.x; s < NN; s += T2D) {
        const int c = s / MM, q = (s % MM) / M, p = s % M;
        const int base = c * MM;
        const df64 zc = v.z(s);
        const df64 nb = v.z(base + q * M + (p + 1) % M) + v.z(base + q * M + (p + M - 1) % M) +
                        v.z(base + ((q + 1) % M) * M + p) + v.z(base + ((q + M - 1) % M) * M + p);
        const df64 az = (df64(4.0f, 0.0f) * zc - nb) * inv_scale;
        const df64 r = df64(v.Bh[s], v.Bl[s]) - az;
        v.Rf[s] = r.hi + r.lo;
      }
      __syncthreads();
    }
  }
  // gauge: zero at class-local (0, 0) of every class
  df64 g0[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) g0[c] = v.z(c * MM);
  __syncthreads();
  for (int s = threadIdx.x; s < NN; s += T2D) {
    const df64 zz = v.z(s) - g0[s / MM];
    v.Zh[s] = zz.hi;
    v.Zl[s] = zz.lo;
  }
  __syncthreads();
}

// (D x)(i, j) of a field held as doubles in w[2][N][N]
template <int M>
__device__ __forceinline__ df64 div_at(const double *w, int i, int j, const df64 &h2) {
  constexpr int N = 2 * M, NN = N * N;
  const df64 ue = dsplit(w[j * N + (i + 1) % N]);
  const df64 uw = dsplit(w[j * N + (i + N - 1) % N]);
  const df64 vn = dsplit(w[NN + ((j + 1) % N) * N + i]);
  const df64 vs = dsplit(w[NN + ((j + N - 1) % N) * N + i]);
  return ((ue - uw) + (vn - vs)) * h2;
}

// (D^T z) for element e of w[2][N][N] (component e / N^2)
template <int M>
__device__ __forceinline__ df64 divT_at(const View2D<M> &v, int e, const df64 &h2) {
  constexpr int N = 2 * M, NN = N * N;
  const int comp = e / NN, cell = e % NN, i = cell % N, j = cell / N;
  if (comp == 0) return (v.z(cell_slot<M>(i - 1, j)) - v.z(cell_slot<M>(i + 1, j))) * h2;
  return (v.z(cell_slot<M>(i, j - 1)) - v.z(cell_slot<M>(i, j + 1))) * h2;
}

template <int M>
__global__ void __launch_bounds__(T2D)
k2d_frame(int B, int nt, const double *__restrict__ wh, const double *__restrict__ params,
          const float *__restrict__ Qg, const float *__restrict__ Ig, double *__restrict__ wout,
          double *__restrict__ lam, BlockStat *__restrict__ bst, SolverOpts o) {
  constexpr int N = 2 * M, NN = N * N, MM = M * M;
  extern __shared__ __align__(16) unsigned char smem2d[];
  View2D<M> v(smem2d);
  const int fr = blockIdx.x;
  if (fr >= B * nt) return;
  const int b = fr / nt, f = fr % nt;
  const double *src = wh + (size_t)fr * 2 * NN;
  const int n_rows = nt * NN + nt;
  const df64 h2((float)N * 0.5f, 0.0f);          // 1 / (2 dx), exact
  const df64 dx(1.0 / N);
  const df64 scale = df64(4.0 / ((double)N * (double)N));   // 4 dx^2
  for (int i = threadIdx.x; i < MM; i += T2D) { v.Q[i] = Qg[i]; v.I[i] = Ig[i]; }
  for (int e = threadIdx.x; e < 2 * NN; e += T2D) v.W[e] = src[e];
  __syncthreads();
  // b = D w_hat on every cell; moments of w_hat
  df64 a0(0.0f, 0.0f);
  float d2 = 0.0f, dinf = 0.0f;
  for (int e = threadIdx.x; e < 2 * NN; e += T2D) {
    const df64 x = dsplit(v.W[e]);
    a0 = a0 + x * x;
  }
  for (int cell = threadIdx.x; cell < NN; cell += T2D) {
    const int i = cell % N, j = cell / N;
    const df64 dv = div_at<M>(v.W, i, j, h2);
    const int s = cell_slot<M>(i, j);
    v.Bh[s] = dv.hi;
    v.Bl[s] = dv.lo;
    if (!(i < 2 && j < 2)) {
      d2 = fmaf(dv.hi, dv.hi, d2);
      dinf = fabs_max(dinf, dv.hi);
    }
  }
  __syncthreads();
  poisson_frame<M>(v, scale);
  // y = D^T z and its moments
  df64 a2(0.0f, 0.0f);
  float pinf = 0.0f, yinf = 0.0f;
  for (int e = threadIdx.x; e < 2 * NN; e += T2D) {
    const df64 y = divT_at<M>(v, e, h2);
    a2 = a2 + y * y;
    yinf = fabs_max(yinf, y.hi);
    const df64 pw = dsplit(v.W[e]) - y;
    pinf = fabs_max(pinf, pw.hi);
  }
  a0 = block_sumdf(a0, v.red);
  a2 = block_sumdf(a2, v.red);
  d2 = block_sumf(d2, v.red);
  dinf = block_max(dinf, v.red);
  pinf = block_max(pinf, v.red);
  yinf = block_max(yinf, v.red);
  // scalar Newton-KKT of the frame (thread 0), broadcast through shared memory
  __shared__ float zs[10];
  __shared__ SliceResult Rs;
  __shared__ float Ks[2];
  if (threadIdx.x == 0) {
    const double* pr = params + (size_t)b * 2;
    const double K = pr[0] * exp(-pr[1] * ((double)f / (double)(nt - 1)));
    Frame2D F;
    F.A1 = a0 - a2;
    F.A2 = a2;
    F.K = df64(K);
    F.dx = dx;
    F.d2 = d2; F.dinf = dinf; F.Pinf = pinf; F.yinf = yinf;
    Z2D z{df64(1.0f, 0.0f), df64(1.0f, 0.0f), df64(0.0f, 0.0f), df64(0.0f, 0.0f)};
    E2D e;
    Rs = newton2d(F, z, e, o);
    zs[0] = z.a.hi; zs[1] = z.a.lo; zs[2] = z.s.hi; zs[3] = z.s.lo;
    zs[4] = z.mu.hi; zs[5] = z.mu.lo; zs[6] = z.kap.hi; zs[7] = z.kap.lo;
    zs[8] = e.alpha.hi; zs[9] = e.alpha.lo;
    Ks[0] = F.K.hi; Ks[1] = F.K.lo;
  }
  __syncthreads();
  const df64 A(zs[0], zs[1]), S(zs[2], zs[3]), MU(zs[4], zs[5]), KAP(zs[6], zs[7]), AL(zs[8], zs[9]);
  const df64 Cc = S - A;
  // write w = a w_hat + c y, lambda_div = mu z; exact residual pieces
  double *dst = wout + (size_t)fr * 2 * NN;
  float ginf = 0.0f, obj = 0.0f;
  df64 w2(0.0f, 0.0f);
  for (int e = threadIdx.x; e < 2 * NN; e += T2D) {
    const df64 y = divT_at<M>(v, e, h2);
    const df64 x = dsplit(v.W[e]);
    const df64 w = A * x + Cc * y;
    const double wd = df_to_double(w);
    dst[e] = wd;
    const df64 gl = AL * w - x + MU * y;
    ginf = fabs_max(ginf, gl.hi);
    const float dwv = (w - x).hi;
    obj = fmaf(dwv, dwv, obj);
    w2 = w2 + w * w;
    v.W[e] = wd;
  }
  double *lb = lam + (size_t)b * n_rows + (size_t)f * NN;
  for (int cell = threadIdx.x; cell < NN; cell += T2D) {
    const int i = cell % N, j = cell / N;
    lb[cell] = (i < 2 && j < 2) ? 0.0 : df_to_double(MU * v.z(cell_slot<M>(i, j)));
  }
  __syncthreads();
  float hinf_all = 0.0f, hinf_act = 0.0f;
  for (int cell = threadIdx.x; cell < NN; cell += T2D) {
    const int i = cell % N, j = cell / N;
    const float dv = div_at<M>(v.W, i, j, h2).hi;
    hinf_all = fabs_max(hinf_all, dv);
    if (!(i < 2 && j < 2)) hinf_act = fabs_max(hinf_act, dv);
  }
  ginf = block_max(ginf, v.red);
  obj = block_sumf(obj, v.red);
  w2 = block_sumdf(w2, v.red);
  hinf_all = block_max(hinf_all, v.red);
  hinf_act = block_max(hinf_act, v.red);
  if (threadIdx.x == 0) {
    const df64 hK = df64(0.5f, 0.0f) * dx * dx * w2 - df64(Ks[0], Ks[1]);
    const float hk = fabsf(hK.hi);
    BlockStat st;
    st.iters = Rs.iters;
    st.backtracks = Rs.backtracks;
    st.corrections = Rs.corrections;
    st.status = Rs.status;
    st.kkt_inf = (double)fmaxf(fmaxf(ginf, hinf_act), hk);
    st.h_inf = (double)fmaxf(hinf_all, hk);
    if (hK.hi != hK.hi || ginf != ginf) { st.kkt_inf = NAN; st.h_inf = NAN; }
    st.obj = 0.5 * (double)obj;
    bst[fr] = st;
    lam[(size_t)b * n_rows + (size_t)nt * NN + f] = df_to_double(KAP);
  }
}

}  // namespace

namespace {

// Adjoint of one frame.  At the solution D_a w = 0, so S = J W^-1 J^T is block diagonal:
// (1/alpha) diag(D_a D_a^T, dx^4 ||w||^2).  Hence b_div = (D_a D_a^T)^-1 D_a gbar (one Poisson
// solve), b_K = w^T gbar / (dx^2 ||w||^2), a = (gbar - D_a^T b_div - b_K dx^2 w) / alpha.
template <int M>
__global__ void __launch_bounds__(T2D)
k2d_frame_bwd(int B, int nt, const double *__restrict__ gw, const double *__restrict__ w,
              const double *__restrict__ lam, const double *__restrict__ params,
              const snap_stats *__restrict__ fst, const float *__restrict__ Qg,
              const float *__restrict__ Ig, double *__restrict__ gout,
              BwdContrib *__restrict__ contrib) {
  constexpr int N = 2 * M, NN = N * N, MM = M * M;
  extern __shared__ __align__(16) unsigned char smem2d[];
  View2D<M> v(smem2d);
  const int fr = blockIdx.x;
  if (fr >= B * nt) return;
  const int b = fr / nt, f = fr % nt;
  const int n_rows = nt * NN + nt;
  const double *gsrc = gw + (size_t)fr * 2 * NN;
  const double *wsrc = w + (size_t)fr * 2 * NN;
  const df64 h2((float)N * 0.5f, 0.0f);
  const df64 dx(1.0 / N);
  const df64 scale = df64(4.0 / ((double)N * (double)N));
  for (int i = threadIdx.x; i < MM; i += T2D) { v.Q[i] = Qg[i]; v.I[i] = Ig[i]; }
  for (int e = threadIdx.x; e < 2 * NN; e += T2D) v.W[e] = gsrc[e];
  __syncthreads();
  df64 dot(0.0f, 0.0f), ww(0.0f, 0.0f);
  for (int e = threadIdx.x; e < 2 * NN; e += T2D) {
    const df64 x = dsplit(wsrc[e]), gx = dsplit(v.W[e]);
    dot = dot + x * gx;
    ww = ww + x * x;
  }
  for (int cell = threadIdx.x; cell < NN; cell += T2D) {
    const int i = cell % N, j = cell / N;
    const df64 dv = div_at<M>(v.W, i, j, h2);
    const int s = cell_slot<M>(i, j);
    v.Bh[s] = dv.hi;
    v.Bl[s] = dv.lo;
  }
  __syncthreads();
  poisson_frame<M>(v, scale);
  dot = block_sumdf(dot, v.red);
  ww = block_sumdf(ww, v.red);
  const double kap = lam[(size_t)b * n_rows + (size_t)nt * NN + f];
  const df64 dx2 = dx * dx;
  const df64 alpha = df64(1.0f, 0.0f) + dsplit(kap) * dx2;
  const df64 bK = dot / (dx2 * ww);
  const df64 ialpha = df64(1.0f, 0.0f) / alpha;
  const bool bad = fst && fst[b].status != SNAP_SAMPLE_OK;
  double *dst = gout + (size_t)fr * 2 * NN;
  for (int e = threadIdx.x; e < 2 * NN; e += T2D) {
    const df64 y = divT_at<M>(v, e, h2);
    const df64 a = (dsplit(v.W[e]) - y - bK * dx2 * dsplit(wsrc[e])) * ialpha;
    dst[e] = bad ? NAN : df_to_double(a);
  }
  if (threadIdx.x == 0) {
    const double *pr = params + (size_t)b * 2;
    const double t = (double)f / (double)(nt - 1);
    const double ex = exp(-pr[1] * t);
    const double bk = df_to_double(bK);
    // h_K = 1/2 dx^2 ||w||^2 - K0 exp(-r2 t): dL/dK0 += b_K e, dL/dr2 += -b_K t K0 e
    contrib[fr] = BwdContrib{bk * ex, -bk * t * pr[0] * ex, 0.0, 0.0};
  }
}

__global__ void k2d_backward_params(int B, int nt, const snap_stats *__restrict__ fst,
                                    const BwdContrib *__restrict__ contrib,
                                    double *__restrict__ gp) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= B) return;
  double s0 = 0.0, s1 = 0.0;
  for (int f = lane; f < nt; f += 32) {
    const BwdContrib c = contrib[(size_t)warp * nt + f];
    s0 += c.bm;
    s1 += c.bex;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if (lane == 0) {
    const bool bad = fst && fst[warp].status != SNAP_SAMPLE_OK;
    gp[(size_t)warp * 2] = bad ? NAN : s0;
    gp[(size_t)warp * 2 + 1] = bad ? NAN : s1;
  }
}

// h(w) of every nominal row of one frame (FP64; a verification kernel)
__global__ void k2d_residual(int B, int nt, int N, const double *__restrict__ w,
                             const double *__restrict__ params, double *__restrict__ h,
                             double *__restrict__ smax) {
  const int fr = blockIdx.x;
  if (fr >= B * nt) return;
  const int b = fr / nt, f = fr % nt;
  const int NN = N * N;
  const int n_rows = nt * NN + nt;
  const double *x = w + (size_t)fr * 2 * NN;
  const double h2 = 0.5 * N;
  double mx = 0.0, w2 = 0.0;
  for (int e = threadIdx.x; e < 2 * NN; e += blockDim.x) w2 = fma(x[e], x[e], w2);
  for (int cell = threadIdx.x; cell < NN; cell += blockDim.x) {
    const int i = cell % N, j = cell / N;
    const double dv = ((x[j * N + (i + 1) % N] - x[j * N + (i + N - 1) % N]) +
                       (x[NN + ((j + 1) % N) * N + i] - x[NN + ((j + N - 1) % N) * N + i])) * h2;
    if (h) h[(size_t)b * n_rows + (size_t)f * NN + cell] = dv;
    const double a = fabs(dv);
    mx = (mx < a || a != a) ? a : mx;
  }
  __shared__ double red[64];
  for (int o = 16; o > 0; o >>= 1) {
    w2 += __shfl_xor_sync(0xffffffffu, w2, o);
    const double t = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = (mx < t || t != t) ? t : mx;
  }
  if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = w2; red[32 + (threadIdx.x >> 5)] = mx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0, m = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      s += red[i];
      m = (m < red[32 + i] || red[32 + i] != red[32 + i]) ? red[32 + i] : m;
    }
    const double *pr = params + (size_t)b * 2;
    const double hk = 0.5 * s / ((double)N * (double)N) - pr[0] * exp(-pr[1] * ((double)f / (double)(nt - 1)));
    if (h) h[(size_t)b * n_rows + (size_t)nt * NN + f] = hk;
    const double a = fabs(hk);
    smax[fr] = (m < a || a != a) ? a : m;
  }
}

__global__ void k2d_rowmax(int B, int nt, const double *__restrict__ smax, double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= B) return;
  double m = 0.0;
  for (int f = lane; f < nt; f += 32) {
    const double a = smax[(size_t)warp * nt + f];
    m = (m < a || a != a) ? a : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_xor_sync(0xffffffffu, m, o);
    m = (m < t || t != t) ? t : m;
  }
  if (lane == 0) out[warp] = m;
}

struct Ws2D {
  BlockStat *bst;
  BwdContrib *contrib;
  double *smax;
};

Ws2D carve_2d(const snap_problem *p, int B, void *ws) {
  char *c = (char *)ws;
  const size_t nfr = (size_t)B * p->desc.nt;
  Ws2D w;
  w.bst = (BlockStat *)c;
  c += snap_align256(sizeof(BlockStat) * nfr);
  w.contrib = (BwdContrib *)c;
  c += snap_align256(sizeof(BwdContrib) * nfr);
  w.smax = (double *)c;
  return w;
}

template <int M>
cudaError_t fwd_m(const snap_problem *p, int B, const double *wh, const double *params, double *w,
                  double *lam, BlockStat *bst, const SolverOpts &o, cudaStream_t s) {
  const size_t bytes = Smem2D<M>::bytes;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k2d_frame<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const float *Q = (const float *)p->dev_const;
  const float *I = Q + (size_t)M * M;
  k2d_frame<M><<<B * p->desc.nt, T2D, bytes, s>>>(B, p->desc.nt, wh, params, Q, I, w, lam, bst, o);
  return cudaGetLastError();
}

template <int M>
cudaError_t bwd_m(const snap_problem *p, int B, const double *gw, const double *w, const double *lam,
                  const double *params, const snap_stats *st, double *gout, BwdContrib *contrib,
                  cudaStream_t s) {
  const size_t bytes = Smem2D<M>::bytes;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k2d_frame_bwd<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const float *Q = (const float *)p->dev_const;
  const float *I = Q + (size_t)M * M;
  k2d_frame_bwd<M><<<B * p->desc.nt, T2D, bytes, s>>>(B, p->desc.nt, gw, w, lam, params, st, Q, I, gout, contrib);
  return cudaGetLastError();
}

}  // namespace

bool supported_2d(int N) { return N == 4 || N == 8 || N == 16 || N == 32 || N == 64; }

size_t ws_bytes_2d(const snap_problem *p, int B) {
  const size_t nfr = (size_t)B * p->desc.nt;
  return snap_align256(sizeof(BlockStat) * nfr) + snap_align256(sizeof(BwdContrib) * nfr) +
         snap_align256(sizeof(double) * nfr);
}

size_t cache_bytes_2d(const snap_problem *p, int B) { (void)p; (void)B; return 0; }

static int warps_blocks2(int nwarps) { return (nwarps * 32 + 127) / 128; }

cudaError_t launch_2d_forward(const snap_problem *p, int B, const double *w_hat,
                              const double *params, const double *w0, double *w, double *lambda,
                              snap_stats *stats, void *cache, const SolverOpts &o, int path,
                              void *ws, cudaStream_t s) {
  (void)cache;
  (void)path;
  if (w0) return cudaErrorNotSupported;
  cudaError_t eu = ensure_2d(p);
  if (eu != cudaSuccess) return eu;
  Ws2D wk = carve_2d(p, B, ws);
  const int N = p->desc.nx;
  cudaError_t e;
  const int pid = snap_prof_begin(s, "k2d_frame");
  switch (N) {
    case 4: e = fwd_m<2>(p, B, w_hat, params, w, lambda, wk.bst, o, s); break;
    case 8: e = fwd_m<4>(p, B, w_hat, params, w, lambda, wk.bst, o, s); break;
    case 16: e = fwd_m<8>(p, B, w_hat, params, w, lambda, wk.bst, o, s); break;
    case 32: e = fwd_m<16>(p, B, w_hat, params, w, lambda, wk.bst, o, s); break;
    case 64: e = fwd_m<32>(p, B, w_hat, params, w, lambda, wk.bst, o, s); break;
    default: return cudaErrorNotSupported;
  }
  snap_prof_end(s, pid);
  if (e != cudaSuccess) return e;
  int launches = 1;
  if (stats) {
    launch_finalize_stats(B, p->desc.nt, wk.bst, o.tol_h, stats, s);
    launches++;
  }
  snap_note_launch(launches);
  return cudaGetLastError();
}

cudaError_t launch_2d_backward(const snap_problem *p, int B, const double *grad_w,
                               const double *w, const double *lambda, const double *params,
                               const snap_stats *stats, const void *cache, double *grad_w_hat,
                               double *grad_params, void *ws, cudaStream_t s) {
  (void)cache;
  cudaError_t eu = ensure_2d(p);
  if (eu != cudaSuccess) return eu;
  Ws2D wk = carve_2d(p, B, ws);
  const int N = p->desc.nx;
  cudaError_t e;
  const int pid = snap_prof_begin(s, "k2d_frame_bwd");
  switch (N) {
    case 4: e = bwd_m<2>(p, B, grad_w, w, lambda, params, stats, grad_w_hat, wk.contrib, s); break;
    case 8: e = bwd_m<4>(p, B, grad_w, w, lambda, params, stats, grad_w_hat, wk.contrib, s); break;
    case 16: e = bwd_m<8>(p, B, grad_w, w, lambda, params, stats, grad_w_hat, wk.contrib, s); break;
    case 32: e = bwd_m<16>(p, B, grad_w, w, lambda, params, stats, grad_w_hat, wk.contrib, s); break;
    case 64: e = bwd_m<32>(p, B, grad_w, w, lambda, params, stats, grad_w_hat, wk.contrib, s); break;
    default: return cudaErrorNotSupported;
  }
  snap_prof_end(s, pid);
  if (e != cudaSuccess) return e;
  int launches = 1;
  if (grad_params) {
    k2d_backward_params<<<warps_blocks2(B), 128, 0, s>>>(B, p->desc.nt, stats, wk.contrib, grad_params);
    launches++;
  }
  snap_note_launch(launches);
  return cudaGetLastError();
}

cudaError_t launch_2d_residual(const snap_problem *p, int B, const double *w,
                               const double *params, double *h, double *h_inf, void *ws,
                               cudaStream_t s) {
  Ws2D wk = carve_2d(p, B, ws);
  k2d_residual<<<B * p->desc.nt, 256, 0, s>>>(B, p->desc.nt, p->desc.nx, w, params, h, wk.smax);
  int launches = 1;
  if (h_inf) {
    k2d_rowmax<<<warps_blocks2(B), 128, 0, s>>>(B, p->desc.nt, wk.smax, h_inf);
    launches++;
  }
  snap_note_launch(launches);
  return cudaGetLastError();
}
