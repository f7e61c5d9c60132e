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

cudaError_t ensure_2d_factor(const snap_problem *p) { return ensure_2d(p); }

void teardown_2d(snap_problem *p) {
  if (p->dev_const) cudaFree(p->dev_const);
  p->dev_const = nullptr;
  delete (Host2D *)p->host_const;
  p->host_const = nullptr;
}

#include "frame_2d.cuh"

namespace {

template <int M>
__global__ void __launch_bounds__(T2D)
k2d_frame(int B, int nt, const double *__restrict__ wh, const double *__restrict__ params,
          const float *__restrict__ Qg, const float *__restrict__ Ig, double *__restrict__ wout,
          double *__restrict__ lam, BlockStat *__restrict__ bst, SolverOpts o) {
  constexpr int NN = 4 * M * M;
  extern __shared__ __align__(16) unsigned char smem2d[];
  View2D<M> v(smem2d);
  const int fr = blockIdx.x;
  if (fr >= B * nt) return;
  const int b = fr / nt, f = fr % nt;
  const size_t n_rows = (size_t)nt * NN + nt;
  frame2d_forward<M>(v, wh + (size_t)fr * 2 * NN, params + (size_t)b * 2, f, nt, Qg, Ig,
                     wout + (size_t)fr * 2 * NN, lam + (size_t)b * n_rows, bst + fr, o);
}

}  // namespace

namespace {

// Adjoint of the frames of a batch, one block per frame (frame2d_backward, frame_2d.cuh).
template <int M>
__global__ void __launch_bounds__(T2D)
k2d_frame_bwd(int B, int nt, const double *__restrict__ gw, const double *__restrict__ w,
              const double *__restrict__ lam, const double *__restrict__ params,
              const snap_stats *__restrict__ fst, const float *__restrict__ Qg,
              const float *__restrict__ Ig, double *__restrict__ gout,
              BwdContrib *__restrict__ contrib) {
  constexpr int NN = 4 * M * M;
  extern __shared__ __align__(16) unsigned char smem2d[];
  View2D<M> v(smem2d);
  const int fr = blockIdx.x;
  if (fr >= B * nt) return;
  const int b = fr / nt, f = fr % nt;
  const size_t n_rows = (size_t)nt * NN + nt;
  const bool bad = fst && fst[b].status != SNAP_SAMPLE_OK;
  frame2d_backward<M>(v, gw + (size_t)fr * 2 * NN, w + (size_t)fr * 2 * NN,
                      lam[(size_t)b * n_rows + (size_t)nt * NN + f], params + (size_t)b * 2, f,
                      nt, bad, Qg, Ig, gout + (size_t)fr * 2 * NN, contrib + fr);
}

__global__ void k2d_backward_params(int B, int nt, const snap_stats *__restrict__ fst,
                                    const BwdContrib *__restrict__ contrib,
                                    double *__restrict__ gp) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= B) return;
  const bool bad = fst && fst[warp].status != SNAP_SAMPLE_OK;
  frame2d_param_grad<false>(contrib + (size_t)warp * nt, nt, bad, gp + (size_t)warp * 2, lane);
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

// every even side 4..64: the class size M = N / 2 is a template parameter of the frame code
bool supported_2d(int N) { return N >= 4 && N <= 64 && N % 2 == 0; }

// FN<M>(args...) for the class size M = N / 2 of a supported side N
#define SNAP_DISPATCH_2D(N, FN, ...)                                                          \
  switch ((N) / 2) {                                                                         \
    case 2: e = FN<2>(__VA_ARGS__); break;   case 3: e = FN<3>(__VA_ARGS__); break;          \
    case 4: e = FN<4>(__VA_ARGS__); break;   case 5: e = FN<5>(__VA_ARGS__); break;          \
    case 6: e = FN<6>(__VA_ARGS__); break;   case 7: e = FN<7>(__VA_ARGS__); break;          \
    case 8: e = FN<8>(__VA_ARGS__); break;   case 9: e = FN<9>(__VA_ARGS__); break;          \
    case 10: e = FN<10>(__VA_ARGS__); break; case 11: e = FN<11>(__VA_ARGS__); break;        \
    case 12: e = FN<12>(__VA_ARGS__); break; case 13: e = FN<13>(__VA_ARGS__); break;        \
    case 14: e = FN<14>(__VA_ARGS__); break; case 15: e = FN<15>(__VA_ARGS__); break;        \
    case 16: e = FN<16>(__VA_ARGS__); break; case 17: e = FN<17>(__VA_ARGS__); break;        \
    case 18: e = FN<18>(__VA_ARGS__); break; case 19: e = FN<19>(__VA_ARGS__); break;        \
    case 20: e = FN<20>(__VA_ARGS__); break; case 21: e = FN<21>(__VA_ARGS__); break;        \
    case 22: e = FN<22>(__VA_ARGS__); break; case 23: e = FN<23>(__VA_ARGS__); break;        \
    case 24: e = FN<24>(__VA_ARGS__); break; case 25: e = FN<25>(__VA_ARGS__); break;        \
    case 26: e = FN<26>(__VA_ARGS__); break; case 27: e = FN<27>(__VA_ARGS__); break;        \
    case 28: e = FN<28>(__VA_ARGS__); break; case 29: e = FN<29>(__VA_ARGS__); break;        \
    case 30: e = FN<30>(__VA_ARGS__); break; case 31: e = FN<31>(__VA_ARGS__); break;        \
    case 32: e = FN<32>(__VA_ARGS__); break;                                                  \
    default: return cudaErrorNotSupported;                                                   \
  }

size_t ws_bytes_2d(const snap_problem *p, int B) {
  const size_t nfr = (size_t)B * p->desc.nt;
  return snap_align256(sizeof(BlockStat) * nfr) + snap_align256(sizeof(BwdContrib) * nfr) +
         snap_align256(sizeof(double) * nfr);
}


static int warps_blocks2(int nwarps) { return (nwarps * 32 + 127) / 128; }

cudaError_t launch_2d_forward(const snap_problem *p, int B, const double *w_hat,
                              const double *params, const double *w0, double *w, double *lambda,
                              snap_stats *stats, const SolverOpts &o, int path,
                              void *ws, cudaStream_t s) {
  (void)path;
  if (w0) return cudaErrorNotSupported;
  cudaError_t eu = ensure_2d(p);
  if (eu != cudaSuccess) return eu;
  Ws2D wk = carve_2d(p, B, ws);
  const int N = p->desc.nx;
  cudaError_t e;
  const int pid = snap_prof_begin(s, "k2d_frame");
  SNAP_DISPATCH_2D(N, fwd_m, p, B, w_hat, params, w, lambda, wk.bst, o, s);
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
                               const snap_stats *stats, double *grad_w_hat,
                               double *grad_params, void *ws, cudaStream_t s) {
  cudaError_t eu = ensure_2d(p);
  if (eu != cudaSuccess) return eu;
  Ws2D wk = carve_2d(p, B, ws);
  const int N = p->desc.nx;
  cudaError_t e;
  const int pid = snap_prof_begin(s, "k2d_frame_bwd");
  SNAP_DISPATCH_2D(N, bwd_m, p, B, grad_w, w, lambda, params, stats, grad_w_hat, wk.contrib, s);
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
