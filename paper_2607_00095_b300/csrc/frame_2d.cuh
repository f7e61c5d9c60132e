// Device side of the 2-D family C frame solve (see kern_2d.cu for the structure used):
// block reductions, the fast-diagonalisation Poisson solve of the four parity classes, the
// closed-form Newton-KKT of a frame in moment coordinates and the whole-frame forward
// projection frame2d_forward, shared by the per-problem kernel and the uneven-batch kernel.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "df64.cuh"
#include "slice_newton.cuh"
#include "snap_internal.h"

namespace {

constexpr int T2D = 256;                 // threads per frame
// float solves per right-hand side: one solve with the split TF32 class products and one
// refinement against the double-float stencil residual leave the frame rows at ~1e-11 (three
// solves: ~5e-12) against the 1e-8 tolerance
constexpr int REFINE = 2;

__device__ __forceinline__ df64 dsplit(double x) {
  float h, l;
  if (df_split(x, h, l)) return df64(h, l);
  return df_from_double_slow(x);         // out of the pair range: FP64 conversion
}

// The same with integer operations only (truncating split, |x - hi - lo| < 2^-46 |x|), for the
// per-element passes, which would otherwise load the FP64 pipe with one conversion per element
__device__ __forceinline__ df64 isplit(double x) {
  float h, l;
  if (df_split_trunc(x, h, l)) return df64(h, l);
  return df_from_double_slow(x);         // out of the pair range: FP64 conversion
}

// dx = 1 / N and 4 dx^2 of the N = 2M grid in double-float, formed at compile time: a
// conversion at run time is FP64-pipe work for every thread ahead of the frame's first loads
template <int M>
struct GridConst {
  static constexpr double dx = 1.0 / (2 * M), sc = 4.0 / ((2.0 * M) * (2.0 * M));
  static constexpr float dx_hi = (float)dx, dx_lo = (float)(dx - (double)dx_hi);
  static constexpr float sc_hi = (float)sc, sc_lo = (float)(sc - (double)sc_hi);
};

// fn(e, x) for every element e of a frame's 2 N^2 doubles x = src[e] (thread-strided), with
// FB loads in flight per thread before the first use (the passes are latency-bound otherwise)
constexpr int FB = 8;
template <int TOT, class Fn>
__device__ __forceinline__ void frame_elems(const double *__restrict__ src, Fn &&fn) {
  for (int e0 = threadIdx.x; e0 < TOT; e0 += T2D * FB) {
    double x[FB];
#pragma unroll
    for (int b = 0; b < FB; ++b) {
      const int e = e0 + b * T2D;
      x[b] = e < TOT ? __ldg(src + e) : 0.0;
    }
#pragma unroll
    for (int b = 0; b < FB; ++b) {
      const int e = e0 + b * T2D;
      if (e < TOT) fn(e, x[b]);
    }
  }
}

// x times an integer factor s of the grid (1 / (2 dx) = M, 1 / (4 dx^2) = M^2) in double-float:
// scaling both parts is exact when M is a power of two; otherwise the exact product
// (TwoProd of the leading part plus the scaled trailing part)
template <int M>
__device__ __forceinline__ df64 mul_grid(df64 x, float s) {
  if constexpr ((M & (M - 1)) == 0) {
    return df_scale2(x, s);
  } else {
    return x * df64(s, 0.0f);
  }
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

// Register-tiled form of fd_solve for M >= 8 (the same four products, the same order of
// every dot product, so the same bits): thread t of the block owns one BL x BL block of the
// output of its class (BL = M / 8; 4 classes x 8 x 8 blocks = 256 threads) and reads each
// operand row once per k as a short vector instead of twice per multiply-add.  Intermediate
// products are kept transposed so that both operands of every product are row slices;
// Qt = Q^T.
template <int BL>
__device__ __forceinline__ void fd_row(const float *p, float (&x)[BL]) {
  if constexpr (BL == 4) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  } else if constexpr (BL == 2) {
    const float2 v = *reinterpret_cast<const float2 *>(p);
    x[0] = v.x; x[1] = v.y;
  } else {
#pragma unroll
    for (int i = 0; i < BL; ++i) x[i] = p[i];
  }
}

// acc[i][j] = sum_k A[k][ia + i] B[k][jb + j] over k = 0 .. M-1 (rows of length M), in k order
template <int M, int BL>
__device__ __forceinline__ void fd_block(const float *A, const float *Bm, int ia, int jb,
                                         float (&acc)[BL][BL]) {
#pragma unroll
  for (int i = 0; i < BL; ++i)
#pragma unroll
    for (int j = 0; j < BL; ++j) acc[i][j] = 0.0f;
#pragma unroll 4
  for (int k = 0; k < M; ++k) {
    float a[BL], b[BL];
    fd_row<BL>(A + k * M + ia, a);
    fd_row<BL>(Bm + k * M + jb, b);
#pragma unroll
    for (int i = 0; i < BL; ++i)
#pragma unroll
      for (int j = 0; j < BL; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
  }
}

template <int M>
__device__ void fd_solve_tiled(float *rf, float *tf, const float *Q, const float *Qt,
                               const float *inv) {
  constexpr int MM = M * M, BL = M / 8;
  static_assert(M >= 8 && M % 8 == 0, "tiled class solve needs M = 8 k");
  const int c = threadIdx.x >> 6, bi = threadIdx.x & 63;
  const int i0 = (bi >> 3) * BL, j0 = (bi & 7) * BL;
  float acc[BL][BL];
  // T = Q^T R, kept as Tt = T^T:  Tt[j][i] = sum_k Q[k][i] R[k][j]
  fd_block<M, BL>(Q, rf + c * MM, i0, j0, acc);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < BL; ++i)
#pragma unroll
    for (int j = 0; j < BL; ++j) tf[c * MM + (j0 + j) * M + i0 + i] = acc[i][j];
  __syncthreads();
  // R = (T Q) .* inv:  R[i][n] = sum_p Tt[p][i] Q[p][n]
  fd_block<M, BL>(tf + c * MM, Q, i0, j0, acc);
#pragma unroll
  for (int i = 0; i < BL; ++i)
#pragma unroll
    for (int j = 0; j < BL; ++j)
      rf[c * MM + (i0 + i) * M + j0 + j] = acc[i][j] * inv[(i0 + i) * M + j0 + j];
  __syncthreads();
  // T = Q R, kept as T3t = T^T:  T3t[n][k] = sum_m Qt[m][k] R[m][n]
  fd_block<M, BL>(Qt, rf + c * MM, i0, j0, acc);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < BL; ++i)
#pragma unroll
    for (int j = 0; j < BL; ++j) tf[c * MM + (j0 + j) * M + i0 + i] = acc[i][j];
  __syncthreads();
  // R = T Q^T:  R[k][j] = sum_n T3t[n][k] Qt[n][j]
  fd_block<M, BL>(tf + c * MM, Qt, i0, j0, acc);
#pragma unroll
  for (int i = 0; i < BL; ++i)
#pragma unroll
    for (int j = 0; j < BL; ++j) rf[c * MM + (i0 + i) * M + j0 + j] = acc[i][j];
  __syncthreads();
}

// Tensor-core form of the class solve for M = 32 (the 64 x 64 frames): the same four products
// C = X^T Y (C[m][n] = sum_k X[k][m] Y[k][n], X and Y row-major M x M in shared memory) as
// warp-level mma.sync m16n8k8 with TF32 operands and FP32 accumulation.  Every operand is
// split into two TF32 values, x = x_big + x_small (x_small = tf32(x - x_big)), and a product
// is accumulated as x_small y_big + x_big y_small + x_big y_big, which keeps about the
// accuracy of the FP32 products (the dropped x_small y_small is below 2^-22 relative); the
// double-float refinement against the exact stencil residual is unchanged.  Eight warps:
// warp w computes rows 16 (w & 1) .. + 15 of the output of class w >> 1, all 32 columns.
// x rounded to TF32 (10 mantissa bits), to nearest with ties away from zero, by integer
// operations on the bit pattern: adding half a TF32 ulp to the magnitude bits carries into the
// kept bits (and into the exponent when the mantissa overflows), the mask drops the rest.
// Finite operands only (the class solve's are).  Integer ALU work: the conversion instruction
// would take the FP64 pipe's issue slots on this GPU.
__device__ __forceinline__ uint32_t fd_tf32(float x) {
  return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}

__device__ __forceinline__ void fd_mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                       uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Layout of the 32 x 32 operands of the tensor-core class solve (class arrays, Q, Q^T and the
// eigenvalue scaling): element (row k, column m) at k 32 + (m ^ 8 (k & 3)).  The XOR moves the
// four rows a fragment load touches (t = 0..3) to four different groups of eight banks, so the
// fragment loads are conflict-free and the accumulator stores two-way instead of eight-way.
__device__ __forceinline__ int fd_sw32(int k, int m) { return k * 32 + (m ^ (8 * (k & 3))); }

// acc[nt][.] = the 16 x 8 output tiles (rows m0 .. m0 + 15, columns 8 nt ..) of X^T Y, M = 32
__device__ __forceinline__ void fd_xty32(const float *X, const float *Y, int m0,
                                         float (&acc)[4][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[nt][e] = 0.0f;
#pragma unroll
  for (int k0 = 0; k0 < 32; k0 += 8) {
    // A = X^T: a0 (m0+g, k0+t), a1 (m0+g+8, k0+t), a2 (m0+g, k0+t+4), a3 (m0+g+8, k0+t+4)
    const float af[4] = {X[fd_sw32(k0 + t, m0 + g)], X[fd_sw32(k0 + t, m0 + g + 8)],
                         X[fd_sw32(k0 + t + 4, m0 + g)], X[fd_sw32(k0 + t + 4, m0 + g + 8)]};
    uint32_t ab[4], as[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      ab[e] = fd_tf32(af[e]);
      as[e] = fd_tf32(af[e] - __uint_as_float(ab[e]));
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      // B = Y: b0 (k0+t, 8 nt + g), b1 (k0+t+4, 8 nt + g)
      const float y0 = Y[fd_sw32(k0 + t, 8 * nt + g)], y1 = Y[fd_sw32(k0 + t + 4, 8 * nt + g)];
      const uint32_t bb0 = fd_tf32(y0), bb1 = fd_tf32(y1);
      const uint32_t bs0 = fd_tf32(y0 - __uint_as_float(bb0));
      const uint32_t bs1 = fd_tf32(y1 - __uint_as_float(bb1));
      fd_mma(acc[nt], as, bb0, bb1);
      fd_mma(acc[nt], ab, bs0, bs1);
      fd_mma(acc[nt], ab, bb0, bb1);
    }
  }
}

// out[m][n] (row-major, M = 32) from the accumulators of fd_xty32, times scale[m][n] if given
__device__ __forceinline__ void fd_store32(float *out, const float (&acc)[4][4], int m0,
                                           const float *scale) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int n = 8 * nt + 2 * t;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = m0 + g + 8 * h;
      float v0 = acc[nt][2 * h], v1 = acc[nt][2 * h + 1];
      if (scale) { v0 *= scale[fd_sw32(m, n)]; v1 *= scale[fd_sw32(m, n + 1)]; }
      out[fd_sw32(m, n)] = v0;
      out[fd_sw32(m, n + 1)] = v1;
    }
  }
}

__device__ void fd_solve_mma32(float *rf, float *tf, const float *Q, const float *Qt,
                               const float *inv) {
  constexpr int MM = 32 * 32;
  const int w = threadIdx.x >> 5, c = w >> 1, m0 = 16 * (w & 1);
  float acc[4][4];
  // T = Q^T R, kept as Tt = T^T = R^T Q
  fd_xty32(rf + c * MM, Q, m0, acc);
  __syncthreads();
  fd_store32(tf + c * MM, acc, m0, nullptr);
  __syncthreads();
  // R = (T Q) .* inv = (Tt^T Q) .* inv
  fd_xty32(tf + c * MM, Q, m0, acc);
  fd_store32(rf + c * MM, acc, m0, inv);
  __syncthreads();
  // T = Q R, kept as T3t = (Q R)^T = R^T Q^T
  fd_xty32(rf + c * MM, Qt, m0, acc);
  __syncthreads();
  fd_store32(tf + c * MM, acc, m0, nullptr);
  __syncthreads();
  // R = T Q^T = T3t^T Q^T
  fd_xty32(tf + c * MM, Qt, m0, acc);
  fd_store32(rf + c * MM, acc, m0, nullptr);
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

// Dynamic shared memory of one frame (N = 2M), float arrays: b (hi, lo), z (hi, lo), r, t
// [4 M^2 = N^2 each], Q, inv, Q^T [M^2 each], reduction scratch (110.8 KB at M = 32: two
// blocks per SM).  The frame's w_hat and w stay in global memory (L1 / L2): every pass reads
// them from there.
template <int M>
struct Smem2D {
  static constexpr int N = 2 * M, NN = N * N, MM = M * M;
  static constexpr size_t bytes = sizeof(float) * (6 * NN + 3 * MM + 64);
};

template <int M>
struct View2D {
  float *Bh, *Bl, *Zh, *Zl, *Rf, *Tf, *Q, *I, *Qt, *red;
  __device__ explicit View2D(unsigned char *base) {
    constexpr int NN = Smem2D<M>::NN, MM = Smem2D<M>::MM;
    float *f = reinterpret_cast<float *>(base);
    Bh = f; Bl = f + NN; Zh = f + 2 * NN; Zl = f + 3 * NN; Rf = f + 4 * NN; Tf = f + 5 * NN;
    Q = f + 6 * NN; I = Q + MM; Qt = I + MM; red = Qt + MM;
  }
  __device__ df64 z(int slot) const { return df64(Zh[slot], Zl[slot]); }
};

// Position of class slot s (= c M^2 + q M + p) in the class work arrays r / t: the
// tensor-core layout for M = 32, the plain one otherwise.
template <int M>
__device__ __forceinline__ int fd_slot(int s) {
  if constexpr (M == 32) return (s & ~1023) + fd_sw32((s >> 5) & 31, s & 31);
  else return s;
}

// The class eigenvectors Q, Q^T and the inverse eigenvalues into shared memory (row-major
// M x M; the tensor-core layout for M = 32).
template <int M>
__device__ __forceinline__ void load_class_factor(View2D<M> &v, const float *__restrict__ Qg,
                                                  const float *__restrict__ Ig) {
  for (int i = threadIdx.x; i < M * M; i += T2D) {
    const int k = i / M, m = i % M;
    const float q = Qg[i];
    v.Q[fd_slot<M>(i)] = q;
    v.I[fd_slot<M>(i)] = Ig[i];
    v.Qt[fd_slot<M>(m * M + k)] = q;
  }
}

// Solve (D D^T) z = b on the four classes of one frame (b already in Bh/Bl), result in
// Zh/Zl with z = 0 at each class's left-out cell.  REFINE float solves, the residual
// r = b - (D D^T) z formed in double-float between them.
template <int M>
__device__ void poisson_frame(View2D<M> &v, const df64 &scale) {
  constexpr int N = 2 * M, NN = N * N, MM = M * M;
  for (int s = threadIdx.x; s < NN; s += T2D) {
    v.Zh[s] = 0.0f;
    v.Zl[s] = 0.0f;
    v.Rf[fd_slot<M>(s)] = v.Bh[s];
  }
  __syncthreads();
  // scale = 4 dx^2 = 1 / M^2: the float solve's correction is scaled by its float image (the
  // next round's residual absorbs that rounding), the exact stencil residual by M^2
  const float scale_f = scale.hi, inv_scale_f = (float)(M * M);
  for (int round = 0; round < REFINE; ++round) {
    if constexpr (M == 32) fd_solve_mma32(v.Rf, v.Tf, v.Q, v.Qt, v.I);
    else if constexpr (M >= 8 && M % 8 == 0) fd_solve_tiled<M>(v.Rf, v.Tf, v.Q, v.Qt, v.I);
    else fd_solve<M>(v.Rf, v.Tf, v.Q, v.I);
    for (int s = threadIdx.x; s < NN; s += T2D) {
      const df64 zz = df_add_fast(v.z(s), df64(v.Rf[fd_slot<M>(s)] * scale_f, 0.0f));
      v.Zh[s] = zz.hi;
      v.Zl[s] = zz.lo;
    }
    __syncthreads();
    if (round + 1 < REFINE) {
      for (int s = threadIdx.x; s < NN; s += T2D) {
        const int c = s / MM, q = (s % MM) / M, p = s % M;
        const int base = c * MM;
        const df64 zc = v.z(s);
        const df64 nb = df_add_fast(df_add_fast(v.z(base + q * M + (p + 1) % M),
                                                 v.z(base + q * M + (p + M - 1) % M)),
                                     df_add_fast(v.z(base + ((q + 1) % M) * M + p),
                                                 v.z(base + ((q + M - 1) % M) * M + p)));
        const df64 az = mul_grid<M>(df_sub_fast(df_scale2(zc, 4.0f), nb), inv_scale_f);
        const df64 r = df_sub_fast(df64(v.Bh[s], v.Bl[s]), az);
        v.Rf[fd_slot<M>(s)] = r.hi + r.lo;
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
    const df64 zz = df_sub_fast(v.z(s), g0[s / MM]);
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

// fn(e, x, y) with x = a[e], y = b[e] for every element e of two frame fields, batched as
// frame_elems
template <int TOT, class Fn>
__device__ __forceinline__ void frame_elems2(const double *__restrict__ a,
                                             const double *__restrict__ b, Fn &&fn) {
  for (int e0 = threadIdx.x; e0 < TOT; e0 += T2D * FB) {
    double x[FB], y[FB];
#pragma unroll
    for (int k = 0; k < FB; ++k) {
      const int e = e0 + k * T2D;
      x[k] = e < TOT ? __ldg(a + e) : 0.0;
      y[k] = e < TOT ? __ldg(b + e) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < FB; ++k) {
      const int e = e0 + k * T2D;
      if (e < TOT) fn(e, x[k], y[k]);
    }
  }
}

// (D x)(i, j) of a field held as float pairs in shared memory, xp[2][N][N]
template <int M>
__device__ __forceinline__ df64 div_at_pairs(const float2 *xp, int i, int j, const df64 &h2) {
  constexpr int N = 2 * M, NN = N * N;
  const float2 ue = xp[j * N + (i + 1) % N], uw = xp[j * N + (i + N - 1) % N];
  const float2 vn = xp[NN + ((j + 1) % N) * N + i], vs = xp[NN + ((j + N - 1) % N) * N + i];
  return mul_grid<M>(df_add_fast(df_sub_fast(df64(ue.x, ue.y), df64(uw.x, uw.y)),
                                 df_sub_fast(df64(vn.x, vn.y), df64(vs.x, vs.y))), h2.hi);
}

// (D w)(i, j) of a field held as doubles in shared memory, component 0 in w0, 1 in w1
template <int M>
__device__ __forceinline__ df64 div_at_smem(const double *w0, const double *w1, int i, int j,
                                            const df64 &h2) {
  constexpr int N = 2 * M;
  const df64 ue = isplit(w0[j * N + (i + 1) % N]);
  const df64 uw = isplit(w0[j * N + (i + N - 1) % N]);
  const df64 vn = isplit(w1[((j + 1) % N) * N + i]);
  const df64 vs = isplit(w1[((j + N - 1) % N) * N + i]);
  return mul_grid<M>(df_add_fast(df_sub_fast(ue, uw), df_sub_fast(vn, vs)), h2.hi);
}

// (D^T z) for element e of w[2][N][N] (component e / N^2)
template <int M>
__device__ __forceinline__ df64 divT_at(const View2D<M> &v, int e, const df64 &h2) {
  constexpr int N = 2 * M, NN = N * N;
  const int comp = e / NN, cell = e % NN, i = cell % N, j = cell / N;
  if (comp == 0) return mul_grid<M>(df_sub_fast(v.z(cell_slot<M>(i - 1, j)), v.z(cell_slot<M>(i + 1, j))), h2.hi);
  return mul_grid<M>(df_sub_fast(v.z(cell_slot<M>(i, j - 1)), v.z(cell_slot<M>(i, j + 1))), h2.hi);
}

// Forward projection of frame f of one sample by the whole block (T2D threads, every thread
// must call it): src / dst are the frame's w_hat / w [2][N][N], pr the sample's parameters
// (K0, r2), lam_s the sample's multipliers (nt N^2 divergence rows, then nt energy rows).
// The block's dynamic shared memory (Smem2D<M>::bytes) is passed in v; *out receives the
// frame's statistics (written by thread 0).
//
// Global memory is touched by batched loads only (frame_elems): w_hat is read once into shared
// memory as float pairs for the divergence stencil (in the Poisson work area, which is free
// until the solve) and twice more, batched, by the element passes after the solve; the written
// w is kept in shared memory (in the right-hand-side and product areas, free after the solve)
// for the residual of the written field.
template <int M>
__device__ void frame2d_forward(View2D<M> &v, const double *__restrict__ src,
                                const double *__restrict__ pr, int f, int nt,
                                const float *__restrict__ Qg, const float *__restrict__ Ig,
                                double *__restrict__ dst, double *__restrict__ lam_s,
                                BlockStat *__restrict__ out, const SolverOpts &o) {
  constexpr int N = 2 * M, NN = N * N;
  const df64 h2((float)N * 0.5f, 0.0f);          // 1 / (2 dx), exact
  const df64 dx(GridConst<M>::dx_hi, GridConst<M>::dx_lo);
  const df64 scale(GridConst<M>::sc_hi, GridConst<M>::sc_lo);   // 4 dx^2
  load_class_factor<M>(v, Qg, Ig);
  // w_hat as float pairs in the Poisson work area (z hi / lo, r, t: 4 N^2 floats = 2 N^2 pairs)
  float2 *xp = reinterpret_cast<float2 *>(v.Zh);
  df64 a0(0.0f, 0.0f);
  float xinf = 0.0f;
  frame_elems<2 * NN>(src, [&](int e, double xd) {
    const df64 x = isplit(xd);
    xp[e] = make_float2(x.hi, x.lo);
    a0 = df_add_fast(a0, x * x);
    xinf = fabs_max(xinf, x.hi);
  });
  __syncthreads();
  // b = D w_hat on every cell
  float d2 = 0.0f, dinf = 0.0f;
  for (int cell = threadIdx.x; cell < NN; cell += T2D) {
    const int i = cell % N, j = cell / N;
    const df64 dv = div_at_pairs<M>(xp, i, j, h2);
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
  // ||y||^2 = ||D^T z||^2 = z . (D D^T z) = z . b (D D^T z = b on every cell: the right-hand
  // side of each class sums to zero), and the stopping-test extremes from bounds:
  // |y_e| <= 2 h2 max |z|, |x_e - y_e| <= max |x| + that (looser bounds make the test stricter)
  df64 a2(0.0f, 0.0f);
  float zinf = 0.0f;
  for (int cell = threadIdx.x; cell < NN; cell += T2D) {
    const df64 zc = v.z(cell);
    a2 = df_add_fast(a2, zc * df64(v.Bh[cell], v.Bl[cell]));
    zinf = fabs_max(zinf, zc.hi);
  }
  a0 = block_sumdf(a0, v.red);
  a2 = block_sumdf(a2, v.red);
  d2 = block_sumf(d2, v.red);
  dinf = block_max(dinf, v.red);
  xinf = block_max(xinf, v.red);
  zinf = block_max(zinf, v.red);
  const float yinf = 2.0f * h2.hi * zinf * (1.0f + 1e-6f), pinf = (xinf + yinf) * (1.0f + 1e-6f);
  // scalar Newton-KKT of the frame (thread 0), broadcast through shared memory
  __shared__ float zs[10];
  __shared__ SliceResult Rs;
  __shared__ float Ks[2];
  if (threadIdx.x == 0) {
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
  // write w = a w_hat + c y (global memory, and in shared memory over its own y), lambda_div
  // = mu z.  On the moment family w = a x + c y the gradient of the Lagrangian is
  // alpha w - x + mu y = p x + r y with the frame's scalar residuals p = alpha a - 1 and
  // r = alpha c + mu (formed in double-float), so ||grad L||_inf comes from the leading parts
  // of x and y; ||w - x||^2 and ||w||^2 follow from the moments (x . y = ||y||^2: y is the
  // orthogonal projection of x onto the range of D_a^T).
  double *w0 = reinterpret_cast<double *>(v.Bh);   // component 0: b hi / lo area (N^2 doubles)
  double *w1 = reinterpret_cast<double *>(v.Rf);   // component 1: r / t area (N^2 doubles)
  const df64 one(1.0f, 0.0f);
  const float pg = (AL * A - one).hi, rg = (AL * Cc + MU).hi;
  float ginf = 0.0f;
  frame_elems<2 * NN>(src, [&](int e, double xd) {
    const df64 y = divT_at<M>(v, e, h2);
    const df64 x = isplit(xd);
    const df64 w = df_add_fast(A * x, Cc * y);
    const double wd = df_to_double(w);
    dst[e] = wd;
    if (e < NN) w0[e] = wd; else w1[e - NN] = wd;
    ginf = fabs_max(ginf, fmaf(pg, x.hi, rg * y.hi));
  });
  const df64 am1 = A - one;
  const df64 obj2 = am1 * am1 * a0 + (df64(2.0f, 0.0f) * am1 * Cc + Cc * Cc) * a2;
  const df64 w2 = A * A * a0 + (df64(2.0f, 0.0f) * A * Cc + Cc * Cc) * a2;
  double *lb = lam_s + (size_t)f * NN;
  for (int cell = threadIdx.x; cell < NN; cell += T2D) {
    const int i = cell % N, j = cell / N;
    lb[cell] = (i < 2 && j < 2) ? 0.0 : df_to_double(MU * v.z(cell_slot<M>(i, j)));
  }
  __syncthreads();
  float hinf_all = 0.0f, hinf_act = 0.0f;
  for (int cell = threadIdx.x; cell < NN; cell += T2D) {
    const int i = cell % N, j = cell / N;
    const float dv = div_at_smem<M>(w0, w1, i, j, h2).hi;   // the written w
    hinf_all = fabs_max(hinf_all, dv);
    if (!(i < 2 && j < 2)) hinf_act = fabs_max(hinf_act, dv);
  }
  ginf = block_max(ginf, v.red);
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
    st.obj = 0.5 * df_to_double(obj2);
    *out = st;
    lam_s[(size_t)nt * NN + f] = df_to_double(KAP);
  }
}

// Adjoint of frame f of one sample by the whole block (T2D threads, every thread must call
// it).  At the solution D_a w = 0, so S = J W^-1 J^T is block diagonal:
// (1/alpha) diag(D_a D_a^T, dx^4 ||w||^2).  Hence b_div = (D_a D_a^T)^-1 D_a gbar (one Poisson
// solve), b_K = w^T gbar / (dx^2 ||w||^2), a = (gbar - D_a^T b_div - b_K dx^2 w) / alpha.
// gsrc / wsrc are the frame's dL/dw and w [2][N][N], kap its energy multiplier, pr the
// sample's parameters (K0, r2); writes a into dst (NaN when bad) and the frame's contribution
// to dL/d(K0, r2) into *contrib (thread 0).
template <int M>
__device__ void frame2d_backward(View2D<M> &v, const double *__restrict__ gsrc,
                                 const double *__restrict__ wsrc, double kap,
                                 const double *__restrict__ pr, int f, int nt, bool bad,
                                 const float *__restrict__ Qg, const float *__restrict__ Ig,
                                 double *__restrict__ dst, BwdContrib *__restrict__ contrib) {
  constexpr int N = 2 * M, NN = N * N;
  const df64 h2((float)N * 0.5f, 0.0f);
  const df64 dx(GridConst<M>::dx_hi, GridConst<M>::dx_lo);
  const df64 scale(GridConst<M>::sc_hi, GridConst<M>::sc_lo);   // 4 dx^2
  load_class_factor<M>(v, Qg, Ig);
  // gbar as float pairs in the Poisson work area for the divergence stencil (as the forward)
  float2 *gp2 = reinterpret_cast<float2 *>(v.Zh);
  df64 dot(0.0f, 0.0f), ww(0.0f, 0.0f);
  frame_elems2<2 * NN>(wsrc, gsrc, [&](int e, double wd, double gd) {
    const df64 x = isplit(wd), gx = isplit(gd);
    gp2[e] = make_float2(gx.hi, gx.lo);
    dot = df_add_fast(dot, x * gx);
    ww = df_add_fast(ww, x * x);
  });
  __syncthreads();
  for (int cell = threadIdx.x; cell < NN; cell += T2D) {
    const int i = cell % N, j = cell / N;
    const df64 dv = div_at_pairs<M>(gp2, i, j, h2);
    const int s = cell_slot<M>(i, j);
    v.Bh[s] = dv.hi;
    v.Bl[s] = dv.lo;
  }
  __syncthreads();
  poisson_frame<M>(v, scale);
  dot = block_sumdf(dot, v.red);
  ww = block_sumdf(ww, v.red);
  const df64 dx2 = dx * dx;
  const df64 alpha = df64(1.0f, 0.0f) + dsplit(kap) * dx2;
  const df64 bK = dot / (dx2 * ww);
  const df64 ialpha = df64(1.0f, 0.0f) / alpha;
  const df64 bKdx2 = bK * dx2;
  frame_elems2<2 * NN>(gsrc, wsrc, [&](int e, double gd, double wd) {
    const df64 y = divT_at<M>(v, e, h2);
    const df64 a = df_sub_fast(df_sub_fast(isplit(gd), y), bKdx2 * isplit(wd)) * ialpha;
    dst[e] = bad ? NAN : df_to_double(a);
  });
  if (threadIdx.x == 0) {
    const double t = (double)f / (double)(nt - 1);
    const double ex = exp(-pr[1] * t);
    const double bk = df_to_double(bK);
    // h_K = 1/2 dx^2 ||w||^2 - K0 exp(-r2 t): dL/dK0 += b_K e, dL/dr2 += -b_K t K0 e
    *contrib = BwdContrib{bk * ex, -bk * t * pr[0] * ex, 0.0, 0.0};
  }
}

// dL/d(K0, r2) of one sample from its nt frame contributions c[0..nt) (one warp, fixed order,
// so the bits do not depend on which warp runs it); kCoherent reads through L2 only
// (contributions written by other blocks of a running kernel).
template <bool kCoherent>
__device__ __forceinline__ void frame2d_param_grad(const BwdContrib *__restrict__ c, int nt,
                                                   bool bad, double *__restrict__ gp, int lane) {
  double s0 = 0.0, s1 = 0.0;
  for (int f = lane; f < nt; f += 32) {
    if (kCoherent) {
      s0 += __ldcg(&c[f].bm);
      s1 += __ldcg(&c[f].bex);
    } else {
      s0 += c[f].bm;
      s1 += c[f].bex;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if (lane == 0) {
    gp[0] = bad ? NAN : s0;
    gp[1] = bad ? NAN : s1;
  }
}

}  // namespace
