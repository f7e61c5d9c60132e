// Host build of the library's scalar slice solver and double-float helpers, for CPU unit
// tests (compiled by nvcc as host code; no kernels).
#include <string.h>

#include "../../paper_2607_00095_b300/csrc/slice_newton.cuh"

template <class T>
static SliceIn<T> make_in(const double *in, int rows, int nint) {
  SliceIn<T> d;
  d.S1 = sl_from<T>(in[0]); d.S2 = sl_from<T>(in[1]);
  d.mx = sl_from<T>(in[2]); d.mn = sl_from<T>(in[3]);
  d.uh0 = sl_from<T>(in[4]); d.uhh = sl_from<T>(in[5]);
  d.n = sl_from<T>(in[6]); d.dx = sl_from<T>(in[7]);
  d.M = sl_from<T>(in[8]); d.E = sl_from<T>(in[9]); d.C = sl_from<T>(in[10]);
  d.rows = rows;
  d.nint = nint;
  return d;
}

static SolverOpts make_opts(const double *od, const int *oi) {
  SolverOpts o;
  o.tol_kkt = od[0]; o.tol_h = od[1]; o.c1 = od[2]; o.delta0 = od[3]; o.w_keep = od[4];
  o.max_iter = oi[0]; o.max_backtracks = oi[1]; o.max_corrections = oi[2]; o.pad = 0;
  return o;
}

template <class T>
static void put(const SliceZ<T> &z, const SliceEval<T> &e, const SliceResult &R, double *oz,
                int *os, double *ores) {
  oz[0] = sl_to_double(z.a); oz[1] = sl_to_double(z.c); oz[2] = sl_to_double(z.p0);
  oz[3] = sl_to_double(z.ph); oz[4] = sl_to_double(z.lm); oz[5] = sl_to_double(z.le);
  oz[6] = sl_to_double(z.lb);
  os[0] = R.iters; os[1] = R.backtracks; os[2] = R.status; os[3] = R.corrections;
  ores[0] = sl_to_double(e.res);
  ores[1] = sl_to_double(e.hm); ores[2] = sl_to_double(e.he); ores[3] = sl_to_double(e.hb);
}

// mode 0: FP64 iteration; mode 1: float then double-float (the mixed path)
extern "C" int harness_slice(int mode, const double *in, int rows, int nint, const double *od,
                             const int *oi, double *oz, int *os, double *ores) {
  const SolverOpts o = make_opts(od, oi);
  if (mode == 0) {
    SliceIn<double> d = make_in<double>(in, rows, nint);
    SliceZ<double> z{1.0, 0.0, in[4], in[5], 0.0, 0.0, 0.0};
    SliceEval<double> e;
    SliceResult R = slice_newton(d, z, e, o);
    put(z, e, R, oz, os, ores);
  } else if (mode == 2) {
    SliceIn<df64> d = make_in<df64>(in, rows, nint);
    SliceZ<df64> z{df64(1.0f, 0.0f), df64(0.0f, 0.0f), d.uh0, d.uhh, df64(0.0f, 0.0f),
                   df64(0.0f, 0.0f), df64(0.0f, 0.0f)};
    SliceEval<df64> e;
    SliceResult R = slice_newton(d, z, e, o);
    put(z, e, R, oz, os, ores);
  } else if (mode == 3) {
    SliceIn<float> d = make_in<float>(in, rows, nint);
    SliceZ<float> z{1.0f, 0.0f, d.uh0, d.uhh, 0.0f, 0.0f, 0.0f};
    SliceEval<float> e;
    SliceResult R = slice_newton(d, z, e, o);
    put(z, e, R, oz, os, ores);
  } else {
    SliceIn<df64> d = make_in<df64>(in, rows, nint);
    SliceZ<df64> z{df64(1.0f, 0.0f), df64(0.0f, 0.0f), d.uh0, d.uhh, df64(0.0f, 0.0f),
                   df64(0.0f, 0.0f), df64(0.0f, 0.0f)};
    SliceEval<df64> e;
    SliceResult R = slice_solve_mixed(d, z, e, o, slice_opts<float>(o, o.tol_kkt), slice_opts<df64>(o, o.tol_kkt));
    put(z, e, R, oz, os, ores);
  }
  return 0;
}

// double-float arithmetic: op 0 add, 1 sub, 2 mul, 3 div; inputs/outputs as doubles
extern "C" void harness_df_op(int op, int n, const double *x, const double *y, double *out) {
  for (int i = 0; i < n; ++i) {
    const df64 a(x[i]), b(y[i]);
    df64 r = op == 0 ? a + b : op == 1 ? a - b : op == 2 ? a * b : a / b;
    out[i] = (double)r;
  }
}

extern "C" void harness_split(int n, const double *x, float *h, float *l, int *ok) {
  for (int i = 0; i < n; ++i) ok[i] = df_split(x[i], h[i], l[i]) ? 1 : 0;
}

extern "C" void harness_split_trunc(int n, const double *x, float *h, float *l, int *ok) {
  for (int i = 0; i < n; ++i) ok[i] = df_split_trunc(x[i], h[i], l[i]) ? 1 : 0;
}

extern "C" void harness_split_trunc_fast(int n, const double *x, float *h, float *l, int *ok) {
  for (int i = 0; i < n; ++i) ok[i] = df_split_trunc_fast(x[i], h[i], l[i]) ? 1 : 0;
}
