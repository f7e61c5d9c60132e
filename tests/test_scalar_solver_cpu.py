"""CPU tests of the library's per-slice scalar solver and double-float arithmetic.

tests/csrc/slice_harness.cu compiles the library headers slice_newton.cuh / df64.cuh as
host code (nvcc, no kernels), so the exact iteration the kernels run can be checked here
against numpy, exact rational arithmetic and the oracle."""
import ctypes as C
import math
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

from oracle import problems, solve
from paper_2607_00095_b300 import synthetic

HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None
dp = C.POINTER(C.c_double)
ip = C.POINTER(C.c_int)
fp = C.POINTER(C.c_float)


def lib():
    global _lib
    if _lib is None:
        out = os.path.join(tempfile.mkdtemp(), "libslice_harness.so")
        subprocess.check_call(["/usr/local/cuda/bin/nvcc", "-O2", "-std=c++17", "-Xcompiler", "-fPIC",
                               "-shared", "-o", out, os.path.join(HERE, "csrc", "slice_harness.cu")])
        L = C.CDLL(out)
        L.harness_slice.argtypes = [C.c_int, dp, C.c_int, C.c_int, dp, ip, dp, ip, dp]
        L.harness_df_op.argtypes = [C.c_int, C.c_int, dp, dp, dp]
        L.harness_split.argtypes = [C.c_int, dp, fp, fp, ip]
        L.harness_split_trunc.argtypes = [C.c_int, dp, fp, fp, ip]
        L.harness_split_trunc_fast.argtypes = [C.c_int, dp, fp, fp, ip]
        _lib = L
    return _lib


def solve_slice(mode, inp, rows=7, nint=126, tol=1e-10, max_iter=50):
    inp = np.ascontiguousarray(inp, np.float64)
    od = np.array([tol, 1e-8, 1e-4, 1e-8, 0.01])
    oi = np.array([max_iter, 30, 0], np.int32)
    oz = np.zeros(7)
    st = np.zeros(4, np.int32)
    res = np.zeros(4)
    lib().harness_slice(mode, inp.ctypes.data_as(dp), rows, nint, od.ctypes.data_as(dp),
                        oi.ctypes.data_as(ip), oz.ctypes.data_as(dp), st.ctypes.data_as(ip),
                        res.ctypes.data_as(dp))
    return oz, st, res


def slice_inputs(uh, pr, b, k, nx, nt, floor=0.05):
    ih = nx // 2
    dx = 1.0 / nx
    row = uh[b, k]
    mask = np.ones(nx, bool)
    mask[0] = mask[ih] = False
    it = row[mask]
    g = pr[b, :nx]
    M = dx * math.fsum(g)
    E0 = dx * math.fsum(g * g)
    E = max(E0 * math.exp(-pr[b, nx] * k / (nt - 1)), M * M + floor)
    return np.array([math.fsum(it), math.fsum(it * it), it.max(), it.min(), row[0], row[ih],
                     nx - 2, dx, M, E, pr[b, nx + 1 + k]])


def test_double_float_ops_accuracy():
    rng = np.random.default_rng(0)
    n = 4000
    x = rng.normal(size=n) * np.exp(rng.uniform(-20, 20, size=n))
    y = rng.normal(size=n) * np.exp(rng.uniform(-20, 20, size=n))
    for op, fn in ((0, lambda a, b: a + b), (1, lambda a, b: a - b), (2, lambda a, b: a * b),
                   (3, lambda a, b: a / b)):
        out = np.zeros(n)
        lib().harness_df_op(op, n, x.ctypes.data_as(dp), y.ctypes.data_as(dp), out.ctypes.data_as(dp))
        for i in range(0, n, 37):
            # exact value of the operation on the df64 images of x, y (both rounded to 48 bits)
            exact = fn(Fraction(x[i]), Fraction(y[i]))
            if op in (0, 1):
                scale = abs(Fraction(x[i])) + abs(Fraction(y[i]))
            else:
                scale = abs(exact)
            err = abs(Fraction(out[i]) - exact) / scale
            assert err < 2.0 ** -44, (op, x[i], y[i], float(err))


def test_split_pair_exactness_and_range():
    rng = np.random.default_rng(1)
    x = rng.normal(size=5000) * np.exp(rng.uniform(-45, 35, size=5000))
    ties = [1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, -(1.0 + 2.0 ** -24), 2.0 - 2.0 ** -25,
            3.0 * (1.0 + 2.0 ** -24), 1.0 + 2.0 ** -24 + 2.0 ** -52]    # float ties and near-ties
    x = np.concatenate([x, [0.0, -0.0, 1.0, -1.0, 2.0 ** -74, 2.0 ** 56, 1.999999999999,
                            np.nextafter(2.0, 0)], ties])
    h = np.zeros(len(x), np.float32)
    l = np.zeros(len(x), np.float32)
    ok = np.zeros(len(x), np.int32)
    lib().harness_split(len(x), x.ctypes.data_as(dp), h.ctypes.data_as(fp), l.ctypes.data_as(fp),
                        ok.ctypes.data_as(ip))
    ax = np.abs(x)
    inrange = (ax == 0) | ((ax >= 2.0 ** -74) & (ax < 2.0 ** 58))
    np.testing.assert_array_equal(ok.astype(bool), inrange)
    for i in np.nonzero(ok)[0]:
        err = abs(Fraction(float(h[i])) + Fraction(float(l[i])) - Fraction(x[i]))
        assert err <= Fraction(abs(x[i])) * Fraction(2) ** -47, (x[i], h[i], l[i])
        assert float(h[i]) == float(np.float32(x[i]))          # h = x rounded to float


def test_fast_truncating_split_matches_truncating_split():
    """The funnel-shift split gives the same pair as the truncating split wherever it accepts
    (every value in range except zero, which it sends to the FP64 path)."""
    rng = np.random.default_rng(3)
    x = rng.normal(size=20000) * np.exp(rng.uniform(-52, 41, size=20000))
    x = np.concatenate([x, [0.0, -0.0, 1.0, -1.0, 2.0 ** -74, -(2.0 ** -74), 2.0 ** 57 * 1.5,
                            np.nextafter(2.0 ** 58, 0), 2.0 ** 58, 2.0 ** -75, np.inf, np.nan]])
    out = []
    for fn in (lib().harness_split_trunc, lib().harness_split_trunc_fast):
        h = np.zeros(len(x), np.float32)
        l = np.zeros(len(x), np.float32)
        ok = np.zeros(len(x), np.int32)
        fn(len(x), x.ctypes.data_as(dp), h.ctypes.data_as(fp), l.ctypes.data_as(fp),
           ok.ctypes.data_as(ip))
        out.append((h, l, ok.astype(bool)))
    (h0, l0, ok0), (h1, l1, ok1) = out
    np.testing.assert_array_equal(ok1, ok0 & (x != 0))
    np.testing.assert_array_equal(h1[ok1], h0[ok1])
    np.testing.assert_array_equal(l1[ok1], l0[ok1])


def test_truncating_split_exactness_and_range():
    """The integer-only split: h = x truncated to 24 significant bits, |x - h - l| < 2^-46 |x|,
    the same range as the rounding split; checked in exact rational arithmetic."""
    rng = np.random.default_rng(2)
    x = rng.normal(size=5000) * np.exp(rng.uniform(-45, 35, size=5000))
    x = np.concatenate([x, [0.0, -0.0, 1.0, -1.0, 2.0 ** -74, -(2.0 ** -74), 2.0 ** 56,
                            np.nextafter(2.0 ** 58, 0), 2.0 ** 58, 2.0 ** -75, np.inf, np.nan,
                            1.999999999999, np.nextafter(2.0, 0), 1.0 + 2.0 ** -24,
                            -(1.0 + 2.0 ** -52)]])
    h = np.zeros(len(x), np.float32)
    l = np.zeros(len(x), np.float32)
    ok = np.zeros(len(x), np.int32)
    lib().harness_split_trunc(len(x), x.ctypes.data_as(dp), h.ctypes.data_as(fp),
                              l.ctypes.data_as(fp), ok.ctypes.data_as(ip))
    ax = np.abs(x)
    inrange = (ax == 0) | ((ax >= 2.0 ** -74) & (ax < 2.0 ** 58))
    np.testing.assert_array_equal(ok.astype(bool), inrange)
    for i in np.nonzero(ok)[0]:
        xf = Fraction(x[i])
        err = abs(Fraction(float(h[i])) + Fraction(float(l[i])) - xf)
        assert err < abs(xf) * Fraction(2) ** -46 or err == 0, (x[i], h[i], l[i])
        # h is x truncated toward zero to 24 significant bits
        assert abs(Fraction(float(h[i]))) <= abs(xf)
        assert abs(xf - Fraction(float(h[i]))) < abs(Fraction(float(h[i]))) * Fraction(2) ** -23 or x[i] == 0


@pytest.mark.parametrize("mode", [0, 1])
def test_scalar_solver_matches_oracle_per_slice(mode):
    nx, nt, B = 128, 12, 4
    uh, pr = synthetic.gen_1d(1001, B, nx, nt, "B")
    ue, le, so, S, b = solve.project_1d("B", nx, nt, pr, uh)
    assert (so["status"] == 0).all()
    U = ue.reshape(B, nt, nx)
    for s in range(B):
        for k in range(1, nt):
            z, st, res = solve_slice(mode, slice_inputs(uh, pr, s, k, nx, nt))
            assert st[2] == 0 and res[0] <= 1e-10
            a, c, p0, ph = z[:4]
            u = a * uh[s, k] + c
            u[0], u[nx // 2] = p0, ph
            assert np.abs(u - U[s, k]).max() <= 1e-8 * np.abs(U[s, k]).max()
            lam = np.array([le[s, nx + k], le[s, nx + nt + k], le[s, nx + 2 * nt + k]])
            assert np.abs(z[4:] - lam).max() <= 1e-6 * np.abs(lam).max()


def test_mixed_and_fp64_solvers_agree_on_burgers_slices():
    """Every slice of 64 samples of the Burgers workload: both precisions converge to the
    same KKT point (within the stopping tolerance)."""
    nx, nt = 128, 100
    uh, pr = synthetic.gen_1d(1001, 64, nx, nt, "B")
    worst = 0.0
    for s in range(64):
        for k in range(1, nt):
            inp = slice_inputs(uh, pr, s, k, nx, nt)
            z1, s1, r1 = solve_slice(1, inp)
            z0, s0, r0 = solve_slice(0, inp)
            assert s1[2] == 0 and s0[2] == 0, (s, k, s1, s0)
            du = max(abs(z1[0] - z0[0]) * np.abs(uh[s, k]).max() + abs(z1[1] - z0[1]),
                     abs(z1[2] - z0[2]), abs(z1[3] - z0[3]))
            worst = max(worst, du)
    assert worst <= 1e-8
