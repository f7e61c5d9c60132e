// Double-float ("double-word") arithmetic on the FP32 pipe: x = hi + lo with two floats,
// |lo| <= ulp(hi) / 2, about 48 significant bits (relative error ~ 2^-47 per operation).
//
// Algorithms: Knuth's TwoSum and Dekker's Fast2Sum for error-free addition, the FMA-based
// TwoProd for error-free multiplication, and the double-word sum / product / quotient of
// Joldes, Muller & Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic" (ACM TOMS 44(2), 2017): AccurateDWPlusDW, DWTimesDW and a
// Newton-corrected quotient.  All float operations are IEEE round-to-nearest (no fast math)
// except the reciprocal df_rcp, which on the device is the hardware approximation
// (rcp.approx, within about 1 ulp; the host build divides): it seeds the quotient, whose
// Newton correction then leaves a relative error of about 2^-46 instead of 2^-48, and it is
// the reciprocal of the float solver phase, whose steps are refined in double-float.
//
// Valid while every intermediate stays in [2^-100, 2^100] in magnitude (or is zero); callers
// check the range of their inputs and fall back to FP64 otherwise.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

// Every function is host + device: the host build runs the same arithmetic in the unit
// tests of the scalar solver on the CPU.
#define DF_INL __host__ __device__ __forceinline__

DF_INL float df_d2f(double x) {
#ifdef __CUDA_ARCH__
  return __double2float_rn(x);
#else
  return (float)x;
#endif
}

// 1/x: the hardware approximation on the device (one instruction on the critical path of
// every float Newton step; the IEEE-rounded form measured 11 % slower per Burgers launch).
DF_INL float df_rcp(float x) {
#ifdef __CUDA_ARCH__
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
#else
  return 1.0f / x;
#endif
}

struct df64 {
  float hi, lo;
  DF_INL df64() {}
  DF_INL df64(float h, float l) : hi(h), lo(l) {}
  DF_INL df64(double d) {
    hi = df_d2f(d);
    lo = df_d2f(d - (double)hi);
  }
  DF_INL explicit df64(int i) : df64((double)i) {}
  DF_INL explicit operator double() const;
};

DF_INL df64 df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return df64(s, e);
}

DF_INL df64 df_fast_two_sum(float a, float b) {  // requires |a| >= |b|
  const float s = a + b;
  const float e = b - (s - a);
  return df64(s, e);
}

DF_INL df64 operator+(df64 x, df64 y) {
  const df64 s = df_two_sum(x.hi, y.hi);
  const df64 t = df_two_sum(x.lo, y.lo);
  const df64 v = df_fast_two_sum(s.hi, s.lo + t.hi);
  return df_fast_two_sum(v.hi, t.lo + v.lo);
}

DF_INL df64 operator-(df64 x) { return df64(-x.hi, -x.lo); }
DF_INL df64 operator-(df64 x, df64 y) { return x + (-y); }

// Sum with one error-free transformation, on the leading parts only (11 operations against 20):
// the error is a few units of 2^-48 (|x| + |y|), the order of the inputs' own representation
// errors, with no bound relative to the sum under cancellation.  For stencils and accumulations
// whose operands are themselves double-float roundings.
DF_INL df64 df_add_fast(df64 x, df64 y) {
  const df64 s = df_two_sum(x.hi, y.hi);
  return df_fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
DF_INL df64 df_sub_fast(df64 x, df64 y) { return df_add_fast(x, df64(-y.hi, -y.lo)); }

// x times a power of two s (exact while the result stays normal)
DF_INL df64 df_scale2(df64 x, float s) { return df64(x.hi * s, x.lo * s); }

DF_INL df64 operator*(df64 x, df64 y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return df_fast_two_sum(p, e);
}

DF_INL df64 operator/(df64 x, df64 y) {
  const float r = df_rcp(y.hi);
  const float q1 = x.hi * r;
  // remainder x - q1 * y, exact in its leading part
  const float p = q1 * y.hi;
  const float pe = fmaf(q1, y.hi, -p);
  const float rem = ((x.hi - p) - pe) + (x.lo - q1 * y.lo);
  const float q2 = rem * r;
  return df_fast_two_sum(q1, q2);
}

DF_INL bool operator<(df64 x, df64 y) {
  return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo);
}
DF_INL bool operator>(df64 x, df64 y) { return y < x; }
DF_INL bool operator<=(df64 x, df64 y) {
  return x.hi < y.hi || (x.hi == y.hi && x.lo <= y.lo);
}
DF_INL bool operator>=(df64 x, df64 y) { return y <= x; }
DF_INL bool operator==(df64 x, df64 y) { return x.hi == y.hi && x.lo == y.lo; }
DF_INL bool operator!=(df64 x, df64 y) { return !(x == y); }

// Accumulate a float pair (h, l) into a double-float sum (used by the moment reductions).
DF_INL void df_acc(df64 &acc, float h, float l) {
  const df64 s = df_two_sum(acc.hi, h);
  acc = df_fast_two_sum(s.hi, s.lo + (acc.lo + l));
}

// Split a double into a float pair: x = h + l within 2^-48 |x| for 2^-74 <= |x| < 2^57 (and
// x = 0).  h is x rounded to float; l is the remainder x - h, an integer multiple of ulp(x)
// that is read off the low words of x and of h widened to double (their difference counts
// the ulps of x between them), converted to float and scaled by +-ulp(x).  Returns false
// when x is non-finite or outside that range.
DF_INL unsigned df_hiword(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2hiint(x);
#else
  unsigned long long b;
  memcpy(&b, &x, 8);
  return (unsigned)(b >> 32);
#endif
}
DF_INL unsigned df_loword(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2loint(x);
#else
  unsigned long long b;
  memcpy(&b, &x, 8);
  return (unsigned)b;
#endif
}
DF_INL unsigned df_fbits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  unsigned b;
  memcpy(&b, &x, 4);
  return b;
#endif
}
DF_INL float df_bitsf(unsigned b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float x;
  memcpy(&x, &b, 4);
  return x;
#endif
}
DF_INL float df_i2f(int i) {
#ifdef __CUDA_ARCH__
  return __int2float_rn(i);
#else
  return (float)i;
#endif
}

DF_INL bool df_split(double x, float &h, float &l) {
  const unsigned hw = df_hiword(x);
  const unsigned lw = df_loword(x);
  const unsigned e = (hw >> 20) & 0x7FFu;
  h = df_d2f(x);
  // low word of h widened to double: float mantissa bits 2..0 land at bits 31..29
  const int D = (int)(lw - ((df_fbits(h) & 7u) << 29));          // (|x| - |h|) / ulp(x)
  const float scale = df_bitsf((hw & 0x80000000u) | ((e - 948u) << 23));   // +-ulp(x)
  l = df_i2f(D) * scale;
  const bool zero = ((hw & 0x7FFFFFFFu) | lw) == 0u;
  if (zero) { h = 0.0f; l = 0.0f; }
  return zero || (e - 949u) <= (1080u - 949u);
}

// Split without any conversion instruction (integer operations and one FP32 add and multiply
// only, so that it keeps off the FP64 pipe, which also executes the double -> float
// conversion): h = x truncated to 24 significant bits; the 29 remaining mantissa bits D are an
// integer multiple of ulp(x); their top 23 bits D >> 6 become an exact float through the 2^23
// bias and are scaled by 2^6 ulp(x).  |x - h - l| < 2^-46 |x| and |l| < ulp(h).  Same range
// and return value as df_split.
DF_INL bool df_split_trunc(double x, float &h, float &l) {
  const unsigned hw = df_hiword(x);
  const unsigned lw = df_loword(x);
  const unsigned e = (hw >> 20) & 0x7FFu;
  const unsigned sgn = hw & 0x80000000u;
  h = df_bitsf(sgn | ((e - 896u) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
  const float f = df_bitsf(0x4B000000u | ((lw & 0x1FFFFFFFu) >> 6)) - 8388608.0f;
  l = f * df_bitsf(sgn | ((e - 942u) << 23));
  const bool zero = ((hw & 0x7FFFFFFFu) | lw) == 0u;
  const bool ok = zero || (e - 949u) <= (1080u - 949u);
  if (!ok || zero) { h = 0.0f; l = 0.0f; }
  return ok;
}

// The same truncating split in fewer operations, for the streaming moment pass: a funnel shift
// places the double's exponent and leading 23 mantissa bits in float position (the exponent
// rebias 1023 -> 127 is a flip of bit 30 for exponents in range), and l is scaled by
// 2^-46 times the power of two of h.  Zero (and every value outside [2^-74, 2^57]) returns
// false with h, l unspecified: the caller takes its FP64 path for that row.
DF_INL bool df_split_trunc_fast(double x, float &h, float &l) {
  const unsigned hw = df_hiword(x);
  const unsigned lw = df_loword(x);
  const unsigned e = (hw >> 20) & 0x7FFu;
#ifdef __CUDA_ARCH__
  const unsigned f = __funnelshift_l(lw, hw, 3);
#else
  const unsigned f = (hw << 3) | (lw >> 29);
#endif
  const unsigned hb = (((f & 0x7FFFFFFFu) ^ 0x40000000u)) | (hw & 0x80000000u);
  h = df_bitsf(hb);
  const float fl = df_bitsf(0x4B000000u | ((lw & 0x1FFFFFFFu) >> 6)) - 8388608.0f;
  l = fl * df_bitsf((hb & 0xFF800000u) - (46u << 23));
  return (e - 949u) <= (1080u - 949u);
}

// The double -> double-float conversion for values outside the range of the integer splits,
// kept out of line: inlined, the compiler predicates this rare fallback instead of branching
// around it, and a predicated conversion still takes an issue slot of the FP64 pipe on every
// call.
static __host__ __device__ __noinline__ df64 df_from_double_slow(double x) { return df64(x); }

// float -> double by integer operations only (no conversion instruction, which would take the
// FP64 pipe): the exponent is rebiased 127 -> 1023 and the mantissa widened; a subnormal float
// is normalised by its leading-zero count; zero, infinities and NaN payloads map bit for bit.
DF_INL double df_f2d(float f) {
#ifdef __CUDA_ARCH__
  const unsigned b = __float_as_uint(f);
  const unsigned ef = (b >> 23) & 0xFFu;
  unsigned m = b & 0x7FFFFFu;
  unsigned eh;
  if (ef == 0u) {
    const int p = 31 - __clz((int)m);            // leading bit of a subnormal (-1 for zero)
    eh = m ? (unsigned)(p + 874) : 0u;           // 2^(p - 149), biased by 1023
    m = m ? ((m << (23 - p)) & 0x7FFFFFu) : 0u;
  } else {
    eh = (ef == 0xFFu) ? 0x7FFu : ef + 896u;
  }
  const unsigned hi = (b & 0x80000000u) | (eh << 20) | (m >> 3);
  const unsigned lo = (m & 7u) << 29;
  return __hiloint2double((int)hi, (int)lo);
#else
  return (double)f;
#endif
}
DF_INL double df_to_double(df64 x) { return df_f2d(x.hi) + df_f2d(x.lo); }
DF_INL df64::operator double() const { return df_to_double(*this); }
