// Double-single arithmetic: a real is the unevaluated sum hi + lo of two floats
// (about 48 significant bits); error-free transformations (Knuth's TwoSum,
// Dekker's product via FMA) keep the rounding error of each operation near
// 2^-46 relative.  Used where FP64 latency and throughput on GB300 (1/64 of the
// FP32 rate per SM) would dominate: the serial-heavy projected eigenproblem.
#pragma once

#include <cuda_runtime.h>

namespace swi {
namespace ds {

struct df {
  float h, l;
};
struct __align__(16) dc {  // complex
  df re, im;
};

__device__ __forceinline__ df mk(float h, float l) { return df{h, l}; }
__device__ __forceinline__ df from_d(double x) {
  const float h = __double2float_rn(x);
  return df{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double to_d(df a) { return (double)a.h + (double)a.l; }

// x = hi + lo from the bit fields of x, on the integer and FP32 pipes (GB300's
// FP64 pipe is the scarce one): hi is x rounded to 24 significant bits, lo the
// signed 29-bit remainder rounded to a float, so |x - hi - lo| <= 2^-48 |x| as
// with an FP64 split.  Magnitudes below 2^-74 (where the remainder would leave
// the float range) and near the top of the float range take the FP64 route.
__device__ __forceinline__ void split_bits(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int top = (unsigned int)(b >> 32);
  const unsigned int sgn = top & 0x80000000u;
  const int e = (int)((top >> 20) & 0x7ff);
  if (e >= 949 && e <= 1149) {
    const unsigned int up = (unsigned int)(b >> 28) & 1u;  // round half up on the first dropped bit
    const unsigned int fb = ((unsigned int)(e - 896) << 23 | ((unsigned int)(b >> 29) & 0x7fffffu)) + up;
    hi = __uint_as_float(sgn | fb);
    const int rem = (int)((unsigned int)b & 0x1fffffffu) - (int)(up << 29);  // x - hi in units of 2^(e-1075)
    const float t = (float)rem * __uint_as_float((unsigned int)(e - 948) << 23);
    lo = sgn ? -t : t;
  } else {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
  }
}

// (s, e) += a * b with a, b double-single: the product is formed exactly up to
// its tail with FMA, the head added with TwoSum (Knuth), errors kept in e.
__device__ __forceinline__ void fma_acc(float& s, float& e, float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  float pe = fmaf(ah, bh, -p);
  pe = fmaf(ah, bl, pe);
  pe = fmaf(al, bh, pe);
  const float t = s + p;
  const float bp = t - s;
  const float err = (s - (t - bp)) + (p - bp);
  s = t;
  e += err + pe;
}

__device__ __forceinline__ df quick_two_sum(float a, float b) {
  const float s = a + b;
  return df{s, b - (s - a)};
}
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return df{s, (a - (s - bb)) + (b - bb)};
}
// Sum with an absolute error ~2^-48 (|a| + |b|) (the low parts are added in
// plain float): normwise accurate, which is what unitary updates need.
__device__ __forceinline__ df add(df a, df b) {
  df s = two_sum(a.h, b.h);
  s.l += a.l + b.l;
  return quick_two_sum(s.h, s.l);
}
// power-of-two scaling (exact)
__device__ __forceinline__ df ldexp_(df a, int e) { return df{ldexpf(a.h, e), ldexpf(a.l, e)}; }
__device__ __forceinline__ df neg(df a) { return df{-a.h, -a.l}; }
__device__ __forceinline__ df sub(df a, df b) { return add(a, neg(b)); }
__device__ __forceinline__ df mul(df a, df b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ df mulf(df a, float b) {
  const float p = a.h * b;
  float e = fmaf(a.h, b, -p);
  e = fmaf(a.l, b, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ df div(df a, df b) {
  const float q1 = a.h / b.h;
  const df r = sub(a, mulf(b, q1));
  const float q2 = r.h / b.h;
  const df r2 = sub(r, mulf(b, q2));
  const float q3 = r2.h / b.h;
  df q = quick_two_sum(q1, q2);
  return add(q, df{q3, 0.f});
}
// 1/sqrt(a) for a > 0: float estimate and two Newton steps in double-single
__device__ __forceinline__ df rsqrt(df a) {
  df x = df{rsqrtf(a.h), 0.f};
  for (int it = 0; it < 2; ++it) {
    // x <- x (3 - a x^2) / 2
    const df ax2 = mul(a, mul(x, x));
    const df t = sub(df{3.f, 0.f}, ax2);
    x = mulf(mul(x, t), 0.5f);
  }
  return x;
}
__device__ __forceinline__ df sqrt_(df a) {
  if (a.h <= 0.f) return df{0.f, 0.f};
  return mul(a, rsqrt(a));
}
__device__ __forceinline__ float approx(df a) { return a.h + a.l; }
__device__ __forceinline__ float absf(df a) { return fabsf(a.h + a.l); }

__device__ __forceinline__ dc cadd(dc a, dc b) { return dc{add(a.re, b.re), add(a.im, b.im)}; }
__device__ __forceinline__ dc csub(dc a, dc b) { return dc{sub(a.re, b.re), sub(a.im, b.im)}; }
__device__ __forceinline__ dc cmul(dc a, dc b) {
  return dc{sub(mul(a.re, b.re), mul(a.im, b.im)), add(mul(a.re, b.im), mul(a.im, b.re))};
}
// conj(a) * b
__device__ __forceinline__ dc cmulc_l(dc a, dc b) {
  return dc{add(mul(a.re, b.re), mul(a.im, b.im)), sub(mul(a.re, b.im), mul(a.im, b.re))};
}
__device__ __forceinline__ dc cscale(dc a, df s) { return dc{mul(a.re, s), mul(a.im, s)}; }
__device__ __forceinline__ dc cconj(dc a) { return dc{a.re, neg(a.im)}; }
__device__ __forceinline__ df cabs2(dc a) { return add(mul(a.re, a.re), mul(a.im, a.im)); }
__device__ __forceinline__ float cabs1f(dc a) { return absf(a.re) + absf(a.im); }
__device__ __forceinline__ dc czero() { return dc{df{0.f, 0.f}, df{0.f, 0.f}}; }
__device__ __forceinline__ dc cfrom(double2 v) { return dc{from_d(v.x), from_d(v.y)}; }
__device__ __forceinline__ double2 cto(dc a) { return make_double2(to_d(a.re), to_d(a.im)); }
__device__ __forceinline__ dc cdiv(dc a, dc b) {
  const df d = cabs2(b);
  const dc n = cmulc_l(b, a);  // conj(b) a
  return dc{div(n.re, d), div(n.im, d)};
}

}  // namespace ds
}  // namespace swi
