// Float-float arithmetic on the FP32 pipe, for the mixed path's FP64-width
// vector work (GB300 executes FP64 at 1/61 of the FP32 rate).  A value is an
// unevaluated sum hi + lo of two floats (48 significand bits); additions use
// Knuth's two-sum and products an FMA-based two-product (error-free
// transformations), so every operation rounds at about 2^-48 relative.  FP64
// values are split into hi + lo by integer operations on their bit patterns (the
// hardware's double <-> float conversions run on the FP64 pipe, as slowly as FP64
// arithmetic itself).  All primitives use the _rn intrinsics so that the
// compiler cannot contract or reassociate them.
#pragma once

#include <cuda_runtime.h>

namespace pfc {

struct ff {
  float hi, lo;
};

// hi = x with its significand cut to 24 bits (toward zero), lo = the remaining 29
// bits rounded to 24: hi + lo = x to 48 bits.  Values below 2^-126 in magnitude
// (far below any the scheme produces) become 0; |lo| below 2^-126 becomes 0.
__device__ __forceinline__ ff ff_of(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  const unsigned sign = h32 & 0x80000000u;
  const int e = (int)((h32 >> 20) & 0x7ffu) - 1023;  // unbiased exponent
  if (e < -126) return {0.0f, 0.0f};
  const unsigned frac23 = ((h32 & 0xfffffu) << 3) | (l32 >> 29);
  const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | frac23);
  const unsigned rest = l32 & 0x1fffffffu;  // 29 bits worth 2^(e - 52) each
  float lo = 0.0f;
  if (rest != 0u && e - 52 >= -126)  // the scale 2^(e - 52) is a normal float
    lo = __fmul_rn(__uint2float_rn(rest), __uint_as_float((unsigned)(e - 52 + 127) << 23));
  return {hi, sign ? -lo : lo};
}
// Exact widening of a float by its bit pattern (no FP64-pipe conversion).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  if (ex == 0u) return 0.0;  // zero (no subnormals here: see ff_of)
  const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(ex - 127 + 1023) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}
__device__ __forceinline__ double ff_to_double(ff a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

// Vectors stored as float pairs: element i of an FP64-sized array holds (hi, lo) of a
// normalised pair (|lo| <= ulp(hi) / 2) in its 8 bytes.  The mixed path keeps its Krylov
// basis this way, so the Arnoldi sweeps need no split per element.
__device__ __forceinline__ ff ld_pair(const double* p, long long i) {
  const float2 t = reinterpret_cast<const float2*>(p)[i];
  return {t.x, t.y};
}
__device__ __forceinline__ void st_pair(double* p, long long i, ff a) {
  reinterpret_cast<float2*>(p)[i] = make_float2(a.hi, a.lo);
}

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  const ff t = two_sum(a.lo, b.lo);
  s = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
// x as a normalised float pair (hi = x rounded to a float, lo = the rest rounded): 2^-48 relative.
__device__ __forceinline__ ff ff_pair_of(double x) {
  const ff a = ff_of(x);
  return fast_two_sum(a.hi, a.lo);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);  // exact error of the product
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_scale(ff a, float c) { return {__fmul_rn(a.hi, c), __fmul_rn(a.lo, c)}; }  // c a power of 2

// A faster split for streaming kernels: hi = x cut to 24 significand bits, lo =
// the next 23 bits, read as 2^(e-23) (1 + m) - 2^(e-23) (one float subtraction, exact):
// hi + lo = x to 2^-46 relative for |x| >= 2^-102; below that lo = 0, and below
// 2^-126 hi = 0 as well.
__device__ __forceinline__ ff ff_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  const unsigned sign = h32 & 0x80000000u;
  const int fexp = (int)((h32 >> 20) & 0x7ffu) - 896;  // float exponent field of hi
  const unsigned mant = __funnelshift_l(l32, h32, 3) & 0x7fffffu;
  if (fexp <= 0) return {0.0f, 0.0f};
  const float hi = __uint_as_float(sign | ((unsigned)fexp << 23) | mant);
  if (fexp <= 23) return {hi, 0.0f};
  const unsigned eb = sign | ((unsigned)(fexp - 23) << 23);
  return {hi, __fsub_rn(__uint_as_float(eb | ((l32 >> 6) & 0x7fffffu)), __uint_as_float(eb))};
}
// x cut to a float (24 significand bits, toward zero; 0 below 2^-126).
__device__ __forceinline__ float f32_cut(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  const int fexp = (int)((h32 >> 20) & 0x7ffu) - 896;
  if (fexp <= 0) return 0.0f;
  return __uint_as_float((h32 & 0x80000000u) | ((unsigned)fexp << 23) | (__funnelshift_l(l32, h32, 3) & 0x7fffffu));
}

// Product a * b as an unnormalised pair (p, e): p = fl(a.hi b.hi), e = its exact
// error plus the cross terms (a.lo b.lo, about 2^-48 of the product, is dropped).
__device__ __forceinline__ ff ff_prod(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return {p, e};
}
// Running sum acc + x with the rounding error of the leading parts kept in lo
// (no renormalisation: lo stays far below hi over the few hundred terms a thread adds).
__device__ __forceinline__ ff ff_acc(ff acc, ff x) {
  const ff s = two_sum(acc.hi, x.hi);
  return {s.hi, __fadd_rn(__fadd_rn(acc.lo, x.lo), s.lo)};
}

// Sums of several float-float terms at the cost of one two-sum per term: the leading parts are
// added with their exact rounding errors (two-sum), the trailing parts and those errors are summed
// in plain FP32 (each far below the leading sum), and the result is renormalised once.  The
// error stays near 2^-46 of the terms' magnitude, like ff_add's, at about half its instructions.
// (e + w) + (n + s) - 4 c: the unscaled 5-point Laplacian.
__device__ __forceinline__ ff ff_lap5(ff c, ff e, ff w, ff n, ff s) {
  const ff a = two_sum(e.hi, w.hi), b = two_sum(n.hi, s.hi);
  const ff t = two_sum(a.hi, b.hi);
  const ff u = two_sum(t.hi, -4.0f * c.hi);  // times 4: exact
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(e.lo, w.lo), __fadd_rn(n.lo, s.lo)),
                             __fadd_rn(__fadd_rn(a.lo, b.lo), __fadd_rn(t.lo, __fmaf_rn(-4.0f, c.lo, u.lo))));
  return fast_two_sum(u.hi, lo);
}
// a0 b0 + a1 b1 + a2 b2 + a3 b3 from the unnormalised products of ff_prod.
__device__ __forceinline__ ff ff_dot4(ff a0, ff b0, ff a1, ff b1, ff a2, ff b2, ff a3, ff b3) {
  const ff p0 = ff_prod(a0, b0), p1 = ff_prod(a1, b1), p2 = ff_prod(a2, b2), p3 = ff_prod(a3, b3);
  const ff s01 = two_sum(p0.hi, p1.hi), s23 = two_sum(p2.hi, p3.hi);
  const ff t = two_sum(s01.hi, s23.hi);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(p0.lo, p1.lo), __fadd_rn(p2.lo, p3.lo)),
                             __fadd_rn(__fadd_rn(s01.lo, s23.lo), t.lo));
  return fast_two_sum(t.hi, lo);
}
// a0 b0 - a1 b1.
__device__ __forceinline__ ff ff_dot2m(ff a0, ff b0, ff a1, ff b1) {
  const ff p0 = ff_prod(a0, b0), p1 = ff_prod(a1, b1);
  const ff t = two_sum(p0.hi, -p1.hi);
  return fast_two_sum(t.hi, __fadd_rn(__fsub_rn(p0.lo, p1.lo), t.lo));
}

}  // namespace pfc
