// Jacobian-vector product of the mixed path in float-float arithmetic.
//
// J v = v/dt - Delta_d w,  w = L_gamma v / 2 + q v (Eq. Jacobi) is linear in v, so
// GMRES only needs it to the accuracy of its own stop test, not bit-for-bit
// FP64.  GB300 executes FP64 at 1/61 of the FP32 rate, so the FP64 stencil is
// bound by the FP64 pipe; here every value is an unevaluated sum hi + lo of two
// floats (48 significand bits, relative rounding about 2^-48 per operation) and
// the stencil runs on the FP32 pipe with error-free transformations: Knuth's
// two-sum for additions and an FMA-based two-product for products.  The FP64
// inputs are split into hi + lo by integer operations on their bit patterns (the
// hardware's double-float conversions run on the FP64 pipe, as slowly as the FP64
// stencil itself); the output takes one FP64 addition.  All primitives use the
// _rn intrinsics so that the compiler cannot contract or reassociate them.
//
// The plain FP64 path keeps k_jvp2d; this kernel serves F32/BF16-factor solves.
#include "pfc_internal.cuh"

namespace pfc {
namespace {

constexpr int TX = 32, TY = 16, R = 3;
constexpr int AX = TX + 2 * R, AY = TY + 2 * R;  // 38 x 22 staged points
constexpr int NT = 256;                          // 32 x 8 threads, 2 outputs each

struct ff {
  float hi, lo;
};

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

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
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);  // exact error of the product
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_scale(ff a, float c) { return {__fmul_rn(a.hi, c), __fmul_rn(a.lo, c)}; }  // c a power of 2

// Unscaled 5-point Laplacian (e + w) + (n + s) - 4 c.
__device__ __forceinline__ ff ff_lap(ff c, ff e, ff w, ff n, ff s) {
  return ff_add(ff_add(ff_add(e, w), ff_add(n, s)), ff_neg(ff_scale(c, 4.0f)));
}

__global__ void __launch_bounds__(NT) k_jvp2d_ff(Geo g, const double* __restrict__ v,
                                                 const double* __restrict__ vscale, const double* __restrict__ q,
                                                 double idt, double* __restrict__ Jv, const int* __restrict__ skip,
                                              const IterArgs* __restrict__ ia) {
  if (skip && *skip) return;
  if (ia) {  // graph mode: J Z_j into V_(j+1)
    v = ia->z;
    q = ia->q;
    idt = ia->idt;
    Jv = ia->w;
  }
  __shared__ ff sV[AY][AX];
  __shared__ ff sQ[AY - 4][AX - 4];
  __shared__ ff sL[AY - 2][AX - 2];
  __shared__ ff sW[AY - 4][AX - 4];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tid = threadIdx.x + threadIdx.y * 32;
  const double sc = vscale ? *vscale : 1.0;
  for (int i = tid; i < AX * AY; i += NT) {
    const int ly = i / AX, lx = i - ly * AX;
    const long long idx = wrap(x0 + lx - R, g.nx) + (long long)g.nx * wrap(y0 + ly - R, g.ny);
    sV[ly][lx] = ff_of(vscale ? sc * v[idx] : v[idx]);
  }
  for (int i = tid; i < (AX - 4) * (AY - 4); i += NT) {
    const int ly = i / (AX - 4), lx = i - ly * (AX - 4);
    const long long idx = wrap(x0 + lx - 1, g.nx) + (long long)g.nx * wrap(y0 + ly - 1, g.ny);
    sQ[ly][lx] = ff_of(q[idx]);
  }
  __syncthreads();
  for (int i = tid; i < (AX - 2) * (AY - 2); i += NT) {
    const int ly = i / (AX - 2) + 1, lx = i - (ly - 1) * (AX - 2) + 1;
    sL[ly - 1][lx - 1] = ff_lap(sV[ly][lx], sV[ly][lx + 1], sV[ly][lx - 1], sV[ly + 1][lx], sV[ly - 1][lx]);
  }
  __syncthreads();
  const ff ih2 = ff_of(g.ih2), hih4 = ff_of(0.5 * g.ih2 * g.ih2), c0 = ff_of(0.5 * (1.0 - g.gamma));
  for (int i = tid; i < (AX - 4) * (AY - 4); i += NT) {
    const int ly = i / (AX - 4) + 2, lx = i - (ly - 2) * (AX - 4) + 2;
    const int a = ly - 1, b = lx - 1;
    const ff Lv = sL[a][b];
    const ff LLv = ff_lap(Lv, sL[a][b + 1], sL[a][b - 1], sL[a + 1][b], sL[a - 1][b]);
    const ff vv = sV[ly][lx];
    // w = c0 v + ih2 Lv + (ih4/2) LLv + q v
    sW[ly - 2][lx - 2] = ff_add(ff_add(ff_mul(c0, vv), ff_mul(ih2, Lv)),
                                ff_add(ff_mul(hih4, LLv), ff_mul(sQ[ly - 2][lx - 2], vv)));
  }
  __syncthreads();
  const ff fidt = ff_of(idt);
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int tx = threadIdx.x, ty = threadIdx.y + 8 * r;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx < g.nx && gy < g.ny) {
      const int a = ty + 1, b = tx + 1;
      const ff Lw = ff_lap(sW[a][b], sW[a][b + 1], sW[a][b - 1], sW[a + 1][b], sW[a - 1][b]);
      const ff out = ff_add(ff_mul(sV[ty + R][tx + R], fidt), ff_neg(ff_mul(ih2, Lw)));
      Jv[gx + (long long)g.nx * gy] = ff_to_double(out);
    }
  }
}

}  // namespace

void launch_jvp2d_ff(const Geo& g, const double* v, const double* vscale, const double* q, double idt, double* Jv,
                     const int* skip, cudaStream_t st, const IterArgs* ia) {
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY);
  k_jvp2d_ff<<<grid, dim3(32, 8), 0, st>>>(g, v, vscale, q, idt, Jv, skip, ia);
  count_launches(1);
}

}  // namespace pfc
