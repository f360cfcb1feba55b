// Float-float ("df64") arithmetic on the FP32 pipes: a value is hi + lo with two
// floats, |lo| <= ulp(hi)/2, about 48 significant bits (relative error ~1e-14).
// Built from the classical error-free transformations: Knuth's TwoSum, the
// Fast2Sum of Dekker (|a| >= |b|), and TwoProd through a fused multiply-add.
// Used for the FP64-accurate products of the refinement residual, where GB300's
// FP64 pipe is far slower than its FP32 pipes.
#pragma once
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace ncs {

struct f2 {
  float hi, lo;
};

__device__ __forceinline__ f2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__device__ __forceinline__ f2 fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ f2 two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ f2 f2_from_double(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

__device__ __forceinline__ double f2_to_double(f2 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  const f2 s = two_sum(a.hi, b.hi);
  const f2 t = two_sum(a.lo, b.lo);
  f2 r = fast_two_sum(s.hi, s.lo + t.hi);
  return fast_two_sum(r.hi, r.lo + t.lo);
}

__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) { return f2_add(a, {-b.hi, -b.lo}); }

__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ f2 f2_mul_f(f2 a, float b) {
  f2 p = two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ f2 f2_sqr(f2 a) {
  f2 p = two_prod(a.hi, a.hi);
  p.lo = fmaf(2.0f * a.hi, a.lo, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

// Table for log: entries i = 0..63 hold c_i = 1 + (i + 0.5)/64 as (log c_i hi, lo, 1/c_i hi, lo).
constexpr int kLogTable = 64;

// log(v) for v > 0 given as float-float: v = 2^e m, m in [1, 2); m = c_i (1 + delta)
// with |delta| <= 1/129; log v = e log 2 + log c_i + log(1 + delta), the last by its
// Taylor series through delta^6 (the delta and delta^2 terms in float-float).
__device__ __forceinline__ f2 f2_log(f2 v, const float4* __restrict__ tab) {
  const int ib = __float_as_int(v.hi);
  const int e = ((ib >> 23) & 0xff) - 127;
  const float m = __int_as_float((ib & 0x007fffff) | 0x3f800000);
  const float vl = ldexpf(v.lo, -e);  // exact scaling of the low word
  const int i = min(kLogTable - 1, (int)((m - 1.0f) * (float)kLogTable));
  const float ci = 1.0f + ((float)i + 0.5f) / (float)kLogTable;
  const float4 t = tab[i];
  // delta = (m - c_i + vl) / c_i
  const f2 num = two_sum(m - ci, vl);  // m - c_i is exact (both in [1, 2), within 1/64)
  const f2 d = f2_mul(num, f2{t.z, t.w});
  // log(1 + d) = d - d^2/2 + d^3 (1/3 - d/4 + d^2/5 - d^3/6)
  const f2 d2 = f2_sqr(d);
  const float dh = d.hi;
  const float tail = dh * dh * dh * (0.333333333f + dh * (-0.25f + dh * (0.2f + dh * (-0.166666667f))));
  f2 r = f2_add(d, f2{-0.5f * d2.hi, -0.5f * d2.lo});
  r = f2_add(r, f2{tail, 0.0f});
  // + log c_i
  r = f2_add(r, f2{t.x, t.y});
  // + e log 2, with log 2 as a float-float constant
  const f2 ln2 = {0.693147182464599609375f, -1.904654323148236e-09f};
  return f2_add(r, f2_mul_f(ln2, (float)e));
}

// G from the float-float squared distance (eqs. Gextonsurface / Gintonsurface):
//   exterior: u - log(1 + u), interior: u + log 4 - log(d^2 + 2d), u = 2/d.
// 1/d from the FP32 reciprocal square root refined by one Newton step in float-float.
template <int MODE>
__device__ __forceinline__ f2 green_f2(f2 d2, const float4* __restrict__ tab) {
  const float y = rsqrt_mufu(d2.hi);
  const f2 yy = two_prod(y, y);
  f2 m = two_prod(d2.hi, yy.hi);
  m.lo = fmaf(d2.hi, yy.lo, fmaf(d2.lo, yy.hi, m.lo));
  const float r = (1.0f - m.hi) - m.lo;  // 1 - d^2 y^2, ~1e-7
  // 1/d = y (1 + r/2 + 3 r^2 / 8): u = 2/d
  const f2 u = fast_two_sum(2.0f * y, y * (r + 0.75f * r * r));
  if (MODE == 0) {
    const f2 v = f2_add(f2{1.0f, 0.0f}, u);
    return f2_sub(u, f2_log(v, tab));
  }
  const f2 d = f2_mul(d2, f2{0.5f * u.hi, 0.5f * u.lo});  // d = d^2 (u/2)
  const f2 v = f2_add(d2, f2{2.0f * d.hi, 2.0f * d.lo});
  const f2 ln4 = {1.38629436492919921875f, -3.809308646296472e-09f};
  return f2_sub(f2_add(u, ln4), f2_log(v, tab));
}

// One pair term in float-float: target offset a (3 float-float words), source
// (hi, lo) quadruples (offset, strength); returns G * rho.
template <int MODE>
__device__ __forceinline__ f2 pair_f2(const f2* a, float4 sh, float4 sl, const float4* __restrict__ tab) {
  f2 dx = two_sum(a[0].hi, -sh.x);
  dx = fast_two_sum(dx.hi, dx.lo + (a[0].lo - sl.x));
  f2 dy = two_sum(a[1].hi, -sh.y);
  dy = fast_two_sum(dy.hi, dy.lo + (a[1].lo - sl.y));
  f2 dz = two_sum(a[2].hi, -sh.z);
  dz = fast_two_sum(dz.hi, dz.lo + (a[2].lo - sl.z));
  const f2 d2 = f2_add(f2_add(f2_sqr(dx), f2_sqr(dy)), f2_sqr(dz));
  return f2_mul(green_f2<MODE>(d2, tab), f2{sh.w, sl.w});
}

}  // namespace ncs
