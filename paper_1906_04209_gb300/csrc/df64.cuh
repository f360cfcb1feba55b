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

// Split on a power-of-two grid: hi = the multiple of q nearest v, lo = v - hi rounded to
// FP32. With |v| <= 2^23 q (q = 2^e, qinv = 2^-e) hi is exact in FP32, and so is the
// difference of two such highs on the same grid (an integer multiple of q below 2^24 q):
// the pair kernels then form an offset's high word with one subtraction, no TwoSum.
// The representation error is |lo| 2^-24 <= q 2^-25.
__device__ __forceinline__ f2 f2_split_grid(double v, double q, double qinv) {
  const double h = rint(v * qinv) * q;
  return {(float)h, (float)(v - h)};
}

// Grid spacing for the offsets of one block: every thread passes the largest |offset| it
// will split (per coordinate, m[3]); the block's maximum B_c gives q_c = 2^(e_c - 23) with
// 2^e_c >= B_c, so |v| <= 2^23 q_c for every offset of the block. All threads must call it;
// `scratch` is 3 words of shared memory, `qs` 6 shared doubles that receive q_c and 1/q_c.
// Non-negative doubles order as their bit patterns.
__device__ __forceinline__ void block_grid(const double* m, unsigned long long* scratch, double* qs) {
  __syncthreads();
  if (threadIdx.x < 3) scratch[threadIdx.x] = 0ull;
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double v = m[c];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&scratch[c], (unsigned long long)__double_as_longlong(v));
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    int e = 0;
    frexp(__longlong_as_double((long long)scratch[threadIdx.x]), &e);  // B = f 2^e, f in [1/2, 1); e = 0 for B = 0
    qs[threadIdx.x] = ldexp(1.0, e - 23);
    qs[3 + threadIdx.x] = ldexp(1.0, 23 - e);
  }
  __syncthreads();
}

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

// a + b in any order: TwoSum on the high words, the low words added once (the
// "sloppy" float-float addition: accurate to ~2^-47 of max(|a|, |b|)).
__device__ __forceinline__ f2 f2_add_sloppy(f2 a, f2 b) {
  const f2 s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

// Table for log: entries i = 0..63 hold c_i = 1 + (i + 0.5)/64 as (log c_i hi, lo, 1/c_i hi, lo).
constexpr int kLogTable = 64;

// log(v / 2^k) for v > 0 given as float-float (v.hi normal, |v.lo| <= ulp(v.hi)).
// v = 2^e m, m in [1, 2); the top six bits of m pick c_i, m = c_i (1 + delta) with
// |delta| <= 1/128, and log v = e log 2 + log c_i + log(1 + delta), the last by its
// Taylor series through delta^6 (delta and delta^2 carried in float-float). The sums
// are ordered so that only two TwoSums and one final renormalisation are needed.
__device__ __forceinline__ f2 f2_log_pow2(f2 v, int k, const float4* __restrict__ tab) {
  const int ib = __float_as_int(v.hi);
  const int e = (ib >> 23) - 127;
  const float m = __int_as_float((ib & 0x007fffff) | 0x3f800000);
  const float vl = v.lo * __int_as_float((127 - e) << 23);  // v.lo / 2^e, exact
  const int i = (ib >> 17) & (kLogTable - 1);
  const float ci = __int_as_float(0x3f800000 | (i << 17) | (1 << 16));
  const float4 t = tab[i];
  // delta = (m - c_i + vl) / c_i; m - c_i is exact (both in [1, 2), 1/128 apart at most)
  const float nh = m - ci;
  const float dh = nh * t.z;
  const f2 d = fast_two_sum(dh, fmaf(nh, t.w, fmaf(vl, t.z, fmaf(nh, t.z, -dh))));
  // log(1 + d) = d - d^2/2 + d^3 (1/3 - d/4 + d^2/5 - d^3/6)
  const float q = d.hi * d.hi;
  const float ql = fmaf(d.hi, d.hi, -q) + 2.0f * d.hi * d.lo;
  const float tail =
      q * d.hi * fmaf(d.hi, fmaf(d.hi, fmaf(d.hi, -0.166666667f, 0.2f), -0.25f), 0.333333333f);
  const float rs = fmaf(-0.5f, q, d.hi);               // |d| > |d^2 / 2|: Fast2Sum
  const float re = (-0.5f * q) - (rs - d.hi);
  const float rl = re + d.lo + fmaf(-0.5f, ql, tail);
  // + log c_i
  const f2 s1 = two_sum(t.x, rs);
  const float l1 = s1.lo + (rl + t.y);
  // + (e - k) log 2, log 2 as a float-float constant
  const float ef = (float)(e - k);
  const float Eh = ef * 0.693147182464599609375f;
  const float El = fmaf(ef, 0.693147182464599609375f, -Eh) + ef * -1.904654323148236e-09f;
  const f2 s2 = two_sum(Eh, s1.hi);
  return fast_two_sum(s2.hi, s2.lo + (l1 + El));
}

// G from the float-float squared distance (eqs. Gextonsurface / Gintonsurface):
//   exterior: G_E = u - log(1 + u),
//   interior: G_I = u + log 4 - log(d^2 + 2d) = u - log((d^2 + 2d) / 4),   u = 2/d.
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
  f2 v;
  if (MODE == 0) {
    v = two_sum(u.hi, 1.0f);
    v = fast_two_sum(v.hi, v.lo + u.lo);
  } else {
    v = f2_add_sloppy(f2_mul(d2, u), d2);  // 2d = d^2 u
  }
  const f2 L = f2_log_pow2(v, MODE == 0 ? 0 : 2, tab);
  return f2_add_sloppy(u, f2{-L.hi, -L.lo});
}

// acc += G * rho for one pair in float-float: target offset a (3 float-float words),
// source (hi, lo) quadruples (offset, strength). The sum is compensated (Ogita, Rump and
// Oishi's Sum2): acc.hi is the running FP32 sum, acc.lo collects every rounding error by
// TwoSum plus the low words, and the caller folds hi + lo into FP64 per tile.
template <int MODE>
__device__ __forceinline__ void pair_f2_acc(const f2* a, float4 sh, float4 sl, const float4* __restrict__ tab,
                                            f2& acc) {
  // offset differences as unnormalised (hi, lo) pairs, |lo| a few ulp of |hi|
  f2 dx = two_sum(a[0].hi, -sh.x), dy = two_sum(a[1].hi, -sh.y), dz = two_sum(a[2].hi, -sh.z);
  dx.lo += a[0].lo - sl.x;
  dy.lo += a[1].lo - sl.y;
  dz.lo += a[2].lo - sl.z;
  // d^2 = sum hi^2 (exact products, two TwoSums) + sum (2 hi lo + lo^2)
  const float px = dx.hi * dx.hi, py = dy.hi * dy.hi, pz = dz.hi * dz.hi;
  const f2 s1 = two_sum(px, py);
  const f2 s2 = two_sum(s1.hi, pz);
  float lo = (s1.lo + s2.lo) + (fmaf(dx.hi, dx.hi, -px) + fmaf(dy.hi, dy.hi, -py) + fmaf(dz.hi, dz.hi, -pz));
  lo = fmaf(fmaf(2.0f, dx.hi, dx.lo), dx.lo, lo);
  lo = fmaf(fmaf(2.0f, dy.hi, dy.lo), dy.lo, lo);
  lo = fmaf(fmaf(2.0f, dz.hi, dz.lo), dz.lo, lo);
  const f2 d2 = fast_two_sum(s2.hi, lo);
  const f2 g = f2_mul(green_f2<MODE>(d2, tab), f2{sh.w, sl.w});
  const f2 t = two_sum(acc.hi, g.hi);
  acc.hi = t.hi;
  acc.lo += t.lo + g.lo;
}

// ---- packed float-float: two independent float-float values per f32x2 register pair --
// The same error-free transformations as above on add/sub/mul/fma.rn.f32x2, which round
// each 32-bit half exactly as the scalar instruction does; a thread evaluates its two
// targets' pairs with one packed instruction where the scalar code issues two. Integer
// steps (exponent and table index of the logarithm), the MUFU reciprocal square root and
// the table loads stay per half.
struct f2x2 {
  f32x2 hi, lo;
};

__device__ __forceinline__ f32x2 x2_neg(f32x2 a) { return a ^ 0x8000000080000000ull; }
__device__ __forceinline__ f32x2 x2_splat(float v) { return x2_pack(v, v); }

__device__ __forceinline__ f2x2 two_sum_x2(f32x2 a, f32x2 b) {
  const f32x2 s = x2_add(a, b);
  const f32x2 bb = x2_sub(s, a);
  return {s, x2_add(x2_sub(a, x2_sub(s, bb)), x2_sub(b, bb))};
}

__device__ __forceinline__ f2x2 fast_two_sum_x2(f32x2 a, f32x2 b) {
  const f32x2 s = x2_add(a, b);
  return {s, x2_sub(b, x2_sub(s, a))};
}

__device__ __forceinline__ f2x2 two_prod_x2(f32x2 a, f32x2 b) {
  const f32x2 p = x2_mul(a, b);
  return {p, x2_fma(a, b, x2_neg(p))};
}

__device__ __forceinline__ f2x2 f2_mul_x2(f2x2 a, f2x2 b) {
  f2x2 p = two_prod_x2(a.hi, b.hi);
  p.lo = x2_fma(a.hi, b.lo, x2_fma(a.lo, b.hi, p.lo));
  return fast_two_sum_x2(p.hi, p.lo);
}

__device__ __forceinline__ f2x2 f2_add_sloppy_x2(f2x2 a, f2x2 b) {
  const f2x2 s = two_sum_x2(a.hi, b.hi);
  return fast_two_sum_x2(s.hi, x2_add(s.lo, x2_add(a.lo, b.lo)));
}

// f2_log_pow2 on both halves (see there).
__device__ __forceinline__ f2x2 f2_log_pow2_x2(f2x2 v, int k, const float4* __restrict__ tab) {
  float vh[2], vlo[2];
  x2_unpack(v.hi, vh[0], vh[1]);
  x2_unpack(v.lo, vlo[0], vlo[1]);
  float m[2], ci[2], sc[2], ef[2];
  float4 t[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int ib = __float_as_int(vh[h]);
    const int e = (ib >> 23) - 127;
    m[h] = __int_as_float((ib & 0x007fffff) | 0x3f800000);
    sc[h] = __int_as_float((127 - e) << 23);
    const int i = (ib >> 17) & (kLogTable - 1);
    ci[h] = __int_as_float(0x3f800000 | (i << 17) | (1 << 16));
    t[h] = tab[i];
    ef[h] = (float)(e - k);
  }
  const f32x2 vl = x2_mul(x2_pack(vlo[0], vlo[1]), x2_pack(sc[0], sc[1]));  // v.lo / 2^e, exact
  const f32x2 tx = x2_pack(t[0].x, t[1].x), ty = x2_pack(t[0].y, t[1].y), tz = x2_pack(t[0].z, t[1].z),
              tw = x2_pack(t[0].w, t[1].w);
  const f32x2 nh = x2_sub(x2_pack(m[0], m[1]), x2_pack(ci[0], ci[1]));
  const f32x2 dh = x2_mul(nh, tz);
  const f2x2 d = fast_two_sum_x2(dh, x2_fma(nh, tw, x2_fma(vl, tz, x2_fma(nh, tz, x2_neg(dh)))));
  const f32x2 q = x2_mul(d.hi, d.hi);
  const f32x2 ql = x2_fma(x2_mul(x2_splat(2.0f), d.hi), d.lo, x2_fma(d.hi, d.hi, x2_neg(q)));
  const f32x2 poly =
      x2_fma(d.hi, x2_fma(d.hi, x2_fma(d.hi, x2_splat(-0.166666667f), x2_splat(0.2f)), x2_splat(-0.25f)),
             x2_splat(0.333333333f));
  const f32x2 tail = x2_mul(x2_mul(q, d.hi), poly);
  const f32x2 m05 = x2_splat(-0.5f);
  const f32x2 rs = x2_fma(m05, q, d.hi);  // |d| > |d^2 / 2|: Fast2Sum
  const f32x2 re = x2_fma(m05, q, x2_neg(x2_sub(rs, d.hi)));
  const f32x2 rl = x2_add(x2_add(re, d.lo), x2_fma(m05, ql, tail));
  const f2x2 s1 = two_sum_x2(tx, rs);
  const f32x2 l1 = x2_add(s1.lo, x2_add(rl, ty));
  const f32x2 E = x2_pack(ef[0], ef[1]);
  const f32x2 Eh = x2_mul(E, x2_splat(0.693147182464599609375f));
  const f32x2 El = x2_fma(E, x2_splat(-1.904654323148236e-09f), x2_fma(E, x2_splat(0.693147182464599609375f), x2_neg(Eh)));
  const f2x2 s2 = two_sum_x2(Eh, s1.hi);
  return fast_two_sum_x2(s2.hi, x2_add(s2.lo, x2_add(l1, El)));
}

template <int MODE>
__device__ __forceinline__ f2x2 green_f2_x2(f2x2 d2, const float4* __restrict__ tab) {
  float a0, a1;
  x2_unpack(d2.hi, a0, a1);
  const f32x2 y = x2_pack(rsqrt_mufu(a0), rsqrt_mufu(a1));
  const f2x2 yy = two_prod_x2(y, y);
  f2x2 m = two_prod_x2(d2.hi, yy.hi);
  m.lo = x2_fma(d2.hi, yy.lo, x2_fma(d2.lo, yy.hi, m.lo));
  const f32x2 r = x2_sub(x2_sub(x2_splat(1.0f), m.hi), m.lo);  // 1 - d^2 y^2, ~1e-7
  // 1/d = y (1 + r/2 + 3 r^2 / 8): u = 2/d
  const f2x2 u = fast_two_sum_x2(x2_mul(x2_splat(2.0f), y), x2_mul(y, x2_fma(x2_mul(x2_splat(0.75f), r), r, r)));
  f2x2 v;
  if (MODE == 0) {
    v = two_sum_x2(u.hi, x2_splat(1.0f));
    v = fast_two_sum_x2(v.hi, x2_add(v.lo, u.lo));
  } else {
    v = f2_add_sloppy_x2(f2_mul_x2(d2, u), d2);  // 2d = d^2 u
  }
  const f2x2 L = f2_log_pow2_x2(v, MODE == 0 ? 0 : 2, tab);
  return f2_add_sloppy_x2(u, f2x2{x2_neg(L.hi), x2_neg(L.lo)});
}

// pair_f2_acc for two targets at once (lane h of every packed value is target h): the
// packed target offsets A[0..2], one staged source (hi, lo) broadcast to both lanes.
// GRID: targets and sources were split by f2_split_grid on the same grid, so the high
// words subtract exactly and each offset is (hi difference, lo difference), unnormalised
// but with |lo| <= q far below |hi| for the separated pairs these kernels sum.
template <int MODE, bool GRID = false>
__device__ __forceinline__ void pair_f2_acc_x2(const f2x2* A, float4 sh, float4 sl, const float4* __restrict__ tab,
                                               f2x2& acc) {
  f2x2 dx, dy, dz;
  if constexpr (GRID) {
    dx = f2x2{x2_sub(A[0].hi, x2_splat(sh.x)), x2_sub(A[0].lo, x2_splat(sl.x))};
    dy = f2x2{x2_sub(A[1].hi, x2_splat(sh.y)), x2_sub(A[1].lo, x2_splat(sl.y))};
    dz = f2x2{x2_sub(A[2].hi, x2_splat(sh.z)), x2_sub(A[2].lo, x2_splat(sl.z))};
  } else {
    dx = two_sum_x2(A[0].hi, x2_splat(-sh.x));
    dy = two_sum_x2(A[1].hi, x2_splat(-sh.y));
    dz = two_sum_x2(A[2].hi, x2_splat(-sh.z));
    dx.lo = x2_add(dx.lo, x2_sub(A[0].lo, x2_splat(sl.x)));
    dy.lo = x2_add(dy.lo, x2_sub(A[1].lo, x2_splat(sl.y)));
    dz.lo = x2_add(dz.lo, x2_sub(A[2].lo, x2_splat(sl.z)));
  }
  const f32x2 px = x2_mul(dx.hi, dx.hi), py = x2_mul(dy.hi, dy.hi), pz = x2_mul(dz.hi, dz.hi);
  const f2x2 s1 = two_sum_x2(px, py);
  const f2x2 s2 = two_sum_x2(s1.hi, pz);
  f32x2 lo = x2_add(x2_add(s1.lo, s2.lo),
                    x2_add(x2_add(x2_fma(dx.hi, dx.hi, x2_neg(px)), x2_fma(dy.hi, dy.hi, x2_neg(py))),
                           x2_fma(dz.hi, dz.hi, x2_neg(pz))));
  const f32x2 two = x2_splat(2.0f);
  lo = x2_fma(x2_fma(two, dx.hi, dx.lo), dx.lo, lo);
  lo = x2_fma(x2_fma(two, dy.hi, dy.lo), dy.lo, lo);
  lo = x2_fma(x2_fma(two, dz.hi, dz.lo), dz.lo, lo);
  const f2x2 d2 = fast_two_sum_x2(s2.hi, lo);
  const f2x2 g = f2_mul_x2(green_f2_x2<MODE>(d2, tab), f2x2{x2_splat(sh.w), x2_splat(sl.w)});
  const f2x2 t = two_sum_x2(acc.hi, g.hi);
  acc.hi = t.hi;
  acc.lo = x2_add(acc.lo, x2_add(t.lo, g.lo));
}

}  // namespace ncs
