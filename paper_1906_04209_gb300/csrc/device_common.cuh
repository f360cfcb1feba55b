// Device helpers shared by the kernels: patch frames and the on-surface Neumann
// Green's functions of the unit sphere (Kaye & Greengard, Section 2.1).
#pragma once
#include <cuda_runtime.h>

namespace ncs {

constexpr double kLn4 = 1.3862943611198906188;
constexpr float kLn2f = 0.69314718055994530942f;

// Patch frame for unit centre c: e1 = (z x c)/|z x c| (x-axis at the poles), e2 = c x e1.
__device__ __forceinline__ void patch_frame(double cx, double cy, double cz, double* e1, double* e2) {
  const double ax = -cy, ay = cx, na2 = ax * ax + ay * ay;
  if (na2 >= 1e-24) {
    const double inv = 1.0 / sqrt(na2);
    e1[0] = ax * inv;
    e1[1] = ay * inv;
    e1[2] = 0.0;
  } else {
    e1[0] = 1.0;
    e1[1] = 0.0;
    e1[2] = 0.0;
  }
  e2[0] = cy * e1[2] - cz * e1[1];
  e2[1] = cz * e1[0] - cx * e1[2];
  e2[2] = cx * e1[1] - cy * e1[0];
}

// Global offset of a local offset (o0, o1, o2) in the frame (e1, e2, c).
__device__ __forceinline__ void frame_apply(const double* e1, const double* e2, double cx, double cy,
                                            double cz, double o0, double o1, double o2, double* g) {
  g[0] = o0 * e1[0] + o1 * e2[0] + o2 * cx;
  g[1] = o0 * e1[1] + o1 * e2[1] + o2 * cy;
  g[2] = o0 * e1[2] + o1 * e2[2] + o2 * cz;
}

// Bare MUFU approximations (PTX rsqrt.approx / lg2.approx with denormals flushed):
// the arguments here are never denormal, and the IEEE-mode wrappers cost extra
// instructions per pair.
__device__ __forceinline__ float rsqrt_mufu(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float lg2_mufu(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// G(d) from d^2, eqs. (Gextonsurface) / (Gintonsurface), one logarithm each:
//   exterior: G_E = u - log(1 + u),           u = 2/d
//   interior: G_I = u + log 4 - log(d^2 + 2d)
template <int MODE>
__device__ __forceinline__ double green64(double d2) {
  const double rinv = rsqrt(d2);
  const double u = 2.0 * rinv;
  if (MODE == 0) return u - log1p(u);
  const double d = d2 * rinv;
  return u + kLn4 - log(fma(2.0, d, d2));
}

// One FP32 pair from half-scaled offsets: every coordinate is multiplied by 1/2, so
// d2h = d^2 / 4 and rh = 1/sqrt(d2h) = 2/d = u. Then
//   exterior: G_E = u - log(1 + u)                                  = rh - log(1 + rh)
//   interior: G_I = u + log 4 - log(d^2 + 2d) = u - log((d^2 + 2d) / 4) = rh - log(d2h + d2h rh)
// Two MUFU operations (rsqrt, lg2) and four FP32 operations per pair besides the squared
// distance; returns acc + G rho.
template <int MODE>
__device__ __forceinline__ float pair32(float d2h, float rho, float acc) {
  const float rh = rsqrt_mufu(d2h);
  const float l = lg2_mufu(MODE == 0 ? 1.0f + rh : fmaf(d2h, rh, d2h));
  return fmaf(fmaf(l, -kLn2f, rh), rho, acc);
}

// log2(x) for normal x > 0 on the FMA and integer pipes instead of the MUFU unit:
// x = 2^e m with m in [sqrt(1/2), sqrt(2)), log2(x) = e + f P(f), f = m - 1, P of
// degree 8 fitted by least squares (coefficients from gen_log2_poly.py; absolute
// error <= 1e-7 for |log2 x| < 1, <= 3 ulp of the result elsewhere). The exponent is
// turned into a float by adding it to the bits of 1.5 * 2^23, so no conversion
// instruction is issued.
__device__ __forceinline__ float lg2_poly(float x) {
  const int i = __float_as_int(x);
  const int e = (i - 0x3f3504f3) >> 23;
  const float f = __int_as_float(i - (e << 23)) - 1.0f;
  float p = 1.224903390e-01f;
  p = fmaf(p, f, -2.088673115e-01f);
  p = fmaf(p, f, 2.178854942e-01f);
  p = fmaf(p, f, -2.387827337e-01f);
  p = fmaf(p, f, 2.876248062e-01f);
  p = fmaf(p, f, -3.607062101e-01f);
  p = fmaf(p, f, 4.809235036e-01f);
  p = fmaf(p, f, -7.213473916e-01f);
  p = fmaf(p, f, 1.442694902e+00f);
  const float ef = __int_as_float(e + 0x4b400000) - 12582912.0f;
  return fmaf(f, p, ef);
}

// pair32 with the logarithm taken by lg2_poly: the pair kernels may use it for a share
// of their pairs so that the MUFU unit and the FMA pipe are both kept busy.
template <int MODE>
__device__ __forceinline__ float pair32_poly(float d2h, float rho, float acc) {
  const float rh = rsqrt_mufu(d2h);
  const float l = lg2_poly(MODE == 0 ? 1.0f + rh : fmaf(d2h, rh, d2h));
  return fmaf(fmaf(l, -kLn2f, rh), rho, acc);
}

// Scalar pair loop (the dense direct kernel, and the tree kernels of NCS_PAIR_X2 = 0
// builds): NCS_PAIR_POLYLOG of every 16 FP32 pairs (0, 1 or 2) take their logarithm with
// lg2_poly on the FMA pipe instead of the MUFU unit, which otherwise bounds the pair
// rate (measured at N = 1e5: one in 16 shortens P2L by ~6 %, two in 16 by ~3 %).
#ifndef NCS_PAIR_POLYLOG
#define NCS_PAIR_POLYLOG 1
#endif

// part[t] += sum over the ns staged sources S (half-scaled offsets, strength in w) of
// G(a_t, s) rho_s for the NT half-scaled targets (ax, ay, az)[t]: sources in groups of
// 8, the last source of a group taking lg2_poly for its first NCS_PAIR_POLYLOG targets.
template <int MODE, int NT>
__device__ __forceinline__ void pair_loop32(const float4* __restrict__ S, int ns, const float* ax, const float* ay,
                                            const float* az, float* part) {
  int s = 0;
  if constexpr (NCS_PAIR_POLYLOG > 0) {
    for (; s + 8 <= ns; s += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4 v = S[s + u];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          const float dx = ax[t] - v.x, dy = ay[t] - v.y, dz = az[t] - v.z;
          const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          if (u == 7 && t < NCS_PAIR_POLYLOG)
            part[t] = pair32_poly<MODE>(d2, v.w, part[t]);
          else
            part[t] = pair32<MODE>(d2, v.w, part[t]);
        }
      }
    }
  }
  for (; s < ns; ++s) {
    const float4 v = S[s];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const float dx = ax[t] - v.x, dy = ay[t] - v.y, dz = az[t] - v.z;
      part[t] = pair32<MODE>(fmaf(dx, dx, fmaf(dy, dy, dz * dz)), v.w, part[t]);
    }
  }
}

// ---- packed pairs: sm_100+ f32x2 arithmetic -------------------------------------------
// add/sub/mul/fma .rn.f32x2 perform two IEEE single-precision operations (one per 32-bit
// half of a 64-bit register) in one instruction, each rounded exactly as the scalar
// instruction would round it. The packed pair loop below evaluates the same operation
// sequence as pair32 / pair32_poly for two sources at once, so a pair's value is unchanged
// and the issue slots of its FP32 arithmetic are halved; that leaves room on the FMA pipe
// for more logarithms by lg2_poly, the MUFU unit being the other bound.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 x2_pack(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void x2_unpack(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 x2_add(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 x2_sub(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 x2_mul(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 x2_fma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// The packed constants of a pair loop, formed once per call.
struct PairX2Consts {
  f32x2 one, nln2, bias, mhalf, three_halves, c[9];
  __device__ __forceinline__ PairX2Consts() {
    one = x2_pack(1.0f, 1.0f);
    mhalf = x2_pack(-0.5f, -0.5f);
    three_halves = x2_pack(1.5f, 1.5f);
    nln2 = x2_pack(-kLn2f, -kLn2f);
    bias = x2_pack(12582912.0f, 12582912.0f);
    const float cf[9] = {1.224903390e-01f,  -2.088673115e-01f, 2.178854942e-01f,
                         -2.387827337e-01f, 2.876248062e-01f,  -3.607062101e-01f,
                         4.809235036e-01f,  -7.213473916e-01f, 1.442694902e+00f};
#pragma unroll
    for (int k = 0; k < 9; ++k) c[k] = x2_pack(cf[k], cf[k]);
  }
};

// lg2_poly on both halves: the same operations, the integer steps per half.
__device__ __forceinline__ f32x2 lg2_poly_x2(f32x2 x, const PairX2Consts& k) {
  float x0, x1;
  x2_unpack(x, x0, x1);
  const int i0 = __float_as_int(x0), i1 = __float_as_int(x1);
  const int e0 = (i0 - 0x3f3504f3) >> 23, e1 = (i1 - 0x3f3504f3) >> 23;
  const f32x2 f = x2_sub(x2_pack(__int_as_float(i0 - (e0 << 23)), __int_as_float(i1 - (e1 << 23))), k.one);
  f32x2 p = k.c[0];
#pragma unroll
  for (int j = 1; j < 9; ++j) p = x2_fma(p, f, k.c[j]);
  const f32x2 ef = x2_sub(x2_pack(__int_as_float(e0 + 0x4b400000), __int_as_float(e1 + 0x4b400000)), k.bias);
  return x2_fma(f, p, ef);
}

// 1/sqrt(x) for normal x > 0 on the FMA and integer pipes instead of the MUFU unit, both
// halves: the seed of Lomont's "Fast Inverse Square Root" (2003), the bits 0x5f375a86 minus
// half the bits of x (relative error ~3.4e-2), then two Newton steps
// y <- y (3/2 - (x/2) y^2), each squaring the relative error (1.75e-3, then 4.7e-6): 7 FP32
// operations and two integer ones per value. Used for a tuned share of the FP32 pairs only,
// whose products the tuner checks against the float-float product.
__device__ __forceinline__ f32x2 rsqrt_newton_x2(f32x2 x, const PairX2Consts& k) {
  float x0, x1;
  x2_unpack(x, x0, x1);
  f32x2 y = x2_pack(__int_as_float(0x5f375a86 - (__float_as_int(x0) >> 1)),
                    __int_as_float(0x5f375a86 - (__float_as_int(x1) >> 1)));
  const f32x2 nhx = x2_mul(k.mhalf, x);
  y = x2_mul(y, x2_fma(x2_mul(nhx, y), y, k.three_halves));
  y = x2_mul(y, x2_fma(x2_mul(nhx, y), y, k.three_halves));
  return y;
}

// Two pairs (one target, the two sources of a staged pair) into the packed accumulator.
// (X, Y) = (x pair, y pair), (Z, W) = (z pair, strength pair) of the sources. POLY: the
// logarithm by lg2_poly on the FMA pipe; RSQ: the reciprocal square root by
// rsqrt_newton_x2 (else both on the MUFU unit).
template <int MODE, bool POLY, bool RSQ = false>
__device__ __forceinline__ f32x2 pair32_x2(f32x2 ax, f32x2 ay, f32x2 az, const ulonglong2& XY,
                                           const ulonglong2& ZW, f32x2 acc, const PairX2Consts& k) {
  const f32x2 dx = x2_sub(ax, XY.x), dy = x2_sub(ay, XY.y), dz = x2_sub(az, ZW.x);
  const f32x2 d2 = x2_fma(dx, dx, x2_fma(dy, dy, x2_mul(dz, dz)));
  f32x2 rh;
  if constexpr (RSQ) {
    rh = rsqrt_newton_x2(d2, k);
  } else {
    float d0, d1;
    x2_unpack(d2, d0, d1);
    rh = x2_pack(rsqrt_mufu(d0), rsqrt_mufu(d1));
  }
  const f32x2 arg = (MODE == 0) ? x2_add(k.one, rh) : x2_fma(d2, rh, d2);
  f32x2 l;
  if constexpr (POLY) {
    l = lg2_poly_x2(arg, k);
  } else {
    float g0, g1;
    x2_unpack(arg, g0, g1);
    l = x2_pack(lg2_mufu(g0), lg2_mufu(g1));
  }
  return x2_fma(x2_fma(l, k.nln2, rh), ZW.y, acc);
}

// Staged sources in the paired layout of pair_loop32x2: sources 2k and 2k+1 share the 32
// bytes S[2k], S[2k+1] = (x0, x1, y0, y1), (z0, z1, w0, w1).
__device__ __forceinline__ void stage_source_x2(float4* S, int idx, float x, float y, float z, float w) {
  float* f = reinterpret_cast<float*>(S) + 8 * (idx >> 1) + (idx & 1);
  f[0] = x;
  f[2] = y;
  f[4] = z;
  f[6] = w;
}
// An odd source count is padded with a zero-strength source far from every target
// (half-scaled offsets have norm below 1.1; this one sits at distance > 2 from them).
__device__ __forceinline__ void stage_pad_x2(float4* S, int ns) {
  if (ns & 1) stage_source_x2(S, ns, 2.0f, 2.0f, 2.0f, 0.0f);
}

// NCS_PAIR_X2_POLY of every 16 two-pair chains (a target against a staged source pair)
// take their logarithms with lg2_poly.
#ifndef NCS_PAIR_X2_POLY
#define NCS_PAIR_X2_POLY 4
#endif

// part[t] = sum over the ns staged sources (paired layout, padded to even) of G(a_t, s)
// rho_s for the NT half-scaled targets: source pairs in groups of 8, the first POLY16
// of every 16 two-pair chains (scaled to a group's 8 NT chains) on lg2_poly and the last
// RSQ16 with the Newton reciprocal square root. Both are run-time choices of the kernels'
// launch configuration (set by ncs_tune), with NCS_PAIR_X2_POLY and 0 as the defaults.
template <int MODE, int NT, int POLY16 = NCS_PAIR_X2_POLY, int RSQ16 = 0>
__device__ __forceinline__ void pair_loop32x2(const float4* __restrict__ S, int ns, const float* ax, const float* ay,
                                              const float* az, float* part) {
  const PairX2Consts k;
  const ulonglong2* S2 = reinterpret_cast<const ulonglong2*>(S);
  f32x2 AX[NT], AY[NT], AZ[NT], P[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    AX[t] = x2_pack(ax[t], ax[t]);
    AY[t] = x2_pack(ay[t], ay[t]);
    AZ[t] = x2_pack(az[t], az[t]);
    P[t] = x2_pack(0.0f, 0.0f);
  }
  constexpr int kPoly = POLY16 * NT / 2;  // poly chains per group of 8 * NT
  constexpr int kRsq = RSQ16 * NT / 2;    // Newton rsqrt chains (the last ones of a group)
  static_assert(kPoly + kRsq <= 8 * NT, "polynomial and Newton shares overlap");
  const int np = (ns + 1) >> 1;
  int s = 0;
  for (; s + 8 <= np; s += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const ulonglong2 XY = S2[2 * (s + u)], ZW = S2[2 * (s + u) + 1];
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        if (u * NT + t < kPoly)
          P[t] = pair32_x2<MODE, true>(AX[t], AY[t], AZ[t], XY, ZW, P[t], k);
        else if (u * NT + t >= 8 * NT - kRsq)
          P[t] = pair32_x2<MODE, false, true>(AX[t], AY[t], AZ[t], XY, ZW, P[t], k);
        else
          P[t] = pair32_x2<MODE, false>(AX[t], AY[t], AZ[t], XY, ZW, P[t], k);
      }
    }
  }
  for (; s < np; ++s) {
    const ulonglong2 XY = S2[2 * s], ZW = S2[2 * s + 1];
#pragma unroll
    for (int t = 0; t < NT; ++t) P[t] = pair32_x2<MODE, false>(AX[t], AY[t], AZ[t], XY, ZW, P[t], k);
  }
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    float lo, hi;
    x2_unpack(P[t], lo, hi);
    part[t] = lo + hi;
  }
}

// 1: the tree's FP32 pair kernels stage sources in the paired layout and run
// pair_loop32x2; 0: float4 staging and pair_loop32.
#ifndef NCS_PAIR_X2
#define NCS_PAIR_X2 1
#endif

}  // namespace ncs
