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

// NCS_PAIR_POLYLOG of every 16 FP32 pairs (0, 1 or 2) take their logarithm with
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

}  // namespace ncs
