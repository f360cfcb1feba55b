// Hot-path kernels of the direct (no tree) matrix-vector product of Kaye & Greengard,
// Section 6 eq. (opinteqnsdisc) with the compressed outgoing representation of
// Section 7.1:
//   rho_j = T f_j                                      (eq. Tmap, Step 3.1)
//   z_i(k) = sum_{j != i} sum_m G(x^z_{i,k}, x_{j,pi(m)}) rho_{j,m}   (Section 7.1)
//   y_i = f_i + P z_i                                  (Step 3.5)
// and the single-layer potential at off-surface targets (Section 2, eqs. urep,
// intBVPansatz with eqs. Gextoffsurface / Gintoffsurface).
#include <cstdint>

#include "device_common.cuh"
#include "df64.cuh"
#include "internal.hpp"

namespace ncs {

template <typename R>
struct Vec4;
template <>
struct Vec4<float> {
  using type = float4;
};
template <>
struct Vec4<double> {
  using type = double4_16a;
};

// ---------------------------------------------------------------------------
// Skeleton offsets s_{j,m} - c_j in the global frame (FP64 and an FP32 copy).
__global__ void skeleton_offsets_kernel(int64_t N, int p, const double* __restrict__ centres,
                                        const double* __restrict__ sloc, double* __restrict__ soff64,
                                        float* __restrict__ soff32) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * p) return;
  const int64_t j = idx / p;
  const int m = (int)(idx % p);
  const double cx = centres[3 * j], cy = centres[3 * j + 1], cz = centres[3 * j + 2];
  double e1[3], e2[3], g[3];
  patch_frame(cx, cy, cz, e1, e2);
  frame_apply(e1, e2, cx, cy, cz, sloc[3 * m], sloc[3 * m + 1], sloc[3 * m + 2], g);
  for (int c = 0; c < 3; ++c) {
    soff64[3 * idx + c] = g[c];
    soff32[3 * idx + c] = (float)g[c];
  }
}

cudaError_t launch_skeleton_offsets(const DeviceData& d, cudaStream_t s) {
  const int64_t n = d.N * d.p;
  const int th = 256;
  count_launch(), skeleton_offsets_kernel<<<(unsigned)((n + th - 1) / th), th, 0, s>>>(d.N, d.p, d.centres, d.sloc,
                                                                       d.soff64, d.soff32);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Step 3.1: rho_i = T f_i for OG_PB patches per block; TT is T transposed (K x p), and
// each thread accumulates 4 consecutive skeleton rows for all OG_PB patches, so one
// coalesced row read of TT and OG_PB shared-memory broadcasts feed 4 * OG_PB FMAs.
constexpr int OG_PB = 8;

template <typename R>
__global__ void __launch_bounds__(128) outgoing_kernel(int64_t N, int p, int K, const R* __restrict__ TT,
                                                       const double* __restrict__ x, R* __restrict__ rho) {
  extern __shared__ unsigned char og_smem[];
  R* xs = reinterpret_cast<R*>(og_smem);  // OG_PB x K
  const int64_t i0 = (int64_t)blockIdx.x * OG_PB;
  const int np = (int)min((int64_t)OG_PB, N - i0);
  for (int idx = threadIdx.x; idx < OG_PB * K; idx += blockDim.x)
    xs[idx] = (idx < np * K) ? (R)x[i0 * K + idx] : (R)0;
  __syncthreads();
  for (int m0 = 4 * threadIdx.x; m0 < p; m0 += 4 * blockDim.x) {
    R acc[OG_PB][4];
#pragma unroll
    for (int ii = 0; ii < OG_PB; ++ii)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[ii][j] = 0;
    for (int k = 0; k < K; ++k) {
      const R* row = TT + (int64_t)k * p + m0;
      R t[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) t[j] = (m0 + j < p) ? row[j] : (R)0;
#pragma unroll
      for (int ii = 0; ii < OG_PB; ++ii) {
        const R xv = xs[ii * K + k];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[ii][j] = fma(t[j], xv, acc[ii][j]);
      }
    }
#pragma unroll
    for (int ii = 0; ii < OG_PB; ++ii)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (ii < np && m0 + j < p) rho[(i0 + ii) * p + m0 + j] = acc[ii][j];
  }
}

cudaError_t launch_outgoing(const DeviceData& d, const double* x, int prec, cudaStream_t s) {
  const unsigned blocks = (unsigned)((d.N + OG_PB - 1) / OG_PB);
  if (prec == NCS_FP64 || prec == NCS_DF64)
    count_launch(), outgoing_kernel<double><<<blocks, 128, OG_PB * d.K * sizeof(double), s>>>(d.N, d.p, d.K, d.TT64, x,
                                                                                d.rho64);
  else
    count_launch(), outgoing_kernel<float><<<blocks, 128, OG_PB * d.K * sizeof(float), s>>>(d.N, d.p, d.K, d.TT32, x,
                                                                              d.rho32);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Direct far-field sums at the Zernike nodes (Section 7.1, without the tree).
// One block row per target patch i; each thread owns DF_NT target nodes. Source
// patches are staged JT at a time in shared memory as (offset from c_i, rho)
// quadruples. Each source patch j uses the coarsest outgoing representation valid at
// its distance (far-field radius <= geodesic(c_i, c_j) - eps, the farthest a node of
// patch i can be from c_i); the self patch is skipped. Offsets are formed in FP64
// (c_j - c_i) before rounding, so the FP32 path keeps relative accuracy even for
// neighbours 3 eps apart. FP32 partial sums are folded into an FP64 accumulator once
// per tile.
constexpr int DF_THREADS = 256;
constexpr int DF_NT = 2;
constexpr int DF_JTMAX = 8;

__device__ __forceinline__ int select_rep(double dist, int nrep, const double* __restrict__ rep_rho) {
  int k = 0;
  while (k + 1 < nrep && rep_rho[k + 1] <= dist) ++k;
  return k;
}

template <typename R, int MODE>
__global__ void __launch_bounds__(DF_THREADS) direct_field_kernel(
    int64_t N, int pt, int Kstar, int JT, int pmax, int nrep, const int* __restrict__ rep_p,
    const int* __restrict__ rep_off, const double* __restrict__ rep_rho, double eps, const double* __restrict__ centres,
    const double* __restrict__ zloc, const R* __restrict__ soff, const R* __restrict__ rho,
    double* __restrict__ z) {
  using V4 = typename Vec4<R>::type;
  extern __shared__ unsigned char df_smem[];
  V4* S = reinterpret_cast<V4*>(df_smem);  // JT * pmax
  __shared__ double D[DF_JTMAX][3];
  __shared__ int toff[DF_JTMAX + 1], tcol[DF_JTMAX];
  const int64_t i = blockIdx.x;
  const double cx = centres[3 * i], cy = centres[3 * i + 1], cz = centres[3 * i + 2];
  double e1[3], e2[3];
  patch_frame(cx, cy, cz, e1, e2);
  R ax[DF_NT], ay[DF_NT], az[DF_NT];
  double acc[DF_NT];
  int kk[DF_NT];
#pragma unroll
  for (int t = 0; t < DF_NT; ++t) {
    kk[t] = (blockIdx.y * DF_NT + t) * DF_THREADS + threadIdx.x;
    double g[3] = {0.0, 0.0, 0.0};
    if (kk[t] < Kstar) frame_apply(e1, e2, cx, cy, cz, zloc[3 * kk[t]], zloc[3 * kk[t] + 1], zloc[3 * kk[t] + 2], g);
    const double sc = (sizeof(R) == 4) ? 0.5 : 1.0;  // FP32: half-scaled offsets
    ax[t] = (R)(sc * g[0]);
    ay[t] = (R)(sc * g[1]);
    az[t] = (R)(sc * g[2]);
    acc[t] = 0.0;
  }
  for (int64_t j0 = 0; j0 < N; j0 += JT) {
    const int nj = (int)min((int64_t)JT, N - j0);
    __syncthreads();
    if (threadIdx.x < nj) {
      const int64_t j = j0 + threadIdx.x;
      double d0 = centres[3 * j] - cx, d1 = centres[3 * j + 1] - cy, d2 = centres[3 * j + 2] - cz;
      D[threadIdx.x][0] = d0;
      D[threadIdx.x][1] = d1;
      D[threadIdx.x][2] = d2;
      int cnt = 0, col = 0;
      if (j != i) {
        const double dist = 2.0 * asin(fmin(1.0, 0.5 * sqrt(d0 * d0 + d1 * d1 + d2 * d2)));
        const int k = select_rep(dist - eps, nrep, rep_rho);
        cnt = rep_p[k];
        col = rep_off[k];
      }
      toff[threadIdx.x + 1] = cnt;
      tcol[threadIdx.x] = col;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      toff[0] = 0;
      for (int jj = 0; jj < nj; ++jj) toff[jj + 1] += toff[jj];
    }
    __syncthreads();
    const int ns = toff[nj];
    for (int idx = threadIdx.x; idx < ns; idx += DF_THREADS) {
      int jj = 0;
      while (idx >= toff[jj + 1]) ++jj;
      const int64_t g = (j0 + jj) * pt + tcol[jj] + (idx - toff[jj]);
      V4 v;
      v.x = (R)D[jj][0] + soff[3 * g];
      v.y = (R)D[jj][1] + soff[3 * g + 1];
      v.z = (R)D[jj][2] + soff[3 * g + 2];
      v.w = rho[g];
      if constexpr (sizeof(R) == 4) {  // the FP32 pairs take half-scaled offsets
        v.x *= 0.5f;
        v.y *= 0.5f;
        v.z *= 0.5f;
      }
      S[idx] = v;
    }
    __syncthreads();
    R part[DF_NT];
#pragma unroll
    for (int t = 0; t < DF_NT; ++t) part[t] = 0;
    if constexpr (sizeof(R) == 4) {
      pair_loop32<MODE, DF_NT>(S, ns, ax, ay, az, part);
    } else {
      for (int s = 0; s < ns; ++s) {
        const V4 v = S[s];
#pragma unroll
        for (int t = 0; t < DF_NT; ++t) {
          const R dx = ax[t] - v.x, dy = ay[t] - v.y, dz = az[t] - v.z;
          part[t] = fma(green64<MODE>(fma(dx, dx, fma(dy, dy, dz * dz))), v.w, part[t]);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < DF_NT; ++t) acc[t] += (double)part[t];
  }
#pragma unroll
  for (int t = 0; t < DF_NT; ++t)
    if (kk[t] < Kstar) z[i * Kstar + kk[t]] = acc[t];
}

// Float-float variant (FP64-accurate on the FP32 pipes); sources staged as (hi, lo).
template <int MODE>
__global__ void __launch_bounds__(DF_THREADS) direct_field_df_kernel(
    int64_t N, int pt, int Kstar, int JT, int pmax, int nrep, const int* __restrict__ rep_p,
    const int* __restrict__ rep_off, const double* __restrict__ rep_rho, double eps,
    const double* __restrict__ centres, const double* __restrict__ zloc, const double* __restrict__ soff,
    const double* __restrict__ rho, const float4* __restrict__ logtab, double* __restrict__ z) {
  extern __shared__ float4 dfd_smem[];
  __shared__ float4 tab[kLogTable];
  __shared__ double D[DF_JTMAX][3];
  __shared__ int toff[DF_JTMAX + 1], tcol[DF_JTMAX];
  float4* Sh = dfd_smem;
  float4* Sl = dfd_smem + JT * pmax;
  for (int t = threadIdx.x; t < kLogTable; t += blockDim.x) tab[t] = logtab[t];
  const int64_t i = blockIdx.x;
  const double cx = centres[3 * i], cy = centres[3 * i + 1], cz = centres[3 * i + 2];
  double e1[3], e2[3];
  patch_frame(cx, cy, cz, e1, e2);
  f2 a[DF_NT][3];
  double acc[DF_NT];
  int kk[DF_NT];
#pragma unroll
  for (int t = 0; t < DF_NT; ++t) {
    kk[t] = (blockIdx.y * DF_NT + t) * DF_THREADS + threadIdx.x;
    double g[3] = {0.0, 0.0, 0.0};
    if (kk[t] < Kstar) frame_apply(e1, e2, cx, cy, cz, zloc[3 * kk[t]], zloc[3 * kk[t] + 1], zloc[3 * kk[t] + 2], g);
    for (int c = 0; c < 3; ++c) a[t][c] = f2_from_double(g[c]);
    acc[t] = 0.0;
  }
  for (int64_t j0 = 0; j0 < N; j0 += JT) {
    const int nj = (int)min((int64_t)JT, N - j0);
    __syncthreads();
    if (threadIdx.x < nj) {
      const int64_t j = j0 + threadIdx.x;
      const double d0 = centres[3 * j] - cx, d1 = centres[3 * j + 1] - cy, d2 = centres[3 * j + 2] - cz;
      D[threadIdx.x][0] = d0;
      D[threadIdx.x][1] = d1;
      D[threadIdx.x][2] = d2;
      int cnt = 0, col = 0;
      if (j != i) {
        const double dist = 2.0 * asin(fmin(1.0, 0.5 * sqrt(d0 * d0 + d1 * d1 + d2 * d2)));
        const int k = select_rep(dist - eps, nrep, rep_rho);
        cnt = rep_p[k];
        col = rep_off[k];
      }
      toff[threadIdx.x + 1] = cnt;
      tcol[threadIdx.x] = col;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      toff[0] = 0;
      for (int jj = 0; jj < nj; ++jj) toff[jj + 1] += toff[jj];
    }
    __syncthreads();
    const int ns = toff[nj];
    for (int idx = threadIdx.x; idx < ns; idx += DF_THREADS) {
      int jj = 0;
      while (idx >= toff[jj + 1]) ++jj;
      const int64_t g = (j0 + jj) * pt + tcol[jj] + (idx - toff[jj]);
      const f2 x = f2_from_double(D[jj][0] + soff[3 * g]), y = f2_from_double(D[jj][1] + soff[3 * g + 1]),
               zz = f2_from_double(D[jj][2] + soff[3 * g + 2]), r = f2_from_double(rho[g]);
      Sh[idx] = make_float4(x.hi, y.hi, zz.hi, r.hi);
      Sl[idx] = make_float4(x.lo, y.lo, zz.lo, r.lo);
    }
    __syncthreads();
    f2 part[DF_NT];
#pragma unroll
    for (int t = 0; t < DF_NT; ++t) part[t] = f2{0.0f, 0.0f};
    if constexpr (DF_NT == 2) {  // both targets in one packed float-float chain
      f2x2 A[3], P{x2_splat(0.0f), x2_splat(0.0f)};
#pragma unroll
      for (int c = 0; c < 3; ++c) A[c] = f2x2{x2_pack(a[0][c].hi, a[1][c].hi), x2_pack(a[0][c].lo, a[1][c].lo)};
      for (int s = 0; s < ns; ++s) pair_f2_acc_x2<MODE>(A, Sh[s], Sl[s], tab, P);
      x2_unpack(P.hi, part[0].hi, part[1].hi);
      x2_unpack(P.lo, part[0].lo, part[1].lo);
    } else {
      for (int s = 0; s < ns; ++s) {
        const float4 h = Sh[s], l = Sl[s];
#pragma unroll
        for (int t = 0; t < DF_NT; ++t) pair_f2_acc<MODE>(a[t], h, l, tab, part[t]);
      }
    }
#pragma unroll
    for (int t = 0; t < DF_NT; ++t) acc[t] += f2_to_double(part[t]);
  }
#pragma unroll
  for (int t = 0; t < DF_NT; ++t)
    if (kk[t] < Kstar) z[i * Kstar + kk[t]] = acc[t];
}

template <typename K>
static cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_direct_field(const DeviceData& d, int mode, int prec, double eps, cudaStream_t s) {
  if (prec == NCS_DF64) {
    int JT = (int)std::min<size_t>(DF_JTMAX, (40 * 1024) / (2 * sizeof(float4) * (size_t)d.pmax));
    if (JT < 1) JT = 1;
    const size_t smem = (size_t)2 * JT * d.pmax * sizeof(float4);
    dim3 grid((unsigned)d.N, (unsigned)((d.Kstar + DF_THREADS * DF_NT - 1) / (DF_THREADS * DF_NT)));
    cudaError_t e;
    if (mode == 0) {
      if ((e = allow_smem(direct_field_df_kernel<0>, smem)) != cudaSuccess) return e;
      count_launch(), direct_field_df_kernel<0><<<grid, DF_THREADS, smem, s>>>(d.N, d.p, d.Kstar, JT, d.pmax, d.nrep, d.rep_p,
                                                               d.rep_off, d.rep_rho, eps, d.centres, d.zloc,
                                                               d.soff64, d.rho64, d.logtab, d.z);
    } else {
      if ((e = allow_smem(direct_field_df_kernel<1>, smem)) != cudaSuccess) return e;
      count_launch(), direct_field_df_kernel<1><<<grid, DF_THREADS, smem, s>>>(d.N, d.p, d.Kstar, JT, d.pmax, d.nrep, d.rep_p,
                                                               d.rep_off, d.rep_rho, eps, d.centres, d.zloc,
                                                               d.soff64, d.rho64, d.logtab, d.z);
    }
    return cudaGetLastError();
  }
  const size_t v4 = (prec == NCS_FP64) ? sizeof(double4_16a) : sizeof(float4);
  int JT = (int)std::min<size_t>(DF_JTMAX, (40 * 1024) / (v4 * (size_t)d.pmax));
  if (JT < 1) JT = 1;
  const size_t smem = (size_t)JT * d.pmax * v4;
  dim3 grid((unsigned)d.N, (unsigned)((d.Kstar + DF_THREADS * DF_NT - 1) / (DF_THREADS * DF_NT)));
  cudaError_t e;
#define NCS_DF(R, M, SOFF, RHO)                                                                            \
  do {                                                                                                     \
    if ((e = allow_smem(direct_field_kernel<R, M>, smem)) != cudaSuccess) return e;                       \
    count_launch(), direct_field_kernel<R, M><<<grid, DF_THREADS, smem, s>>>(d.N, d.p, d.Kstar, JT, d.pmax, d.nrep, d.rep_p, \
                                                             d.rep_off, d.rep_rho, eps, d.centres, d.zloc, \
                                                             SOFF, RHO, d.z);                              \
  } while (0)
  if (prec == NCS_FP64) {
    if (mode == 0)
      NCS_DF(double, 0, d.soff64, d.rho64);
    else
      NCS_DF(double, 1, d.soff64, d.rho64);
  } else {
    if (mode == 0)
      NCS_DF(float, 0, d.soff32, d.rho32);
    else
      NCS_DF(float, 1, d.soff32, d.rho32);
  }
#undef NCS_DF
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Step 3.5: y_i = x_i + P z_i. PT is P transposed (Kstar x K).
// A block takes BP patches; their z rows are staged transposed in shared memory
// (zT[q][i], row stride BP + 1 so that the staging stores spread over the banks), and
// each thread accumulates a 4-patch x 4-output register tile over all Kstar nodes: per
// node four shared loads of z and four loads of PT (L1/L2 resident, 270 KB in FP32)
// feed 16 FMAs.
constexpr int AP_THREADS = 288;

template <typename R, int BP>
__global__ void __launch_bounds__(AP_THREADS) apply_P_kernel(int64_t N, int K, int Kstar, const R* __restrict__ PT,
                                                             const double* __restrict__ z,
                                                             const double* __restrict__ x, double* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char ap_smem[];
  constexpr int SB = BP + 1;
  R* zT = reinterpret_cast<R*>(ap_smem);  // Kstar x SB
  const int64_t i0 = (int64_t)blockIdx.x * BP;
  const int np = (int)min((int64_t)BP, N - i0);
  for (int idx = threadIdx.x; idx < BP * Kstar; idx += blockDim.x) {
    const int ii = idx / Kstar, q = idx - ii * Kstar;
    zT[q * SB + ii] = (ii < np) ? (R)z[(i0 + ii) * Kstar + q] : (R)0;
  }
  __syncthreads();
  const int nJ = (K + 3) / 4, nW = nJ * (BP / 4);
  for (int w = threadIdx.x; w < nW; w += blockDim.x) {
    const int j0 = 4 * (w % nJ), a0 = 4 * (w / nJ);
    R acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c] = 0;
    for (int q = 0; q < Kstar; ++q) {
      const R* pr = PT + (int64_t)q * K + j0;
      R pv[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) pv[c] = (j0 + c < K) ? __ldg(pr + c) : (R)0;
      const R* zr = zT + q * SB + a0;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const R zv = zr[a];
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = fma(pv[c], zv, acc[a][c]);
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (a0 + a < np && j0 + c < K) {
          const int64_t o = (i0 + a0 + a) * K + j0 + c;
          y[o] = x[o] + (double)acc[a][c];
        }
  }
}

// prec: NCS_FP32 runs the transform in FP32 (the FP32 product), otherwise FP64.
cudaError_t launch_apply_P(const DeviceData& d, const double* x, double* y, int prec, cudaStream_t s) {
  if (prec == NCS_FP32) {
    constexpr int BP = 32;
    const size_t smem = (size_t)(BP + 1) * d.Kstar * sizeof(float);
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(apply_P_kernel<float, BP>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    const unsigned blocks = (unsigned)((d.N + BP - 1) / BP);
    count_launch(), apply_P_kernel<float, BP><<<blocks, AP_THREADS, smem, s>>>(d.N, d.K, d.Kstar, d.PT32, d.z, x, y);
  } else {
    constexpr int BP = 16;
    const size_t smem = (size_t)(BP + 1) * d.Kstar * sizeof(double);
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(apply_P_kernel<double, BP>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    const unsigned blocks = (unsigned)((d.N + BP - 1) / BP);
    count_launch(), apply_P_kernel<double, BP><<<blocks, AP_THREADS, smem, s>>>(d.N, d.K, d.Kstar, d.PT64, d.z, x, y);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Off-surface single-layer potential u(x) = sum_j sum_m G(x, s_jm) rho_jm, FP64,
// one block per target with a block reduction.
template <int MODE>
__global__ void __launch_bounds__(256) eval_kernel(int64_t N, int p, int pt, const double* __restrict__ centres,
                                                   const double* __restrict__ soff, const double* __restrict__ rho,
                                                   const double* __restrict__ targets, int64_t skip,
                                                   const int64_t* __restrict__ skip_off,
                                                   const int* __restrict__ skip_idx, double* __restrict__ out) {
  __shared__ double red[256];
  const int64_t t = blockIdx.x;
  const double x0 = targets[3 * t], x1 = targets[3 * t + 1], x2 = targets[3 * t + 2];
  const double rx = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
  // patches left out for this target: those evaluated by the near-patch quadrature
  const int64_t s0 = skip_off ? skip_off[t] : 0, s1 = skip_off ? skip_off[t + 1] : 0;
  double acc = 0.0;
  for (int64_t h = threadIdx.x; h < N * p; h += blockDim.x) {
    const int64_t j = h / p;
    if (j == skip) continue;                 // a patch left out (its own points as targets)
    bool near = false;
    for (int64_t q = s0; q < s1; ++q) near |= (skip_idx[q] == j);
    if (near) continue;
    const int64_t g = j * pt + (h - j * p);  // representation 0 (the finest) of patch j
    const double s0 = centres[3 * j] + soff[3 * g], s1 = centres[3 * j + 1] + soff[3 * g + 1],
                 s2 = centres[3 * j + 2] + soff[3 * g + 2];
    const double d0 = x0 - s0, d1 = x1 - s1, d2 = x2 - s2;
    const double d = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    const double xx = x0 * s0 + x1 * s1 + x2 * s2;
    double gval;
    if (MODE == 0)
      gval = 2.0 / d + log((rx - xx) / (1.0 - xx + d));  // eq. (Gextoffsurface)
    else
      gval = 2.0 / d + log(2.0 / (1.0 - xx + d));  // eq. (Gintoffsurface)
    acc = fma(gval, rho[g], acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[t] = red[0];
}

cudaError_t launch_eval(const DeviceData& d, int mode, int64_t M, const double* targets, double* out,
                        cudaStream_t s, int64_t skip) {
  if (M == 0) return cudaSuccess;
  if (mode == 0)
    count_launch(), eval_kernel<0><<<(unsigned)M, 256, 0, s>>>(d.N, d.p0, d.p, d.centres, d.soff64, d.rho64, targets,
                                                               skip, nullptr, nullptr, out);
  else
    count_launch(), eval_kernel<1><<<(unsigned)M, 256, 0, s>>>(d.N, d.p0, d.p, d.centres, d.soff64, d.rho64, targets,
                                                               skip, nullptr, nullptr, out);
  return cudaGetLastError();
}

cudaError_t launch_eval_skip(const DeviceData& d, int mode, int64_t M, const double* targets, double* out,
                             const int64_t* skip_off, const int* skip_idx, cudaStream_t s) {
  if (M == 0) return cudaSuccess;
  if (mode == 0)
    count_launch(), eval_kernel<0><<<(unsigned)M, 256, 0, s>>>(d.N, d.p0, d.p, d.centres, d.soff64, d.rho64, targets,
                                                               -1, skip_off, skip_idx, out);
  else
    count_launch(), eval_kernel<1><<<(unsigned)M, 256, 0, s>>>(d.N, d.p0, d.p, d.centres, d.soff64, d.rho64, targets,
                                                               -1, skip_off, skip_idx, out);
  return cudaGetLastError();
}

}  // namespace ncs
