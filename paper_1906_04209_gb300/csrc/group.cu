// Grouped solve of many small spheres (Section 7, Step 3, for a batch of independent
// instances of eq. opinteqnsdisc): every sphere of a group shares K (and with it the
// Zernike transform P) and the problem mode; each keeps its own eps, layout, outgoing
// operator (T, skeletons, ID ladder), I and GMRES state. One launch per product stage and
// per Krylov step serves every instance of the group:
//   * group_outgoing_kernel: rho_j = T_b x_j, one block per patch, T_b of its instance;
//   * group_direct_kernel / group_direct_df_kernel: the direct compressed sums of Section
//     7.1 at every patch's Zernike nodes over the other patches of its own instance;
//   * the Zernike transform y = x + P z over all patches at once (P is common);
//   * segmented GMRES: projections, updates, norms, Givens rotations and back substitution
//     per instance (its segment of every vector), steps skipped once an instance is done.
// The layout (patch-major over the concatenated instances): patch i of the group belongs
// to instance pinst[i]; its outgoing coefficients start at roff[i] (the instances' skeleton
// counts differ); instance b owns patches [pbase[b], pbase[b + 1]).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "device_common.cuh"
#include "df64.cuh"
#include "internal.hpp"

namespace ncs {

namespace {

constexpr int GO_THREADS = 128;
constexpr int GD_THREADS = 256;
constexpr int GD_NT = 2;
constexpr int GD_JT = 8;

__device__ __forceinline__ int group_rep(double dist, int nrep, const double* __restrict__ rho_min) {
  int k = 0;
  while (k + 1 < nrep && rho_min[k + 1] <= dist) ++k;
  return k;
}

template <typename R>
__global__ void __launch_bounds__(GO_THREADS) group_outgoing_kernel(GroupDev g, const double* __restrict__ x) {
  const int64_t i = blockIdx.x;
  const int b = g.pinst[i];
  const int pt = g.inst_ptot[b], K = g.K;
  const R* TT = (sizeof(R) == 8 ? (const R*)g.TT64 : (const R*)g.TT32) + g.tt_off[b];  // K x pt
  R* rho = (sizeof(R) == 8 ? (R*)g.rho64 : (R*)g.rho32) + g.roff[i];
  extern __shared__ unsigned char go_smem[];
  R* xs = reinterpret_cast<R*>(go_smem);
  for (int k = threadIdx.x; k < K; k += blockDim.x) xs[k] = (R)x[i * K + k];
  __syncthreads();
  for (int m = threadIdx.x; m < pt; m += blockDim.x) {
    R acc = 0;
    for (int k = 0; k < K; ++k) acc = fma(TT[(int64_t)k * pt + m], xs[k], acc);
    rho[m] = acc;
  }
}

// The direct compressed sums at the Zernike nodes of patch i over the other patches of its
// instance (FP32 or FP64 pairs; offsets formed in FP64 from c_j - c_i before rounding; each
// source patch at the coarsest representation valid at its distance).
template <typename R, int MODE>
__global__ void __launch_bounds__(GD_THREADS) group_direct_kernel(GroupDev g, int JT) {
  using V4 = typename std::conditional<sizeof(R) == 4, float4, double4_16a>::type;
  extern __shared__ unsigned char gd_smem[];
  V4* S = reinterpret_cast<V4*>(gd_smem);  // JT * pmax
  __shared__ double D[GD_JT][3];
  __shared__ int toff[GD_JT + 1], tcol[GD_JT];
  const int64_t i = blockIdx.x;
  const int b = g.pinst[i];
  const int Kstar = g.Kstar;
  const double eps = g.inst_eps[b];
  const int nrep = g.inst_nrep[b], rb = g.inst_repbase[b];
  const double* zloc = g.zloc + (int64_t)3 * Kstar * b;
  const R* soff = sizeof(R) == 8 ? (const R*)g.soff64 : (const R*)g.soff32;
  const R* rho = sizeof(R) == 8 ? (const R*)g.rho64 : (const R*)g.rho32;
  const double cx = g.centres[3 * i], cy = g.centres[3 * i + 1], cz = g.centres[3 * i + 2];
  double e1[3], e2[3];
  patch_frame(cx, cy, cz, e1, e2);
  R ax[GD_NT], ay[GD_NT], az[GD_NT];
  double acc[GD_NT];
  int kk[GD_NT];
#pragma unroll
  for (int t = 0; t < GD_NT; ++t) {
    kk[t] = (blockIdx.y * GD_NT + t) * GD_THREADS + threadIdx.x;
    double q[3] = {0.0, 0.0, 0.0};
    if (kk[t] < Kstar) frame_apply(e1, e2, cx, cy, cz, zloc[3 * kk[t]], zloc[3 * kk[t] + 1], zloc[3 * kk[t] + 2], q);
    const double sc = (sizeof(R) == 4) ? 0.5 : 1.0;  // FP32: half-scaled offsets
    ax[t] = (R)(sc * q[0]);
    ay[t] = (R)(sc * q[1]);
    az[t] = (R)(sc * q[2]);
    acc[t] = 0.0;
  }
  const int64_t lo = g.pbase[b], hi = g.pbase[b + 1];
  for (int64_t j0 = lo; j0 < hi; j0 += JT) {
    const int nj = (int)min((int64_t)JT, hi - j0);
    __syncthreads();
    if (threadIdx.x < nj) {
      const int64_t j = j0 + threadIdx.x;
      const double d0 = g.centres[3 * j] - cx, d1 = g.centres[3 * j + 1] - cy, d2 = g.centres[3 * j + 2] - cz;
      D[threadIdx.x][0] = d0;
      D[threadIdx.x][1] = d1;
      D[threadIdx.x][2] = d2;
      int cnt = 0, col = 0;
      if (j != i) {
        const double dist = 2.0 * asin(fmin(1.0, 0.5 * sqrt(d0 * d0 + d1 * d1 + d2 * d2)));
        const int k = group_rep(dist - eps, nrep, g.rep_rho + rb);
        cnt = g.rep_p[rb + k];
        col = g.rep_off[rb + k];
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
    for (int idx = threadIdx.x; idx < ns; idx += GD_THREADS) {
      int jj = 0;
      while (idx >= toff[jj + 1]) ++jj;
      const int64_t s = g.roff[j0 + jj] + tcol[jj] + (idx - toff[jj]);
      V4 v;
      v.x = (R)D[jj][0] + soff[3 * s];
      v.y = (R)D[jj][1] + soff[3 * s + 1];
      v.z = (R)D[jj][2] + soff[3 * s + 2];
      v.w = rho[s];
      if constexpr (sizeof(R) == 4) {
        v.x *= 0.5f;
        v.y *= 0.5f;
        v.z *= 0.5f;
      }
      S[idx] = v;
    }
    __syncthreads();
    R part[GD_NT];
#pragma unroll
    for (int t = 0; t < GD_NT; ++t) part[t] = 0;
    if constexpr (sizeof(R) == 4) {
      pair_loop32<MODE, GD_NT>(reinterpret_cast<const float4*>(S), ns, ax, ay, az, part);
    } else {
      for (int s = 0; s < ns; ++s) {
        const V4 v = S[s];
#pragma unroll
        for (int t = 0; t < GD_NT; ++t) {
          const R dx = ax[t] - v.x, dy = ay[t] - v.y, dz = az[t] - v.z;
          part[t] = fma(green64<MODE>(fma(dx, dx, fma(dy, dy, dz * dz))), v.w, part[t]);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < GD_NT; ++t) acc[t] += (double)part[t];
  }
#pragma unroll
  for (int t = 0; t < GD_NT; ++t)
    if (kk[t] < Kstar) g.z[i * Kstar + kk[t]] = acc[t];
}

// Float-float variant (FP64-accurate on the FP32 pipes): sources staged as (hi, lo).
template <int MODE>
__global__ void __launch_bounds__(GD_THREADS) group_direct_df_kernel(GroupDev g, int JT) {
  extern __shared__ float4 gdd_smem[];
  __shared__ float4 tab[kLogTable];
  __shared__ double D[GD_JT][3];
  __shared__ int toff[GD_JT + 1], tcol[GD_JT];
  float4* Sh = gdd_smem;
  float4* Sl = gdd_smem + JT * g.pmax;
  for (int t = threadIdx.x; t < kLogTable; t += blockDim.x) tab[t] = g.logtab[t];
  const int64_t i = blockIdx.x;
  const int b = g.pinst[i];
  const int Kstar = g.Kstar;
  const double eps = g.inst_eps[b];
  const int nrep = g.inst_nrep[b], rb = g.inst_repbase[b];
  const double* zloc = g.zloc + (int64_t)3 * Kstar * b;
  const double cx = g.centres[3 * i], cy = g.centres[3 * i + 1], cz = g.centres[3 * i + 2];
  double e1[3], e2[3];
  patch_frame(cx, cy, cz, e1, e2);
  f2 a[GD_NT][3];
  double acc[GD_NT];
  int kk[GD_NT];
#pragma unroll
  for (int t = 0; t < GD_NT; ++t) {
    kk[t] = (blockIdx.y * GD_NT + t) * GD_THREADS + threadIdx.x;
    double q[3] = {0.0, 0.0, 0.0};
    if (kk[t] < Kstar) frame_apply(e1, e2, cx, cy, cz, zloc[3 * kk[t]], zloc[3 * kk[t] + 1], zloc[3 * kk[t] + 2], q);
    for (int c = 0; c < 3; ++c) a[t][c] = f2_from_double(q[c]);
    acc[t] = 0.0;
  }
  const int64_t lo = g.pbase[b], hi = g.pbase[b + 1];
  for (int64_t j0 = lo; j0 < hi; j0 += JT) {
    const int nj = (int)min((int64_t)JT, hi - j0);
    __syncthreads();
    if (threadIdx.x < nj) {
      const int64_t j = j0 + threadIdx.x;
      const double d0 = g.centres[3 * j] - cx, d1 = g.centres[3 * j + 1] - cy, d2 = g.centres[3 * j + 2] - cz;
      D[threadIdx.x][0] = d0;
      D[threadIdx.x][1] = d1;
      D[threadIdx.x][2] = d2;
      int cnt = 0, col = 0;
      if (j != i) {
        const double dist = 2.0 * asin(fmin(1.0, 0.5 * sqrt(d0 * d0 + d1 * d1 + d2 * d2)));
        const int k = group_rep(dist - eps, nrep, g.rep_rho + rb);
        cnt = g.rep_p[rb + k];
        col = g.rep_off[rb + k];
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
    for (int idx = threadIdx.x; idx < ns; idx += GD_THREADS) {
      int jj = 0;
      while (idx >= toff[jj + 1]) ++jj;
      const int64_t s = g.roff[j0 + jj] + tcol[jj] + (idx - toff[jj]);
      const f2 x = f2_from_double(D[jj][0] + g.soff64[3 * s]), y = f2_from_double(D[jj][1] + g.soff64[3 * s + 1]),
               zz = f2_from_double(D[jj][2] + g.soff64[3 * s + 2]), r = f2_from_double(g.rho64[s]);
      Sh[idx] = make_float4(x.hi, y.hi, zz.hi, r.hi);
      Sl[idx] = make_float4(x.lo, y.lo, zz.lo, r.lo);
    }
    __syncthreads();
    f2 part[GD_NT];
    {
      f2x2 A[3], P{x2_splat(0.0f), x2_splat(0.0f)};
#pragma unroll
      for (int c = 0; c < 3; ++c) A[c] = f2x2{x2_pack(a[0][c].hi, a[1][c].hi), x2_pack(a[0][c].lo, a[1][c].lo)};
      for (int s = 0; s < ns; ++s) pair_f2_acc_x2<MODE>(A, Sh[s], Sl[s], tab, P);
      x2_unpack(P.hi, part[0].hi, part[1].hi);
      x2_unpack(P.lo, part[0].lo, part[1].lo);
    }
#pragma unroll
    for (int t = 0; t < GD_NT; ++t) acc[t] += f2_to_double(part[t]);
  }
#pragma unroll
  for (int t = 0; t < GD_NT; ++t)
    if (kk[t] < Kstar) g.z[i * Kstar + kk[t]] = acc[t];
}

// ---- segmented GMRES: instance b owns entries [pbase[b] K, pbase[b + 1] K) of every vector
// and its own state st[b], Hessenberg block, rotations, g and y.

// h[b][j] = V_j . w over instance b's segment, j <= m_b; one block per (instance, column slice)
__global__ void __launch_bounds__(256) group_dots_kernel(GroupDev g, const double* __restrict__ V, int64_t ld,
                                                         const double* __restrict__ w, double* __restrict__ hout) {
  const int b = blockIdx.x;
  const GmresState* st = g.st + b;
  if (st->done) return;
  const int k = st->m;
  const int64_t lo = g.pbase[b] * (int64_t)g.K, hi = g.pbase[b + 1] * (int64_t)g.K;
  __shared__ double red[256];
  for (int j = blockIdx.y; j <= k; j += gridDim.y) {
    const double* v = V + j * ld;
    double acc = 0.0;
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) acc = fma(v[e], w[e], acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) hout[(int64_t)b * (g.maxit + 1) + j] = red[0];
    __syncthreads();
  }
}

// w -= sum_j h[b][j] V_j on instance b's segment; per block the partial |w|^2
__global__ void __launch_bounds__(256) group_update_kernel(GroupDev g, const double* __restrict__ V, int64_t ld,
                                                           double* __restrict__ w, const double* __restrict__ h) {
  const int b = blockIdx.x;
  const GmresState* st = g.st + b;
  if (st->done) return;
  const int k = st->m;
  const int64_t lo = g.pbase[b] * (int64_t)g.K, hi = g.pbase[b + 1] * (int64_t)g.K;
  extern __shared__ double hs[];
  __shared__ double red[256];
  for (int j = threadIdx.x; j <= k; j += blockDim.x) hs[j] = h[(int64_t)b * (g.maxit + 1) + j];
  __syncthreads();
  double nrm = 0.0;
  for (int64_t e = lo + (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < hi; e += (int64_t)gridDim.y * blockDim.x) {
    double a = 0.0;
    for (int j = 0; j <= k; ++j) a = fma(hs[j], V[j * ld + e], a);
    const double we = w[e] - a;
    w[e] = we;
    nrm = fma(we, we, nrm);
  }
  red[threadIdx.x] = nrm;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) g.pnorm[(int64_t)b * gridDim.y + blockIdx.y] = red[0];
}

// Column m_b of instance b's Hessenberg matrix and its rotations (one warp per instance).
__global__ void group_givens_kernel(GroupDev g, int nb) {
  const int b = blockIdx.x;
  GmresState* st = g.st + b;
  if (st->done) return;
  double s = 0.0;
  for (int q = threadIdx.x; q < nb; q += 32) s += g.pnorm[(int64_t)b * nb + q];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x != 0) return;
  const int k = st->m, ldh = g.maxit + 1;
  double* H = g.H + (int64_t)b * ldh * g.maxit;
  double* cs = g.cs + (int64_t)b * g.maxit;
  double* sn = g.sn + (int64_t)b * g.maxit;
  double* gg = g.g + (int64_t)b * ldh;
  const double* h1 = g.h1 + (int64_t)b * ldh;
  const double* h2 = g.h2 + (int64_t)b * ldh;
  const double hn = sqrt(s);
  double* col = H + (int64_t)k * ldh;
  bool finite = isfinite(hn);
  for (int j = 0; j <= k; ++j) {
    col[j] = h1[j] + h2[j];
    finite = finite && isfinite(col[j]);
  }
  if (k == 0) gg[0] = st->beta;
  for (int j = 0; j < k; ++j) {
    const double a = col[j], c = col[j + 1];
    col[j] = cs[j] * a + sn[j] * c;
    col[j + 1] = -sn[j] * a + cs[j] * c;
  }
  const double a = col[k];
  const double rr = hypot(a, hn);
  st->hn = hn;
  st->m = k + 1;
  if (!finite || !(rr > 0.0)) {
    st->flag = finite ? kGmresBreakdown : kGmresNonFinite;
    st->done = 1;
    st->m = k;
    return;
  }
  cs[k] = a / rr;
  sn[k] = hn / rr;
  col[k] = rr;
  col[k + 1] = 0.0;
  gg[k + 1] = -sn[k] * gg[k];
  gg[k] = cs[k] * gg[k];
  const double res = fabs(gg[k + 1]) / st->beta;
  st->res = res;
  if (res <= st->tol) {
    st->flag = kGmresConverged;
    st->done = 1;
  } else if (hn == 0.0) {
    st->flag = kGmresHappy;
    st->done = 1;
  } else if (k + 1 >= st->maxit) {
    st->done = 1;
  }
}

// V_{m_b}[seg_b] = vk[seg_b] = w[seg_b] / hn_b (m_b already advanced)
__global__ void group_normalize_kernel(GroupDev g, const double* __restrict__ w, double* __restrict__ V, int64_t ld) {
  const int b = blockIdx.x;
  const GmresState* st = g.st + b;
  if (st->done) return;
  const double a = 1.0 / st->hn;
  double* v = V + (int64_t)st->m * ld;
  const int64_t lo = g.pbase[b] * (int64_t)g.K, hi = g.pbase[b + 1] * (int64_t)g.K;
  for (int64_t e = lo + (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < hi; e += (int64_t)gridDim.y * blockDim.x) {
    const double x = a * w[e];
    v[e] = x;
    g.vk[e] = x;
  }
}

// y_b = R_b^-1 g_b (one thread per instance)
__global__ void group_backsolve_kernel(GroupDev g) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= g.B) return;
  const GmresState* st = g.st + b;
  const int m = st->m, ldh = g.maxit + 1;
  const double* H = g.H + (int64_t)b * ldh * g.maxit;
  const double* gg = g.g + (int64_t)b * ldh;
  double* y = g.y + (int64_t)b * g.maxit;
  for (int i = m - 1; i >= 0; --i) {
    double t = gg[i];
    for (int j = i + 1; j < m; ++j) t -= H[(int64_t)j * ldh + i] * y[j];
    y[i] = t / H[(int64_t)i * ldh + i];
  }
}

// e[seg_b] = sum_{j < m_b} y_b[j] V_j[seg_b]
__global__ void group_combination_kernel(GroupDev g, const double* __restrict__ V, int64_t ld, double* __restrict__ e) {
  const int b = blockIdx.x;
  const int m = g.st[b].m;
  const double* y = g.y + (int64_t)b * g.maxit;
  const int64_t lo = g.pbase[b] * (int64_t)g.K, hi = g.pbase[b + 1] * (int64_t)g.K;
  for (int64_t q = lo + (int64_t)blockIdx.y * blockDim.x + threadIdx.x; q < hi; q += (int64_t)gridDim.y * blockDim.x) {
    double a = 0.0;
    for (int j = 0; j < m; ++j) a = fma(y[j], V[j * ld + q], a);
    e[q] = a;
  }
}

// out[b] = a . c over instance b's segment (one block per instance)
__global__ void __launch_bounds__(256) group_seg_dot_kernel(GroupDev g, const double* __restrict__ a,
                                                            const double* __restrict__ c, double* __restrict__ out) {
  const int b = blockIdx.x;
  const int64_t lo = g.pbase[b] * (int64_t)g.K, hi = g.pbase[b + 1] * (int64_t)g.K;
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) acc = fma(a[e], c[e], acc);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[b] = red[0];
}

// out[b] = I_b . sum over instance b's patches of x_i (eq. getI)
__global__ void __launch_bounds__(128) group_isigma_kernel(GroupDev g, const double* __restrict__ x,
                                                           double* __restrict__ out) {
  const int b = blockIdx.x;
  const int K = g.K;
  __shared__ double red[128];
  double acc = 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double s = 0.0;
    for (int64_t i = g.pbase[b]; i < g.pbase[b + 1]; ++i) s += x[i * K + k];
    acc = fma(g.I[(int64_t)b * K + k], s, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[b] = red[0];
}

// x[seg_b] = a_b x[seg_b], per-instance scalars
__global__ void group_scale_kernel(GroupDev g, const double* __restrict__ a, double* __restrict__ x) {
  const int b = blockIdx.x;
  const int64_t lo = g.pbase[b] * (int64_t)g.K, hi = g.pbase[b + 1] * (int64_t)g.K;
  const double s = a[b];
  for (int64_t e = lo + (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < hi; e += (int64_t)gridDim.y * blockDim.x)
    x[e] *= s;
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

int group_seg_blocks(int64_t maxseg) { return (int)std::max<int64_t>(1, std::min<int64_t>(8, (maxseg + 2047) / 2048)); }

cudaError_t launch_group_field(const GroupDev& g, const double* x, int prec, cudaStream_t s) {
  cudaError_t e;
  if (prec == NCS_FP32) {
    count_launch(), group_outgoing_kernel<float><<<(unsigned)g.P, GO_THREADS, g.K * sizeof(float), s>>>(g, x);
  } else {
    count_launch(), group_outgoing_kernel<double><<<(unsigned)g.P, GO_THREADS, g.K * sizeof(double), s>>>(g, x);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const dim3 grid((unsigned)g.P, (unsigned)((g.Kstar + GD_THREADS * GD_NT - 1) / (GD_THREADS * GD_NT)));
  // source patches staged per tile: at most GD_JT, within 40 KB of shared memory
  const size_t v4 = prec == NCS_FP64 ? sizeof(double4_16a) : prec == NCS_DF64 ? 2 * sizeof(float4) : sizeof(float4);
  const int JT = (int)std::max<size_t>(1, std::min<size_t>(GD_JT, (40 * 1024) / (v4 * (size_t)g.pmax)));
  const size_t sm = (size_t)JT * g.pmax * v4;
  if (prec == NCS_FP32) {
    auto k = g.mode == 0 ? &group_direct_kernel<float, 0> : &group_direct_kernel<float, 1>;
    if ((e = allow_smem(k, sm)) != cudaSuccess) return e;
    count_launch(), k<<<grid, GD_THREADS, sm, s>>>(g, JT);
  } else if (prec == NCS_DF64) {
    auto k = g.mode == 0 ? &group_direct_df_kernel<0> : &group_direct_df_kernel<1>;
    if ((e = allow_smem(k, sm)) != cudaSuccess) return e;
    count_launch(), k<<<grid, GD_THREADS, sm, s>>>(g, JT);
  } else {
    auto k = g.mode == 0 ? &group_direct_kernel<double, 0> : &group_direct_kernel<double, 1>;
    if ((e = allow_smem(k, sm)) != cudaSuccess) return e;
    count_launch(), k<<<grid, GD_THREADS, sm, s>>>(g, JT);
  }
  return cudaGetLastError();
}

cudaError_t launch_group_arnoldi(const GroupDev& g, const double* V, double* w, cudaStream_t s) {
  const int64_t ld = g.P * (int64_t)g.K;
  const int nb = g.seg_blocks;
  const size_t hsm = (size_t)(g.maxit + 1) * sizeof(double);
  for (int pass = 0; pass < 2; ++pass) {
    count_launch(), group_dots_kernel<<<dim3(g.B, 4), 256, 0, s>>>(g, V, ld, w, pass == 0 ? g.h1 : g.h2);
    count_launch(), group_update_kernel<<<dim3(g.B, nb), 256, hsm, s>>>(g, V, ld, w, pass == 0 ? g.h1 : g.h2);
  }
  count_launch(), group_givens_kernel<<<g.B, 32, 0, s>>>(g, nb);
  count_launch(), group_normalize_kernel<<<dim3(g.B, nb), 256, 0, s>>>(g, w, const_cast<double*>(V), ld);
  return cudaGetLastError();
}

cudaError_t launch_group_solution(const GroupDev& g, const double* V, double* e, cudaStream_t s) {
  count_launch(), group_backsolve_kernel<<<(g.B + 31) / 32, 32, 0, s>>>(g);
  count_launch(), group_combination_kernel<<<dim3(g.B, g.seg_blocks), 256, 0, s>>>(g, V, g.P * (int64_t)g.K, e);
  return cudaGetLastError();
}

cudaError_t launch_group_dots(const GroupDev& g, const double* a, const double* c, double* out, cudaStream_t s) {
  count_launch(), group_seg_dot_kernel<<<g.B, 256, 0, s>>>(g, a, c, out);
  return cudaGetLastError();
}

cudaError_t launch_group_isigma(const GroupDev& g, const double* x, double* out, cudaStream_t s) {
  count_launch(), group_isigma_kernel<<<g.B, 128, 0, s>>>(g, x, out);
  return cudaGetLastError();
}

cudaError_t launch_group_scale(const GroupDev& g, const double* a, double* x, cudaStream_t s) {
  count_launch(), group_scale_kernel<<<dim3(g.B, g.seg_blocks), 256, 0, s>>>(g, a, x);
  return cudaGetLastError();
}

}  // namespace ncs
