// Device part of the tree product (Kaye & Greengard, Section 7, Step 3.2-3.4):
//   P2L   : skeleton sources of the interaction list summed onto a group's incoming
//           grid (parity-restricted Chebyshev radii x equispaced angles, Section 7.3);
//   coef  : grid values -> Chebyshev-Fourier coefficients (the "q^2 to form the
//           interpolant" of Step 3.4, done as an angular DFT then a radial transform);
//   direct: sources evaluated directly at the Zernike nodes (leaf neighbours, and
//           groups too small to profit from a grid);
//   L2P   : every patch interpolates the grids of its groups at its Zernike nodes.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <vector>

#include "device_common.cuh"
#include "df64.cuh"
#include "internal.hpp"
#include "numerics.hpp"

namespace ncs {

namespace {

template <typename R>
struct V4T;
template <>
struct V4T<float> {
  using type = float4;
};
template <>
struct V4T<double> {
  using type = double4_16a;
};

template <typename T>
cudaError_t up(T** d, const std::vector<T>& h) {
  cudaError_t e = cudaMalloc(d, std::max<size_t>(1, h.size()) * sizeof(T));
  if (e != cudaSuccess) return e;
  if (!h.empty()) e = cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

template <typename T>
void fr(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

constexpr int P2L_THREADS = 256;
constexpr int P2L_NT = 2;
// source patches staged per shared-memory tile of a P2L work item
#ifndef NCS_P2L_JT
#define NCS_P2L_JT 16
#endif
constexpr int P2L_JT = NCS_P2L_JT;
// the float-float P2L stages (hi, lo) pairs of float4: 8 patches per tile keep its shared
// memory (43 KB at p = 169) at the FP32 kernel's, and its blocks per SM with it
constexpr int P2L_DF_JT = 8;

// One block per work item (grid group g, a slice of its interaction-list patches). JT
// source patches per shared-memory tile, POLY of every 16 packed pair chains with the
// logarithm on the FMA pipe (FP32 only): both chosen at run time (KernelConfig).
template <typename R, int MODE, int JT = P2L_JT, int POLY = NCS_PAIR_X2_POLY, int RSQ = 0>
__global__ void __launch_bounds__(P2L_THREADS) p2l_kernel(
    const int* __restrict__ witem_group, const int* __restrict__ witem_rep, const int* __restrict__ rep_p,
    const int* __restrict__ rep_off, int pt, const int64_t* __restrict__ witem_lo, const int64_t* __restrict__ witem_hi,
    const int* __restrict__ isrc, const double* __restrict__ gcen, const int* __restrict__ gshape,
    const int64_t* __restrict__ goff, const int* __restrict__ shape_nr, const int* __restrict__ shape_nth,
    const R* __restrict__ gpos, const double* __restrict__ centres, const R* __restrict__ soff,
    const R* __restrict__ rho, double* __restrict__ grid) {
  using V4 = typename V4T<R>::type;
  extern __shared__ unsigned char p2l_smem[];
  __shared__ double D[JT][3];
  const int item = blockIdx.x;
  const int g = witem_group[item];
  const int rk = witem_rep[item];
  const int p = rep_p[rk], col = rep_off[rk];
  V4* S = reinterpret_cast<V4*>(p2l_smem);
  const int64_t lo = witem_lo[item], hi = witem_hi[item];
  const int sh = gshape[g];
  const int q = shape_nr[sh] * shape_nth[sh];
  const int64_t off = goff[g];
  const double gx = gcen[3 * g], gy = gcen[3 * g + 1], gz = gcen[3 * g + 2];
  for (int base = 0; base < q; base += P2L_THREADS * P2L_NT) {
    R ax[P2L_NT], ay[P2L_NT], az[P2L_NT];
    double acc[P2L_NT];
#pragma unroll
    for (int t = 0; t < P2L_NT; ++t) {
      const int a = base + t * P2L_THREADS + threadIdx.x;
      const R sc = (sizeof(R) == 4) ? (R)0.5 : (R)1;  // FP32: half-scaled offsets
      if (a < q) {
        ax[t] = sc * gpos[3 * (off + a)];
        ay[t] = sc * gpos[3 * (off + a) + 1];
        az[t] = sc * gpos[3 * (off + a) + 2];
      } else {
        ax[t] = ay[t] = az[t] = (R)0;
      }
      acc[t] = 0.0;
    }
    for (int64_t s0 = lo; s0 < hi; s0 += JT) {
      const int nj = (int)min((int64_t)JT, hi - s0);
      __syncthreads();
      if (threadIdx.x < nj * 3) {
        const int jj = threadIdx.x / 3, c = threadIdx.x - 3 * jj;
        const int j = isrc[s0 + jj];
        D[jj][c] = centres[3 * j + c] - (c == 0 ? gx : (c == 1 ? gy : gz));
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < nj * p; idx += P2L_THREADS) {
        const int jj = idx / p;
        const int64_t gsrc = (int64_t)isrc[s0 + jj] * pt + col + (idx - jj * p);
        V4 v;
        v.x = (R)D[jj][0] + soff[3 * gsrc];
        v.y = (R)D[jj][1] + soff[3 * gsrc + 1];
        v.z = (R)D[jj][2] + soff[3 * gsrc + 2];
        v.w = rho[gsrc];
        if constexpr (sizeof(R) == 4) {  // the FP32 pairs take half-scaled offsets
          v.x *= 0.5f;
          v.y *= 0.5f;
          v.z *= 0.5f;
          if constexpr (NCS_PAIR_X2 != 0) {
            stage_source_x2(reinterpret_cast<float4*>(S), idx, v.x, v.y, v.z, v.w);
            continue;
          }
        }
        S[idx] = v;
      }
      const int ns = nj * p;
      if constexpr (sizeof(R) == 4 && NCS_PAIR_X2 != 0) {
        if (threadIdx.x == 0) stage_pad_x2(reinterpret_cast<float4*>(S), ns);
      }
      __syncthreads();
      R part[P2L_NT];
#pragma unroll
      for (int t = 0; t < P2L_NT; ++t) part[t] = 0;
      // warps whose every target slot lies beyond the grid skip the pair work
      const int wbase = base + (threadIdx.x & ~31);
      const int nact = (wbase >= q) ? 0 : ((wbase + P2L_THREADS >= q) ? 1 : P2L_NT);
      if constexpr (sizeof(R) == 4) {
        if constexpr (NCS_PAIR_X2 != 0) {
          if (nact == P2L_NT)
            pair_loop32x2<MODE, P2L_NT, POLY, RSQ>(S, ns, ax, ay, az, part);
          else if (nact == 1)
            pair_loop32x2<MODE, 1, POLY, RSQ>(S, ns, ax, ay, az, part);
        } else {
          if (nact == P2L_NT)
            pair_loop32<MODE, P2L_NT>(S, ns, ax, ay, az, part);
          else if (nact == 1)
            pair_loop32<MODE, 1>(S, ns, ax, ay, az, part);
        }
      } else if (nact > 0) {
        for (int s = 0; s < ns; ++s) {
          const V4 v = S[s];
#pragma unroll
          for (int t = 0; t < P2L_NT; ++t) {
            const R dx = ax[t] - v.x, dy = ay[t] - v.y, dz = az[t] - v.z;
            part[t] = fma(green64<MODE>(fma(dx, dx, fma(dy, dy, dz * dz))), v.w, part[t]);
          }
        }
      }
#pragma unroll
      for (int t = 0; t < P2L_NT; ++t) acc[t] += (double)part[t];
    }
#pragma unroll
    for (int t = 0; t < P2L_NT; ++t) {
      const int a = base + t * P2L_THREADS + threadIdx.x;
      if (a < q) atomicAdd(&grid[off + a], acc[t]);
    }
  }
}

// Grid values -> coefficients. Layout per group: A[m][j] then B[m][j],
// m = 0..nth/2-1, j = 0..nr-1, for the expansion
//   F(r, th) = sum_m sum_j (A_mj cos m th + B_mj sin m th) T_{2j + (m mod 2)}(r / R).
// Angular: C_m(r_a) = (2 - delta_m0)/nth sum_b F_ab cos(m th_b), S_m likewise with sin.
// Radial (parity-restricted Chebyshev on the 2 nr first-kind nodes of [-R, R]):
//   A_mj = (2 - delta_d0)/nr sum_a C_m(r_a) T_d(x_a), d = 2j + (m mod 2),
//   x_a = cos((2a + 1) pi / (4 nr)).
template <typename R>
__global__ void __launch_bounds__(256) coef_kernel(int g0, const int* __restrict__ gshape, const int64_t* __restrict__ goff,
                                                   const int* __restrict__ shape_nr, const int* __restrict__ shape_nth,
                                                   const double* __restrict__ grid, double* __restrict__ coef) {
  extern __shared__ double cf_smem[];
  const int g = g0 + blockIdx.x;
  const int sh = gshape[g];
  const int nr = shape_nr[sh], nth = shape_nth[sh], q = nr * nth, mh = nth / 2;
  const int64_t off = goff[g];
  double* F = cf_smem;        // q
  double* CS = cf_smem + q;   // 2 * mh * nr: C then S, [m][a]
  // tables (after F and CS, sized for the largest shape): cos and sin of 2 pi k / nth, and
  // the Chebyshev values T_d(x_a) = cos(d (2a + 1) pi / (4 nr)), d < 2 nr
  R* CT = reinterpret_cast<R*>(cf_smem + 2 * q);
  R* ST = CT + nth;
  R* TD = ST + nth;  // [d][a]
  for (int i = threadIdx.x; i < q; i += blockDim.x) F[i] = grid[off + i];
  for (int k = threadIdx.x; k < nth; k += blockDim.x) sincospi((R)(2 * k) / (R)nth, &ST[k], &CT[k]);
  for (int i = threadIdx.x; i < 2 * nr * nr; i += blockDim.x) {
    const int d = i / nr, a = i - d * nr;
    TD[i] = cospi((R)(d * (2 * a + 1)) / (R)(4 * nr));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < mh * nr; i += blockDim.x) {
    const int m = i / nr, a = i - m * nr;
    R c = 0, s = 0;
    int k = 0;  // (m * b) mod nth
    for (int b = 0; b < nth; ++b) {
      const R f = (R)F[a * nth + b];
      c = fma(f, CT[k], c);
      s = fma(f, ST[k], s);
      k += m;
      if (k >= nth) k -= nth;
    }
    const R w = (m == 0 ? (R)1 : (R)2) / (R)nth;
    CS[m * nr + a] = (double)(w * c);
    CS[mh * nr + m * nr + a] = (double)(w * s);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < mh * nr; i += blockDim.x) {
    const int m = i / nr, j = i - m * nr;
    const int d = 2 * j + (m & 1);
    const R* Td = TD + d * nr;
    R A = 0, B = 0;
    for (int a = 0; a < nr; ++a) {
      A = fma((R)CS[m * nr + a], Td[a], A);
      B = fma((R)CS[mh * nr + m * nr + a], Td[a], B);
    }
    const R w = (d == 0 ? (R)1 : (R)2) / (R)nr;
    coef[off + i] = (double)(w * A);
    coef[off + mh * nr + i] = (double)(w * B);
  }
}

// Direct sums at the Zernike nodes over a per-patch source list (overwrites z).
// direct lists: one block per target patch, DT_NT Zernike nodes per thread
#ifndef NCS_DT_NT
#define NCS_DT_NT 2
#endif
constexpr int DT_NT = NCS_DT_NT;
constexpr int DT_THREADS = 512 / DT_NT;
// the float-float direct lists keep two nodes per thread (register pressure)
constexpr int DTD_NT = 2;
constexpr int DTD_THREADS = 256;
constexpr int DT_JT = 8;
// the paired staging pads an odd source count by one: even tile counts keep the padded
// count within the tile's shared memory (an odd count only occurs in a partial tile)
static_assert(P2L_JT % 2 == 0 && DT_JT % 2 == 0, "tile source counts must be even");

template <typename R, int MODE, int POLY = NCS_PAIR_X2_POLY, int RSQ = 0>
__global__ void __launch_bounds__(DT_THREADS) direct_list_kernel(
    int pt, int Kstar, int pmax, const int* __restrict__ rep_p, const int* __restrict__ rep_off,
    const int64_t* __restrict__ pd_off, const int* __restrict__ pd, const int* __restrict__ pdk,
    const double* __restrict__ centres, const double* __restrict__ zloc, const R* __restrict__ soff,
    const R* __restrict__ rho, double* __restrict__ z) {
  using V4 = typename V4T<R>::type;
  extern __shared__ unsigned char dt_smem[];
  V4* S = reinterpret_cast<V4*>(dt_smem);
  __shared__ double D[DT_JT][3];
  __shared__ int toff[DT_JT + 1], tcol[DT_JT];
  const int64_t i = blockIdx.x;
  const double cx = centres[3 * i], cy = centres[3 * i + 1], cz = centres[3 * i + 2];
  double e1[3], e2[3];
  patch_frame(cx, cy, cz, e1, e2);
  R ax[DT_NT], ay[DT_NT], az[DT_NT];
  double acc[DT_NT];
  int kk[DT_NT];
#pragma unroll
  for (int t = 0; t < DT_NT; ++t) {
    kk[t] = (blockIdx.y * DT_NT + t) * DT_THREADS + threadIdx.x;
    double gq[3] = {0.0, 0.0, 0.0};
    if (kk[t] < Kstar) frame_apply(e1, e2, cx, cy, cz, zloc[3 * kk[t]], zloc[3 * kk[t] + 1], zloc[3 * kk[t] + 2], gq);
    const double sc = (sizeof(R) == 4) ? 0.5 : 1.0;  // FP32: half-scaled offsets
    ax[t] = (R)(sc * gq[0]);
    ay[t] = (R)(sc * gq[1]);
    az[t] = (R)(sc * gq[2]);
    acc[t] = 0.0;
  }
  const int64_t lo = pd_off[i], hi = pd_off[i + 1];
  for (int64_t s0 = lo; s0 < hi; s0 += DT_JT) {
    const int nj = (int)min((int64_t)DT_JT, hi - s0);
    __syncthreads();
    if (threadIdx.x < nj) {
      const int64_t j = pd[s0 + threadIdx.x];
      const int k = pdk[s0 + threadIdx.x];
      for (int c = 0; c < 3; ++c) D[threadIdx.x][c] = centres[3 * j + c] - centres[3 * i + c];
      toff[threadIdx.x + 1] = rep_p[k];
      tcol[threadIdx.x] = rep_off[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      toff[0] = 0;
      for (int jj = 0; jj < nj; ++jj) toff[jj + 1] += toff[jj];
    }
    __syncthreads();
    const int ns = toff[nj];
    for (int idx = threadIdx.x; idx < ns; idx += DT_THREADS) {
      int jj = 0;
      while (idx >= toff[jj + 1]) ++jj;
      const int64_t gsrc = (int64_t)pd[s0 + jj] * pt + tcol[jj] + (idx - toff[jj]);
      V4 v;
      v.x = (R)D[jj][0] + soff[3 * gsrc];
      v.y = (R)D[jj][1] + soff[3 * gsrc + 1];
      v.z = (R)D[jj][2] + soff[3 * gsrc + 2];
      v.w = rho[gsrc];
      if constexpr (sizeof(R) == 4) {  // the FP32 pairs take half-scaled offsets
        v.x *= 0.5f;
        v.y *= 0.5f;
        v.z *= 0.5f;
        if constexpr (NCS_PAIR_X2 != 0) {
          stage_source_x2(reinterpret_cast<float4*>(S), idx, v.x, v.y, v.z, v.w);
          continue;
        }
      }
      S[idx] = v;
    }
    if constexpr (sizeof(R) == 4 && NCS_PAIR_X2 != 0) {
      if (threadIdx.x == 0) stage_pad_x2(reinterpret_cast<float4*>(S), ns);
    }
    __syncthreads();
    R part[DT_NT];
#pragma unroll
    for (int t = 0; t < DT_NT; ++t) part[t] = 0;
    if constexpr (sizeof(R) == 4) {
      if constexpr (NCS_PAIR_X2 != 0)
        pair_loop32x2<MODE, DT_NT, POLY, RSQ>(S, ns, ax, ay, az, part);
      else
        pair_loop32<MODE, DT_NT>(S, ns, ax, ay, az, part);
    } else {
      for (int s = 0; s < ns; ++s) {
        const V4 v = S[s];
#pragma unroll
        for (int t = 0; t < DT_NT; ++t) {
          const R dx = ax[t] - v.x, dy = ay[t] - v.y, dz = az[t] - v.z;
          part[t] = fma(green64<MODE>(fma(dx, dx, fma(dy, dy, dz * dz))), v.w, part[t]);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < DT_NT; ++t) acc[t] += (double)part[t];
  }
#pragma unroll
  for (int t = 0; t < DT_NT; ++t)
    if (kk[t] < Kstar) z[i * Kstar + kk[t]] = acc[t];
}

// Value at (rho = r/R, cos th, sin th) of a group expansion with coefficients C
// (A[m][j] then B[m][j]): Clenshaw in y = T_2(rho) over the even (T_2j) and odd
// (T_2j+1) radial series, cos/sin(m th) by the angle-addition recurrence.
template <typename R>
__device__ __forceinline__ R eval_expansion(const R* C, int nr, int mh, R rho, R ct, R st) {
  const R y = fma((R)2 * rho, rho, (R)-1);
  const R y2 = y + y;
  R cm = 1, sm = 0, val = 0;
  for (int m = 0; m < mh; ++m) {
    const R* A = C + m * nr;
    const R* B = C + mh * nr + m * nr;
    R ba1 = 0, ba2 = 0, bb1 = 0, bb2 = 0;
    for (int j = nr - 1; j >= 0; --j) {
      const R ta = fma(y2, ba1, A[j] - ba2);
      const R tb = fma(y2, bb1, B[j] - bb2);
      ba2 = ba1;
      ba1 = ta;
      bb2 = bb1;
      bb1 = tb;
    }
    R sa, sb;
    if ((m & 1) == 0) {  // phi_0 = 1, phi_1 = y: sum = b0 - y b1
      sa = fma(-y, ba2, ba1);
      sb = fma(-y, bb2, bb1);
    } else {  // phi_0 = rho, phi_1 = T_3(rho) = rho (2y - 1): sum = rho (b0 - b1)
      sa = rho * (ba1 - ba2);
      sb = rho * (bb1 - bb2);
    }
    val = fma(cm, sa, fma(sm, sb, val));
    const R cn = cm * ct - sm * st;
    sm = sm * ct + cm * st;
    cm = cn;
  }
  return val;
}

// Polar coordinates, in the frame of a group centred at g (unit) with radius Rg, of
// the point g + (dx, dy, dz): rho = geodesic distance / Rg, and the angle's cos/sin.
__device__ __forceinline__ void group_polar(double dx, double dy, double dz, const double* g, double Rg,
                                            double* rho, double* ct, double* st) {
  double f1[3], f2[3];
  patch_frame(g[0], g[1], g[2], f1, f2);
  const double u1 = dx * f1[0] + dy * f1[1] + dz * f1[2];
  const double u2 = dx * f2[0] + dy * f2[1] + dz * f2[2];
  const double u3 = dx * g[0] + dy * g[1] + dz * g[2];
  const double sr = sqrt(u1 * u1 + u2 * u2);
  *rho = atan2(sr, 1.0 + u3) / Rg;
  *ct = sr > 0.0 ? u1 / sr : 1.0;
  *st = sr > 0.0 ? u2 / sr : 0.0;
}

// L2P: z_i(k) += expansion of every listed grid group of patch i at node k.
template <typename R>
__global__ void __launch_bounds__(512) l2p_kernel(int Kstar, const int64_t* __restrict__ pg_off,
                                                  const int* __restrict__ pg, const double* __restrict__ gcen,
                                                  const double* __restrict__ gR, const int* __restrict__ gshape,
                                                  const int64_t* __restrict__ goff, const int* __restrict__ shape_nr,
                                                  const int* __restrict__ shape_nth, const double* __restrict__ coef,
                                                  const double* __restrict__ centres, const double* __restrict__ zloc,
                                                  double* __restrict__ z) {
  extern __shared__ unsigned char lp_smem[];
  R* C = reinterpret_cast<R*>(lp_smem);
  const int64_t i = blockIdx.x;
  const int k = threadIdx.x;
  const double cx = centres[3 * i], cy = centres[3 * i + 1], cz = centres[3 * i + 2];
  double e1[3], e2[3], zo[3] = {0.0, 0.0, 0.0};
  patch_frame(cx, cy, cz, e1, e2);
  if (k < Kstar) frame_apply(e1, e2, cx, cy, cz, zloc[3 * k], zloc[3 * k + 1], zloc[3 * k + 2], zo);
  double acc = 0.0;
  for (int64_t s = pg_off[i]; s < pg_off[i + 1]; ++s) {
    const int g = pg[s];
    const int sh = gshape[g];
    const int nr = shape_nr[sh], nth = shape_nth[sh], q = nr * nth;
    const int64_t off = goff[g];
    __syncthreads();
    for (int t = threadIdx.x; t < q; t += blockDim.x) C[t] = (R)coef[off + t];
    __syncthreads();
    if (k >= Kstar) continue;
    const double* gc = gcen + 3 * g;
    double rho, ct, st;
    group_polar((cx - gc[0]) + zo[0], (cy - gc[1]) + zo[1], (cz - gc[2]) + zo[2], gc, gR[g], &rho, &ct, &st);
    acc += (double)eval_expansion<R>(C, nr, nth / 2, (R)rho, (R)ct, (R)st);
  }
  if (k < Kstar) z[i * Kstar + k] += acc;
}

// Downward pass: grid values of each linked child group += the parent group's
// expansion at the child's grid points (one block per link; a child has one link).
template <typename R>
__global__ void __launch_bounds__(256) l2l_kernel(int l0, const int* __restrict__ l2l_child,
                                                  const int* __restrict__ l2l_parent, const double* __restrict__ gcen,
                                                  const double* __restrict__ gR, const int* __restrict__ gshape,
                                                  const int64_t* __restrict__ goff, const int* __restrict__ shape_nr,
                                                  const int* __restrict__ shape_nth, const double* __restrict__ coef,
                                                  const double* __restrict__ gpos, double* __restrict__ grid) {
  extern __shared__ unsigned char ll_smem[];
  R* C = reinterpret_cast<R*>(ll_smem);
  const int ch = l2l_child[l0 + blockIdx.x], pa = l2l_parent[l0 + blockIdx.x];
  const int shp = gshape[pa], shc = gshape[ch];
  const int nrp = shape_nr[shp], nthp = shape_nth[shp], qp = nrp * nthp;
  const int qc = shape_nr[shc] * shape_nth[shc];
  const int64_t offp = goff[pa], offc = goff[ch];
  for (int t = threadIdx.x; t < qp; t += blockDim.x) C[t] = (R)coef[offp + t];
  __syncthreads();
  const double* gp = gcen + 3 * pa;
  const double* gq = gcen + 3 * ch;
  const double Dx = gq[0] - gp[0], Dy = gq[1] - gp[1], Dz = gq[2] - gp[2];
  for (int a = threadIdx.x; a < qc; a += blockDim.x) {
    const double* o = gpos + 3 * (offc + a);
    double rho, ct, st;
    group_polar(Dx + o[0], Dy + o[1], Dz + o[2], gp, gR[pa], &rho, &ct, &st);
    grid[offc + a] += (double)eval_expansion<R>(C, nrp, nthp / 2, (R)rho, (R)ct, (R)st);
  }
}

// ---- FP32 L2P / L2L ----------------------------------------------------------------
// The FP32 product evaluates the expansions with polar coordinates formed in FP32: per
// (patch or child, group) threads 0..11 build the rotation M from the evaluation points'
// local frame into the group frame (uploaded per group) and the offset of their origin,
// and every point then needs 9 FMAs, a square root and an atan2 on the FP32 pipes. Each
// thread evaluates two points, so every coefficient load from shared memory serves both.

// Clenshaw as eval_expansion for NP points at once, the A and B coefficients of each
// (m, j) interleaved.
template <int NP>
__device__ __forceinline__ void eval_expansion_ab(const float2* C, int nr, int mh, const float* rho,
                                                  const float* ct, const float* st, float* out) {
  float y[NP], y2[NP], cm[NP], sm[NP], val[NP];
#pragma unroll
  for (int t = 0; t < NP; ++t) {
    y[t] = fmaf(2.0f * rho[t], rho[t], -1.0f);
    y2[t] = y[t] + y[t];
    cm[t] = 1.0f;
    sm[t] = 0.0f;
    val[t] = 0.0f;
  }
  for (int m = 0; m < mh; ++m) {
    const float2* c = C + m * nr;
    float ba1[NP], ba2[NP], bb1[NP], bb2[NP];
#pragma unroll
    for (int t = 0; t < NP; ++t) ba1[t] = ba2[t] = bb1[t] = bb2[t] = 0.0f;
    for (int j = nr - 1; j >= 0; --j) {
      const float2 ab = c[j];
#pragma unroll
      for (int t = 0; t < NP; ++t) {
        const float ta = fmaf(y2[t], ba1[t], ab.x - ba2[t]);
        const float tb = fmaf(y2[t], bb1[t], ab.y - bb2[t]);
        ba2[t] = ba1[t];
        ba1[t] = ta;
        bb2[t] = bb1[t];
        bb1[t] = tb;
      }
    }
#pragma unroll
    for (int t = 0; t < NP; ++t) {
      float sa, sb;
      if ((m & 1) == 0) {
        sa = fmaf(-y[t], ba2[t], ba1[t]);
        sb = fmaf(-y[t], bb2[t], bb1[t]);
      } else {
        sa = rho[t] * (ba1[t] - ba2[t]);
        sb = rho[t] * (bb1[t] - bb2[t]);
      }
      val[t] = fmaf(cm[t], sa, fmaf(sm[t], sb, val[t]));
      const float cn = cm[t] * ct[t] - sm[t] * st[t];
      sm[t] = fmaf(sm[t], ct[t], cm[t] * st[t]);
      cm[t] = cn;
    }
  }
#pragma unroll
  for (int t = 0; t < NP; ++t) out[t] = val[t];
}

// Stages group coefficients (FP64, A block then B block) as interleaved FP32 pairs.
__device__ __forceinline__ void stage_ab(const double* __restrict__ coef, int nr, int mh, float2* C) {
  const int h = mh * nr;
  for (int t = threadIdx.x; t < h; t += blockDim.x) C[t] = make_float2((float)coef[t], (float)coef[h + t]);
}

// FP32 patch frame (same rule as patch_frame).
__device__ __forceinline__ void patch_frame32(float cx, float cy, float cz, float* e1, float* e2) {
  const float ax = -cy, ay = cx, na2 = fmaf(ax, ax, ay * ay);
  if (na2 >= 1e-24f) {
    const float inv = rsqrtf(na2);
    e1[0] = ax * inv;
    e1[1] = ay * inv;
  } else {
    e1[0] = 1.0f;
    e1[1] = 0.0f;
  }
  e1[2] = 0.0f;
  e2[0] = cy * e1[2] - cz * e1[1];
  e2[1] = cz * e1[0] - cx * e1[2];
  e2[2] = cx * e1[1] - cy * e1[0];
}

// Threads 0..11 fill M (caller synchronises): M[3r + c] = F_r . a_c for the group frame
// rows F_r and the local frame columns a_c, M[9 + r] = F_r . (o - g) for the local
// origin o and group centre g. Thread t < 9 passes in acol the column a_(t mod 3)
// (ignored when identity is set: the local frame is then the global one).
__device__ __forceinline__ void group_transform32(const float* __restrict__ F, const double* __restrict__ g,
                                                  const float* acol, bool identity, double ox, double oy,
                                                  double oz, float* M) {
  const int t = threadIdx.x;
  if (t < 9) {
    const int r = t / 3, c = t - 3 * (t / 3);
    const float* f = F + 3 * r;
    M[t] = identity ? f[c] : fmaf(f[0], acol[0], fmaf(f[1], acol[1], f[2] * acol[2]));
  } else if (t < 12) {
    const float* f = F + 3 * (t - 9);
    M[t] = fmaf(f[0], (float)(ox - g[0]), fmaf(f[1], (float)(oy - g[1]), f[2] * (float)(oz - g[2])));
  }
}

// Polar coordinates in the group frame of the local point v, given M from group_transform32.
__device__ __forceinline__ void polar32(const float* M, float v0, float v1, float v2, float invR, float* rho,
                                        float* ct, float* st) {
  const float u1 = fmaf(M[0], v0, fmaf(M[1], v1, fmaf(M[2], v2, M[9])));
  const float u2 = fmaf(M[3], v0, fmaf(M[4], v1, fmaf(M[5], v2, M[10])));
  const float u3 = fmaf(M[6], v0, fmaf(M[7], v1, fmaf(M[8], v2, M[11])));
  const float sr2 = fmaf(u1, u1, u2 * u2);
  if (sr2 > 0.0f) {
    const float ir = rsqrtf(sr2);
    const float sr = sr2 * ir;
    *rho = atan2f(sr, 1.0f + u3) * invR;
    *ct = u1 * ir;
    *st = u2 * ir;
  } else {
    *rho = 0.0f;
    *ct = 1.0f;
    *st = 0.0f;
  }
}

// L2P of the FP32 product: NCS_L2P_NP Zernike nodes per thread (K* <= 512)
#ifndef NCS_L2P_NP
#define NCS_L2P_NP 4
#endif
constexpr int L2P_NP = NCS_L2P_NP;
constexpr int L2P32_THREADS = 512 / L2P_NP;

// L2P, FP32 product: z_i(k) += expansion of every listed grid group of patch i at node k.
__global__ void __launch_bounds__(L2P32_THREADS) l2p_f32_kernel(
    int Kstar, const int64_t* __restrict__ pg_off, const int* __restrict__ pg, const double* __restrict__ gcen,
    const double* __restrict__ gR, const float* __restrict__ gframe, const int* __restrict__ gshape,
    const int64_t* __restrict__ goff, const int* __restrict__ shape_nr, const int* __restrict__ shape_nth,
    const double* __restrict__ coef, const double* __restrict__ centres, const double* __restrict__ zloc,
    double* __restrict__ z) {
  extern __shared__ unsigned char lp32_smem[];
  float2* C = reinterpret_cast<float2*>(lp32_smem);
  __shared__ float M[12];
  const int64_t i = blockIdx.x;
  int k[L2P_NP];
  float v[L2P_NP][3];
#pragma unroll
  for (int t = 0; t < L2P_NP; ++t) {
    k[t] = (int)threadIdx.x + t * L2P32_THREADS;
    for (int c = 0; c < 3; ++c) v[t][c] = (k[t] < Kstar) ? (float)zloc[3 * k[t] + c] : 0.0f;
  }
  const double cx = centres[3 * i], cy = centres[3 * i + 1], cz = centres[3 * i + 2];
  float acol[3] = {0.0f, 0.0f, 0.0f};  // column (threadIdx mod 3) of the patch frame (e1, e2, c)
  if (threadIdx.x < 9) {
    float e1[3], e2[3];
    patch_frame32((float)cx, (float)cy, (float)cz, e1, e2);
    const int c = threadIdx.x % 3;
    const float cc[3] = {(float)cx, (float)cy, (float)cz};
#pragma unroll
    for (int k = 0; k < 3; ++k) acol[k] = c == 0 ? e1[k] : (c == 1 ? e2[k] : cc[k]);
  }
  double acc[L2P_NP];
#pragma unroll
  for (int t = 0; t < L2P_NP; ++t) acc[t] = 0.0;
  for (int64_t s = pg_off[i]; s < pg_off[i + 1]; ++s) {
    const int g = pg[s];
    const int sh = gshape[g];
    const int nr = shape_nr[sh], mh = shape_nth[sh] / 2;
    __syncthreads();
    stage_ab(coef + goff[g], nr, mh, C);
    group_transform32(gframe + 9 * (size_t)g, gcen + 3 * g, acol, false, cx, cy, cz, M);
    __syncthreads();
    const float invR = (float)(1.0 / gR[g]);
    float rho[L2P_NP], ct[L2P_NP], st[L2P_NP], out[L2P_NP];
#pragma unroll
    for (int t = 0; t < L2P_NP; ++t) polar32(M, v[t][0], v[t][1], v[t][2], invR, &rho[t], &ct[t], &st[t]);
    eval_expansion_ab<L2P_NP>(C, nr, mh, rho, ct, st, out);
#pragma unroll
    for (int t = 0; t < L2P_NP; ++t) acc[t] += (double)out[t];
  }
#pragma unroll
  for (int t = 0; t < L2P_NP; ++t)
    if (k[t] < Kstar) z[i * Kstar + k[t]] += acc[t];
}

constexpr int L2L32_THREADS = 256;

// Downward pass, FP32 product: the child's grid points are given by their FP32 offsets
// from the child centre in the global frame (local frame = identity); two points per
// thread per round.
__global__ void __launch_bounds__(L2L32_THREADS) l2l_f32_kernel(
    int l0, const int* __restrict__ l2l_child, const int* __restrict__ l2l_parent, const double* __restrict__ gcen,
    const double* __restrict__ gR, const float* __restrict__ gframe, const int* __restrict__ gshape,
    const int64_t* __restrict__ goff, const int* __restrict__ shape_nr, const int* __restrict__ shape_nth,
    const double* __restrict__ coef, const float* __restrict__ gpos, double* __restrict__ grid) {
  extern __shared__ unsigned char ll32_smem[];
  float2* C = reinterpret_cast<float2*>(ll32_smem);
  __shared__ float M[12];
  const int ch = l2l_child[l0 + blockIdx.x], pa = l2l_parent[l0 + blockIdx.x];
  const int shp = gshape[pa], shc = gshape[ch];
  const int nrp = shape_nr[shp], mhp = shape_nth[shp] / 2;
  const int qc = shape_nr[shc] * shape_nth[shc];
  const int64_t offc = goff[ch];
  stage_ab(coef + goff[pa], nrp, mhp, C);
  const double* q = gcen + 3 * ch;
  group_transform32(gframe + 9 * (size_t)pa, gcen + 3 * pa, nullptr, true, q[0], q[1], q[2], M);
  __syncthreads();
  const float invR = (float)(1.0 / gR[pa]);
  for (int a0 = threadIdx.x; a0 < qc; a0 += 2 * L2L32_THREADS) {
    const int a[2] = {a0, a0 + L2L32_THREADS};
    float rho[2], ct[2], st[2], out[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int aa = a[t] < qc ? a[t] : a0;
      const float* o = gpos + 3 * (offc + aa);
      polar32(M, o[0], o[1], o[2], invR, &rho[t], &ct[t], &st[t]);
    }
    eval_expansion_ab<2>(C, nrp, mhp, rho, ct, st, out);
#pragma unroll
    for (int t = 0; t < 2; ++t)
      if (a[t] < qc) grid[offc + a[t]] += (double)out[t];
  }
}

// ---- float-float variants (FP64-accurate on the FP32 pipes) -----------------------
// Sources are staged as (hi, lo) float4 pairs formed from the FP64 offsets and
// strengths; tile sums are folded into an FP64 accumulator.
template <int MODE>
__global__ void __launch_bounds__(P2L_THREADS) p2l_df_kernel(
    const int* __restrict__ witem_group, const int* __restrict__ witem_rep, const int* __restrict__ rep_p,
    const int* __restrict__ rep_off, int pt, const int64_t* __restrict__ witem_lo, const int64_t* __restrict__ witem_hi,
    const int* __restrict__ isrc, const double* __restrict__ gcen, const int* __restrict__ gshape,
    const int64_t* __restrict__ goff, const int* __restrict__ shape_nr, const int* __restrict__ shape_nth,
    const double* __restrict__ gpos, const double* __restrict__ centres, const double* __restrict__ soff,
    const double* __restrict__ rho, const float4* __restrict__ logtab, double* __restrict__ grid) {
  extern __shared__ float4 p2d_smem[];
  __shared__ float4 tab[kLogTable];
  __shared__ double D[P2L_DF_JT][3];
  const int item = blockIdx.x;
  const int g = witem_group[item];
  const int rk = witem_rep[item];
  const int p = rep_p[rk], col = rep_off[rk];
  float4* Sh = p2d_smem;
  float4* Sl = p2d_smem + P2L_DF_JT * p;
  for (int t = threadIdx.x; t < kLogTable; t += blockDim.x) tab[t] = logtab[t];
  const int64_t lo = witem_lo[item], hi = witem_hi[item];
  const int sh = gshape[g];
  const int q = shape_nr[sh] * shape_nth[sh];
  const int64_t off = goff[g];
  const double gx = gcen[3 * g], gy = gcen[3 * g + 1], gz = gcen[3 * g + 2];
  // one grid for the high words of every offset of the item (targets and sources), so
  // that the pair loop subtracts them exactly (f2_split_grid)
  __shared__ unsigned long long gbits[3];
  __shared__ double qs[6];  // grid spacing per coordinate, then its inverse
  {
    const double gc[3] = {gx, gy, gz};
    double m[3] = {0.0, 0.0, 0.0};
    for (int ap = threadIdx.x; ap < q; ap += P2L_THREADS)
      for (int c = 0; c < 3; ++c) m[c] = fmax(m[c], fabs(gpos[3 * (off + ap) + c]));
    const int64_t npts = (hi - lo) * p;
    for (int64_t idx = threadIdx.x; idx < npts; idx += P2L_THREADS) {
      const int64_t jj = idx / p;
      const int j = isrc[lo + jj];
      const int64_t gs = (int64_t)j * pt + col + (idx - jj * p);
      for (int c = 0; c < 3; ++c) m[c] = fmax(m[c], fabs((centres[3 * j + c] - gc[c]) + soff[3 * gs + c]));
    }
    block_grid(m, gbits, qs);
  }
  constexpr int NT = 2;
  for (int base = 0; base < q; base += P2L_THREADS * NT) {
    f2 a[NT][3];
    double acc[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int ap = base + t * P2L_THREADS + threadIdx.x;
      for (int c = 0; c < 3; ++c) a[t][c] = f2_split_grid(ap < q ? gpos[3 * (off + ap) + c] : 0.0, qs[c], qs[3 + c]);
      acc[t] = 0.0;
    }
    for (int64_t s0 = lo; s0 < hi; s0 += P2L_DF_JT) {
      const int nj = (int)min((int64_t)P2L_DF_JT, hi - s0);
      __syncthreads();
      if (threadIdx.x < nj * 3) {
        const int jj = threadIdx.x / 3, c = threadIdx.x - 3 * jj;
        D[jj][c] = centres[3 * isrc[s0 + jj] + c] - (c == 0 ? gx : (c == 1 ? gy : gz));
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < nj * p; idx += P2L_THREADS) {
        const int jj = idx / p;
        const int64_t gs = (int64_t)isrc[s0 + jj] * pt + col + (idx - jj * p);
        const f2 x = f2_split_grid(D[jj][0] + soff[3 * gs], qs[0], qs[3]),
                 y = f2_split_grid(D[jj][1] + soff[3 * gs + 1], qs[1], qs[4]),
                 z = f2_split_grid(D[jj][2] + soff[3 * gs + 2], qs[2], qs[5]), r = f2_from_double(rho[gs]);
        Sh[idx] = make_float4(x.hi, y.hi, z.hi, r.hi);
        Sl[idx] = make_float4(x.lo, y.lo, z.lo, r.lo);
      }
      __syncthreads();
      const int ns = nj * p;
      f2 part[NT];
#pragma unroll
      for (int t = 0; t < NT; ++t) part[t] = f2{0.0f, 0.0f};
      const int wbase = base + (threadIdx.x & ~31);
      const int nact = (wbase >= q) ? 0 : ((wbase + P2L_THREADS >= q) ? 1 : NT);
      if (nact == NT) {
        // both targets in one packed float-float chain
        f2x2 A[3], P{x2_splat(0.0f), x2_splat(0.0f)};
#pragma unroll
        for (int c = 0; c < 3; ++c) A[c] = f2x2{x2_pack(a[0][c].hi, a[1][c].hi), x2_pack(a[0][c].lo, a[1][c].lo)};
        for (int s = 0; s < ns; ++s) pair_f2_acc_x2<MODE, true>(A, Sh[s], Sl[s], tab, P);
        x2_unpack(P.hi, part[0].hi, part[1].hi);
        x2_unpack(P.lo, part[0].lo, part[1].lo);
      } else if (nact == 1) {
        for (int s = 0; s < ns; ++s) pair_f2_acc<MODE>(a[0], Sh[s], Sl[s], tab, part[0]);
      }
#pragma unroll
      for (int t = 0; t < NT; ++t) acc[t] += f2_to_double(part[t]);
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int ap = base + t * P2L_THREADS + threadIdx.x;
      if (ap < q) atomicAdd(&grid[off + ap], acc[t]);
    }
  }
}

template <int MODE>
__global__ void __launch_bounds__(DTD_THREADS) direct_list_df_kernel(
    int pt, int Kstar, const int* __restrict__ rep_p, const int* __restrict__ rep_off,
    const int64_t* __restrict__ pd_off, const int* __restrict__ pd, const int* __restrict__ pdk,
    const double* __restrict__ centres, const double* __restrict__ zloc, const double* __restrict__ soff,
    const double* __restrict__ rho, const float4* __restrict__ logtab, int pmax, double* __restrict__ z) {
  extern __shared__ float4 dtd_smem[];
  __shared__ float4 tab[kLogTable];
  __shared__ double D[DT_JT][3];
  __shared__ int toff[DT_JT + 1], tcol[DT_JT];
  float4* Sh = dtd_smem;
  float4* Sl = dtd_smem + DT_JT * pmax;
  for (int t = threadIdx.x; t < kLogTable; t += blockDim.x) tab[t] = logtab[t];
  const int64_t i = blockIdx.x;
  const double cx = centres[3 * i], cy = centres[3 * i + 1], cz = centres[3 * i + 2];
  double e1[3], e2[3];
  patch_frame(cx, cy, cz, e1, e2);
  f2 a[DTD_NT][3];
  double acc[DTD_NT];
  int kk[DTD_NT];
  double gq[DTD_NT][3];
  double m[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int t = 0; t < DTD_NT; ++t) {
    kk[t] = (blockIdx.y * DTD_NT + t) * DTD_THREADS + threadIdx.x;
    for (int c = 0; c < 3; ++c) gq[t][c] = 0.0;
    if (kk[t] < Kstar)
      frame_apply(e1, e2, cx, cy, cz, zloc[3 * kk[t]], zloc[3 * kk[t] + 1], zloc[3 * kk[t] + 2], gq[t]);
    for (int c = 0; c < 3; ++c) m[c] = fmax(m[c], fabs(gq[t][c]));
    acc[t] = 0.0;
  }
  const int64_t lo = pd_off[i], hi = pd_off[i + 1];
  // one grid for the high words of the block's offsets (its nodes and every listed
  // source), so that the pair loop subtracts them exactly (f2_split_grid)
  __shared__ unsigned long long gbits[3];
  __shared__ double qs[6];  // grid spacing per coordinate, then its inverse
  {
    for (int64_t s0 = lo; s0 < hi; ++s0) {
      const int64_t j = pd[s0];
      const int k = pdk[s0];
      const int pk = rep_p[k];
      for (int mm = threadIdx.x; mm < pk; mm += DTD_THREADS) {
        const int64_t gs = j * pt + rep_off[k] + mm;
        for (int c = 0; c < 3; ++c) m[c] = fmax(m[c], fabs((centres[3 * j + c] - centres[3 * i + c]) + soff[3 * gs + c]));
      }
    }
    block_grid(m, gbits, qs);
  }
#pragma unroll
  for (int t = 0; t < DTD_NT; ++t)
    for (int c = 0; c < 3; ++c) a[t][c] = f2_split_grid(gq[t][c], qs[c], qs[3 + c]);
  for (int64_t s0 = lo; s0 < hi; s0 += DT_JT) {
    const int nj = (int)min((int64_t)DT_JT, hi - s0);
    __syncthreads();
    if (threadIdx.x < nj) {
      const int64_t j = pd[s0 + threadIdx.x];
      const int k = pdk[s0 + threadIdx.x];
      for (int c = 0; c < 3; ++c) D[threadIdx.x][c] = centres[3 * j + c] - centres[3 * i + c];
      toff[threadIdx.x + 1] = rep_p[k];
      tcol[threadIdx.x] = rep_off[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      toff[0] = 0;
      for (int jj = 0; jj < nj; ++jj) toff[jj + 1] += toff[jj];
    }
    __syncthreads();
    const int ns = toff[nj];
    for (int idx = threadIdx.x; idx < ns; idx += DTD_THREADS) {
      int jj = 0;
      while (idx >= toff[jj + 1]) ++jj;
      const int64_t gs = (int64_t)pd[s0 + jj] * pt + tcol[jj] + (idx - toff[jj]);
      const f2 x = f2_split_grid(D[jj][0] + soff[3 * gs], qs[0], qs[3]),
               y = f2_split_grid(D[jj][1] + soff[3 * gs + 1], qs[1], qs[4]),
               zz = f2_split_grid(D[jj][2] + soff[3 * gs + 2], qs[2], qs[5]), r = f2_from_double(rho[gs]);
      Sh[idx] = make_float4(x.hi, y.hi, zz.hi, r.hi);
      Sl[idx] = make_float4(x.lo, y.lo, zz.lo, r.lo);
    }
    __syncthreads();
    f2 part[DTD_NT];
#pragma unroll
    for (int t = 0; t < DTD_NT; ++t) part[t] = f2{0.0f, 0.0f};
    static_assert(DTD_NT == 2, "the packed float-float chain serves two targets");
    {
      f2x2 A[3], P{x2_splat(0.0f), x2_splat(0.0f)};
#pragma unroll
      for (int c = 0; c < 3; ++c) A[c] = f2x2{x2_pack(a[0][c].hi, a[1][c].hi), x2_pack(a[0][c].lo, a[1][c].lo)};
      for (int s = 0; s < ns; ++s) pair_f2_acc_x2<MODE, true>(A, Sh[s], Sl[s], tab, P);
      x2_unpack(P.hi, part[0].hi, part[1].hi);
      x2_unpack(P.lo, part[0].lo, part[1].lo);
    }
#pragma unroll
    for (int t = 0; t < DTD_NT; ++t) acc[t] += f2_to_double(part[t]);
  }
#pragma unroll
  for (int t = 0; t < DTD_NT; ++t)
    if (kk[t] < Kstar) z[i * Kstar + kk[t]] = acc[t];
}

// Float-float expansion value (same recurrences as eval_expansion).
__device__ __forceinline__ f2 eval_expansion_f2(const float2* C, int nr, int mh, f2 rho, f2 ct, f2 st) {
  const f2 y = f2_add(f2_mul(f2{2.0f * rho.hi, 2.0f * rho.lo}, rho), f2{-1.0f, 0.0f});
  const f2 y2 = f2{2.0f * y.hi, 2.0f * y.lo};
  f2 cm = {1.0f, 0.0f}, sm = {0.0f, 0.0f}, val = {0.0f, 0.0f};
  for (int m = 0; m < mh; ++m) {
    const float2* A = C + m * nr;
    const float2* B = C + mh * nr + m * nr;
    f2 ba1 = {0.f, 0.f}, ba2 = {0.f, 0.f}, bb1 = {0.f, 0.f}, bb2 = {0.f, 0.f};
    for (int j = nr - 1; j >= 0; --j) {
      const f2 ta = f2_add(f2_mul(y2, ba1), f2_sub(f2{A[j].x, A[j].y}, ba2));
      const f2 tb = f2_add(f2_mul(y2, bb1), f2_sub(f2{B[j].x, B[j].y}, bb2));
      ba2 = ba1;
      ba1 = ta;
      bb2 = bb1;
      bb1 = tb;
    }
    f2 sa, sb;
    if ((m & 1) == 0) {
      sa = f2_sub(ba1, f2_mul(y, ba2));
      sb = f2_sub(bb1, f2_mul(y, bb2));
    } else {
      sa = f2_mul(rho, f2_sub(ba1, ba2));
      sb = f2_mul(rho, f2_sub(bb1, bb2));
    }
    val = f2_add(val, f2_add(f2_mul(cm, sa), f2_mul(sm, sb)));
    const f2 cn = f2_sub(f2_mul(cm, ct), f2_mul(sm, st));
    sm = f2_add(f2_mul(sm, ct), f2_mul(cm, st));
    cm = cn;
  }
  return val;
}

// L2P in float-float: node position in the group's polar coordinates from FP64,
// coefficients as (hi, lo).
__global__ void __launch_bounds__(512) l2p_df_kernel(int Kstar, const int64_t* __restrict__ pg_off,
                                                     const int* __restrict__ pg, const double* __restrict__ gcen,
                                                     const double* __restrict__ gR, const int* __restrict__ gshape,
                                                     const int64_t* __restrict__ goff, const int* __restrict__ shape_nr,
                                                     const int* __restrict__ shape_nth, const double* __restrict__ coef,
                                                     const double* __restrict__ centres, const double* __restrict__ zloc,
                                                     double* __restrict__ z) {
  extern __shared__ float2 lpd_smem[];
  const int64_t i = blockIdx.x;
  const int k = threadIdx.x;
  const double cx = centres[3 * i], cy = centres[3 * i + 1], cz = centres[3 * i + 2];
  double e1[3], e2[3], zo[3] = {0.0, 0.0, 0.0};
  patch_frame(cx, cy, cz, e1, e2);
  if (k < Kstar) frame_apply(e1, e2, cx, cy, cz, zloc[3 * k], zloc[3 * k + 1], zloc[3 * k + 2], zo);
  double acc = 0.0;
  for (int64_t s = pg_off[i]; s < pg_off[i + 1]; ++s) {
    const int g = pg[s];
    const int sh = gshape[g];
    const int nr = shape_nr[sh], nth = shape_nth[sh], q = nr * nth;
    const int64_t off = goff[g];
    __syncthreads();
    for (int t = threadIdx.x; t < q; t += blockDim.x) {
      const f2 v = f2_from_double(coef[off + t]);
      lpd_smem[t] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
    if (k >= Kstar) continue;
    const double* gc = gcen + 3 * g;
    double rho, ct, st;
    group_polar((cx - gc[0]) + zo[0], (cy - gc[1]) + zo[1], (cz - gc[2]) + zo[2], gc, gR[g], &rho, &ct, &st);
    acc += f2_to_double(eval_expansion_f2(lpd_smem, nr, nth / 2, f2_from_double(rho), f2_from_double(ct),
                                          f2_from_double(st)));
  }
  if (k < Kstar) z[i * Kstar + k] += acc;
}

__global__ void __launch_bounds__(256) l2l_df_kernel(int l0, const int* __restrict__ l2l_child,
                                                     const int* __restrict__ l2l_parent, const double* __restrict__ gcen,
                                                     const double* __restrict__ gR, const int* __restrict__ gshape,
                                                     const int64_t* __restrict__ goff, const int* __restrict__ shape_nr,
                                                     const int* __restrict__ shape_nth, const double* __restrict__ coef,
                                                     const double* __restrict__ gpos, double* __restrict__ grid) {
  extern __shared__ float2 lld_smem[];
  const int ch = l2l_child[l0 + blockIdx.x], pa = l2l_parent[l0 + blockIdx.x];
  const int shp = gshape[pa], shc = gshape[ch];
  const int nrp = shape_nr[shp], nthp = shape_nth[shp], qp = nrp * nthp;
  const int qc = shape_nr[shc] * shape_nth[shc];
  const int64_t offp = goff[pa], offc = goff[ch];
  for (int t = threadIdx.x; t < qp; t += blockDim.x) {
    const f2 v = f2_from_double(coef[offp + t]);
    lld_smem[t] = make_float2(v.hi, v.lo);
  }
  __syncthreads();
  const double* gp = gcen + 3 * pa;
  const double* gq = gcen + 3 * ch;
  const double Dx = gq[0] - gp[0], Dy = gq[1] - gp[1], Dz = gq[2] - gp[2];
  for (int a = threadIdx.x; a < qc; a += blockDim.x) {
    const double* o = gpos + 3 * (offc + a);
    double rho, ct, st;
    group_polar(Dx + o[0], Dy + o[1], Dz + o[2], gp, gR[pa], &rho, &ct, &st);
    grid[offc + a] += f2_to_double(eval_expansion_f2(lld_smem, nrp, nthp / 2, f2_from_double(rho),
                                                     f2_from_double(ct), f2_from_double(st)));
  }
}

}  // namespace

void tree_upload(const TreeHost& t, const Precomputed& pc, TreeDevice& d) {
  tree_free(d);
  (void)pc;
  d.ngroups = (int)t.gR.size();
  d.nitems = (int)t.witem_group.size();
  d.nshapes = (int)t.shapes.size();
  d.ngrid = t.total_grid_points;
  d.N = (int64_t)t.pd_off.size() - 1;
  std::vector<int> snr(d.nshapes), snth(d.nshapes);
  d.max_q = d.max_nr = d.max_nth = 0;
  for (int s = 0; s < d.nshapes; ++s) {
    snr[s] = t.shapes[s].nr;
    snth[s] = t.shapes[s].nth;
    d.max_q = std::max(d.max_q, t.shapes[s].q());
    d.max_nr = std::max(d.max_nr, snr[s]);
    d.max_nth = std::max(d.max_nth, snth[s]);
  }
  // grid-point offsets from the group centre in the global frame (FP64 and FP32)
  std::vector<double> gp64(3 * (size_t)d.ngrid);
  std::vector<float> gf(9 * (size_t)d.ngroups);
  for (int g = 0; g < d.ngroups; ++g) {
    const GridShape& s = t.shapes[t.gshape[g]];
    const double* c = &t.gcen[3 * g];
    double e1[3], e2[3];
    const double ax = -c[1], ay = c[0], na2 = ax * ax + ay * ay;
    if (na2 >= 1e-24) {
      const double inv = 1.0 / std::sqrt(na2);
      e1[0] = ax * inv;
      e1[1] = ay * inv;
      e1[2] = 0.0;
    } else {
      e1[0] = 1.0;
      e1[1] = 0.0;
      e1[2] = 0.0;
    }
    e2[0] = c[1] * e1[2] - c[2] * e1[1];
    e2[1] = c[2] * e1[0] - c[0] * e1[2];
    e2[2] = c[0] * e1[1] - c[1] * e1[0];
    for (int k = 0; k < 3; ++k) {
      gf[9 * (size_t)g + k] = (float)e1[k];
      gf[9 * (size_t)g + 3 + k] = (float)e2[k];
      gf[9 * (size_t)g + 6 + k] = (float)c[k];
    }
    for (int a = 0; a < s.nr; ++a) {
      const double r = t.gR[g] * std::cos((2.0 * a + 1.0) * kPi / (4.0 * s.nr));
      for (int b = 0; b < s.nth; ++b) {
        const double th = 2.0 * kPi * b / s.nth;
        double o[3];
        local_offset(r, th, o);
        const size_t idx = (size_t)t.goff[g] + (size_t)a * s.nth + b;
        for (int k = 0; k < 3; ++k) gp64[3 * idx + k] = o[0] * e1[k] + o[1] * e2[k] + o[2] * c[k];
      }
    }
  }
  std::vector<float> gp32(gp64.begin(), gp64.end());
  auto chk = [](cudaError_t e) {
    if (e != cudaSuccess) throw std::runtime_error(std::string("tree upload: ") + cudaGetErrorString(e));
  };
  chk(up(&d.gcen, t.gcen));
  chk(up(&d.gR, t.gR));
  chk(up(&d.gshape, t.gshape));
  chk(up(&d.goff, t.goff));
  chk(up(&d.shape_nr, snr));
  chk(up(&d.shape_nth, snth));
  chk(up(&d.witem_group, t.witem_group));
  chk(up(&d.witem_rep, t.witem_rep));
  chk(up(&d.witem_lo, t.witem_lo));
  chk(up(&d.witem_hi, t.witem_hi));
  chk(up(&d.isrc, t.isrc));
  chk(up(&d.pg_off, t.pg_off));
  chk(up(&d.pg, t.pg));
  chk(up(&d.pd_off, t.pd_off));
  chk(up(&d.pd, t.pd));
  chk(up(&d.pdk, t.pdk));
  chk(up(&d.gpos64, gp64));
  chk(up(&d.l2l_child, t.l2l_child));
  chk(up(&d.l2l_parent, t.l2l_parent));
  d.gl_off = t.gl_off;
  d.l2l_off = t.l2l_off;
  chk(up(&d.gpos32, gp32));
  chk(up(&d.gframe, gf));
  chk(cudaMalloc(&d.grid, std::max<int64_t>(1, d.ngrid) * sizeof(double)));
  chk(cudaMalloc(&d.coef, std::max<int64_t>(1, d.ngrid) * sizeof(double)));
}

void tree_free(TreeDevice& d) {
  fr(d.gcen);
  fr(d.gR);
  fr(d.gshape);
  fr(d.goff);
  fr(d.shape_nr);
  fr(d.shape_nth);
  fr(d.witem_group);
  fr(d.witem_rep);
  fr(d.witem_lo);
  fr(d.witem_hi);
  fr(d.isrc);
  fr(d.pg_off);
  fr(d.pg);
  fr(d.pd_off);
  fr(d.pd);
  fr(d.pdk);
  fr(d.gpos64);
  fr(d.l2l_child);
  fr(d.l2l_parent);
  d.gl_off.clear();
  d.l2l_off.clear();
  fr(d.gpos32);
  fr(d.gframe);
  fr(d.grid);
  fr(d.coef);
  d.ngroups = d.nitems = 0;
  d.ngrid = 0;
}

template <typename K>
static cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Top-down over levels: coefficients of the level's grid groups (their grids now hold
// their own P2L sums plus everything passed down), then the grid-to-grid transfer into
// the nearest grid descendants whose parent is at this level.
template <typename R>
static cudaError_t downward(const TreeDevice& t, cudaStream_t s) {
  cudaError_t e;
  using CR = typename std::conditional<std::is_same<R, f2>::value, double, R>::type;
  const size_t csm = (size_t)t.max_q * sizeof(double) + (size_t)t.max_nth * t.max_nr * sizeof(double) +
                     (2 * (size_t)t.max_nth + 2 * (size_t)t.max_nr * t.max_nr) * sizeof(CR);
  if ((e = allow_smem(coef_kernel<CR>, csm)) != cudaSuccess) return e;
  const int nl = (int)t.gl_off.size() - 1;
  for (int l = 0; l < nl; ++l) {
    const int g0 = t.gl_off[l], ng = t.gl_off[l + 1] - g0;
    if (ng > 0) {
      count_launch(), coef_kernel<CR><<<ng, 256, csm, s>>>(g0, t.gshape, t.goff, t.shape_nr, t.shape_nth, t.grid, t.coef);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int l0 = t.l2l_off[l], nlk = t.l2l_off[l + 1] - l0;
    if (nlk > 0) {
      if constexpr (std::is_same<R, f2>::value) {
        const size_t sm = (size_t)t.max_q * sizeof(float2);
        if ((e = allow_smem(l2l_df_kernel, sm)) != cudaSuccess) return e;
        count_launch(), l2l_df_kernel<<<nlk, 256, sm, s>>>(l0, t.l2l_child, t.l2l_parent, t.gcen, t.gR, t.gshape, t.goff, t.shape_nr,
                                           t.shape_nth, t.coef, t.gpos64, t.grid);
      } else if constexpr (std::is_same<R, float>::value) {
        const size_t sm = (size_t)t.max_q * sizeof(float);
        if ((e = allow_smem(l2l_f32_kernel, sm)) != cudaSuccess) return e;
        count_launch(), l2l_f32_kernel<<<nlk, L2L32_THREADS, sm, s>>>(l0, t.l2l_child, t.l2l_parent, t.gcen, t.gR,
                                                                      t.gframe, t.gshape, t.goff, t.shape_nr,
                                                                      t.shape_nth, t.coef, t.gpos32, t.grid);
      } else {
        const size_t sm = (size_t)t.max_q * sizeof(R);
        if ((e = allow_smem(l2l_kernel<R>, sm)) != cudaSuccess) return e;
        count_launch(), l2l_kernel<R><<<nlk, 256, sm, s>>>(l0, t.l2l_child, t.l2l_parent, t.gcen, t.gR, t.gshape, t.goff,
                                           t.shape_nr, t.shape_nth, t.coef, t.gpos64, t.grid);
      }
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// The FP32 pair kernels' run-time variants (KernelConfig): source patches per P2L tile
// and the share of logarithms taken on the FMA pipe. Every variant has the same
// parameters, so one pointer type serves them all.
template <int MODE, int JT, int POLY>
static auto p2l32_variant_rsq(int rsq) -> decltype(&p2l_kernel<float, MODE, JT, POLY, 0>) {
  switch (rsq) {
    case 0: return &p2l_kernel<float, MODE, JT, POLY, 0>;
    case 4: return &p2l_kernel<float, MODE, JT, POLY, 4>;
    case 8: return &p2l_kernel<float, MODE, JT, POLY, 8>;
    default: return nullptr;
  }
}

template <int MODE, int JT>
static auto p2l32_variant(int poly, int rsq) -> decltype(&p2l_kernel<float, MODE, JT, 0, 0>) {
  switch (poly) {
    case 0: return p2l32_variant_rsq<MODE, JT, 0>(rsq);
    case 2: return p2l32_variant_rsq<MODE, JT, 2>(rsq);
    case 4: return p2l32_variant_rsq<MODE, JT, 4>(rsq);
    case 6: return p2l32_variant_rsq<MODE, JT, 6>(rsq);
    default: return nullptr;
  }
}

template <int MODE>
static auto p2l32_variant(int jt, int poly, int rsq) -> decltype(&p2l_kernel<float, MODE, 16, 0, 0>) {
  if (jt == 8) return p2l32_variant<MODE, 8>(poly, rsq);
  if (jt == 16) return p2l32_variant<MODE, 16>(poly, rsq);
  return nullptr;
}

template <int MODE, int POLY>
static auto direct32_variant_rsq(int rsq) -> decltype(&direct_list_kernel<float, MODE, POLY, 0>) {
  switch (rsq) {
    case 0: return &direct_list_kernel<float, MODE, POLY, 0>;
    case 4: return &direct_list_kernel<float, MODE, POLY, 4>;
    case 8: return &direct_list_kernel<float, MODE, POLY, 8>;
    default: return nullptr;
  }
}

template <int MODE>
static auto direct32_variant(int poly, int rsq) -> decltype(&direct_list_kernel<float, MODE, 0, 0>) {
  switch (poly) {
    case 0: return direct32_variant_rsq<MODE, 0>(rsq);
    case 2: return direct32_variant_rsq<MODE, 2>(rsq);
    case 4: return direct32_variant_rsq<MODE, 4>(rsq);
    case 6: return direct32_variant_rsq<MODE, 6>(rsq);
    default: return nullptr;
  }
}

bool kernel_config_valid(const KernelConfig& k) {
  const auto poly_ok = [](int p) { return p == 0 || p == 2 || p == 4 || p == 6; };
  const auto rsq_ok = [](int r) { return r == 0 || r == 4 || r == 8; };
  return (k.p2l_tile == 8 || k.p2l_tile == 16) && poly_ok(k.p2l_poly) && poly_ok(k.direct_poly) &&
         rsq_ok(k.p2l_rsq) && rsq_ok(k.direct_rsq);
}

template <typename R, int MODE>
static cudaError_t tree_field_impl(const DeviceData& dd, const TreeDevice& t, cudaStream_t s, cudaEvent_t* ev) {
  const R* soff = (sizeof(R) == 8) ? (const R*)dd.soff64 : (const R*)dd.soff32;
  const R* rho = (sizeof(R) == 8) ? (const R*)dd.rho64 : (const R*)dd.rho32;
  const R* gpos = (sizeof(R) == 8) ? (const R*)t.gpos64 : (const R*)t.gpos32;
  using V4 = typename V4T<R>::type;
  cudaError_t e;
  if (ev) cudaEventRecord(ev[0], s);
  if (t.nitems > 0) {
    e = cudaMemsetAsync(t.grid, 0, t.ngrid * sizeof(double), s);
    if (e != cudaSuccess) return e;
    auto kern = &p2l_kernel<R, MODE>;
    int jt = P2L_JT;
    if constexpr (std::is_same<R, float>::value) {
      kern = p2l32_variant<MODE>(t.cfg.p2l_tile, t.cfg.p2l_poly, t.cfg.p2l_rsq);
      jt = t.cfg.p2l_tile;
      if (!kern) return cudaErrorInvalidValue;
    }
    const size_t smem = (size_t)jt * dd.pmax * sizeof(V4);
    if ((e = allow_smem(kern, smem)) != cudaSuccess) return e;
    count_launch(), kern<<<t.nitems, P2L_THREADS, smem, s>>>(t.witem_group, t.witem_rep, dd.rep_p, dd.rep_off, dd.p,
                                                             t.witem_lo, t.witem_hi, t.isrc, t.gcen, t.gshape, t.goff,
                                                             t.shape_nr, t.shape_nth, gpos, dd.centres, soff, rho,
                                                             t.grid);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], s);
    if ((e = downward<R>(t, s)) != cudaSuccess) return e;
  } else if (ev) {
    cudaEventRecord(ev[1], s);
  }
  if (ev) cudaEventRecord(ev[2], s);
  {
    auto kern = &direct_list_kernel<R, MODE>;
    if constexpr (std::is_same<R, float>::value) {
      kern = direct32_variant<MODE>(t.cfg.direct_poly, t.cfg.direct_rsq);
      if (!kern) return cudaErrorInvalidValue;
    }
    const size_t smem = (size_t)DT_JT * dd.pmax * sizeof(V4);
    if ((e = allow_smem(kern, smem)) != cudaSuccess) return e;
    dim3 grid((unsigned)dd.N, (unsigned)((dd.Kstar + DT_THREADS * DT_NT - 1) / (DT_THREADS * DT_NT)));
    count_launch(), kern<<<grid, DT_THREADS, smem, s>>>(dd.p, dd.Kstar, dd.pmax, dd.rep_p, dd.rep_off, t.pd_off, t.pd,
                                                                t.pdk, dd.centres, dd.zloc, soff, rho, dd.z);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (ev) cudaEventRecord(ev[3], s);
  if (t.nitems > 0) {
    if (dd.Kstar > 512) return cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)t.max_q * sizeof(R);
    if constexpr (std::is_same<R, float>::value) {
      if ((e = allow_smem(l2p_f32_kernel, smem)) != cudaSuccess) return e;
      count_launch(), l2p_f32_kernel<<<(unsigned)dd.N, L2P32_THREADS, smem, s>>>(
          dd.Kstar, t.pg_off, t.pg, t.gcen, t.gR, t.gframe, t.gshape, t.goff, t.shape_nr, t.shape_nth, t.coef,
          dd.centres, dd.zloc, dd.z);
    } else {
      if ((e = allow_smem(l2p_kernel<R>, smem)) != cudaSuccess) return e;
      count_launch(), l2p_kernel<R><<<(unsigned)dd.N, 512, smem, s>>>(dd.Kstar, t.pg_off, t.pg, t.gcen, t.gR, t.gshape,
                                                                     t.goff, t.shape_nr, t.shape_nth, t.coef,
                                                                     dd.centres, dd.zloc, dd.z);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (ev) cudaEventRecord(ev[4], s);
  return cudaSuccess;
}

template <int MODE>
static cudaError_t tree_field_df(const DeviceData& dd, const TreeDevice& t, cudaStream_t s, cudaEvent_t* ev) {
  cudaError_t e;
  if (ev) cudaEventRecord(ev[0], s);
  if (t.nitems > 0) {
    if ((e = cudaMemsetAsync(t.grid, 0, t.ngrid * sizeof(double), s)) != cudaSuccess) return e;
    const size_t smem = (size_t)2 * P2L_DF_JT * dd.pmax * sizeof(float4);
    if ((e = allow_smem(p2l_df_kernel<MODE>, smem)) != cudaSuccess) return e;
    count_launch(), p2l_df_kernel<MODE><<<t.nitems, P2L_THREADS, smem, s>>>(t.witem_group, t.witem_rep, dd.rep_p, dd.rep_off, dd.p,
                                                           t.witem_lo, t.witem_hi, t.isrc, t.gcen, t.gshape, t.goff,
                                                           t.shape_nr, t.shape_nth, t.gpos64, dd.centres, dd.soff64,
                                                           dd.rho64, dd.logtab, t.grid);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], s);
    if ((e = downward<f2>(t, s)) != cudaSuccess) return e;
  } else if (ev) {
    cudaEventRecord(ev[1], s);
  }
  if (ev) cudaEventRecord(ev[2], s);
  {
    const size_t smem = (size_t)2 * DT_JT * dd.pmax * sizeof(float4);
    if ((e = allow_smem(direct_list_df_kernel<MODE>, smem)) != cudaSuccess) return e;
    dim3 grid((unsigned)dd.N, (unsigned)((dd.Kstar + DTD_THREADS * DTD_NT - 1) / (DTD_THREADS * DTD_NT)));
    count_launch(), direct_list_df_kernel<MODE><<<grid, DTD_THREADS, smem, s>>>(dd.p, dd.Kstar, dd.rep_p, dd.rep_off, t.pd_off, t.pd,
                                                              t.pdk, dd.centres, dd.zloc, dd.soff64, dd.rho64,
                                                              dd.logtab, dd.pmax, dd.z);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (ev) cudaEventRecord(ev[3], s);
  if (t.nitems > 0) {
    if (dd.Kstar > 512) return cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)t.max_q * sizeof(float2);
    if ((e = allow_smem(l2p_df_kernel, smem)) != cudaSuccess) return e;
    count_launch(), l2p_df_kernel<<<(unsigned)dd.N, 512, smem, s>>>(dd.Kstar, t.pg_off, t.pg, t.gcen, t.gR, t.gshape, t.goff,
                                                   t.shape_nr, t.shape_nth, t.coef, dd.centres, dd.zloc, dd.z);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (ev) cudaEventRecord(ev[4], s);
  return cudaSuccess;
}

cudaError_t launch_tree_field(const DeviceData& d, const TreeDevice& t, int mode, int prec, cudaStream_t s,
                              cudaEvent_t* ev) {
  if (prec == NCS_DF64) return mode == 0 ? tree_field_df<0>(d, t, s, ev) : tree_field_df<1>(d, t, s, ev);
  if (prec == NCS_FP64)
    return mode == 0 ? tree_field_impl<double, 0>(d, t, s, ev) : tree_field_impl<double, 1>(d, t, s, ev);
  return mode == 0 ? tree_field_impl<float, 0>(d, t, s, ev) : tree_field_impl<float, 1>(d, t, s, ev);
}

}  // namespace ncs
