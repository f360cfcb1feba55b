// The one-patch interpolative decompositions on the device (see sketch.hpp):
//   * sketch_kernel: Y += Omega[:, r0:r1] A[r0:r1, :], A_tl = G(|x_t - x_l|) evaluated once
//     per entry in float-float (the pair kernels' green_f2) and the product accumulated in
//     float-float on the FP32 pipes (Omega holds FP32 values, so each product's error is
//     exact by TwoProd), folded into the FP64 sketch every 256 training rows; each block owns
//     all sketch rows (up to 256) of 32 fine points, stages 32 training rows of Omega and of
//     A per step in shared memory and accumulates 8 rows x 4 points per thread (for ID
//     tolerances below 1e-12, sketch64_kernel forms the same sums in FP64);
//   * column-pivoted Householder QR of the leading sketch rows in FP64, one pivot/reflector
//     block and one column-update kernel per step (a warp per column), the host reading
//     the stopping flag every 16 steps;
//   * X = R11^-1 R12 by one back-substitution per column, T = W B[skeleton] + X W B[rest]
//     in FP64.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "df64.cuh"
#include "internal.hpp"
#include "sketch.hpp"

namespace ncs {

// Status of the device CPQR, read by the host every few steps.
struct CpqrStatus {
  int done;    // the stopping rule fired
  int p;       // completed steps (the rank once done)
  double r00;  // |R_00|
  double vv;   // |v|^2 of the current Householder vector
};

namespace {

constexpr int SK_ROWS = 256;   // sketch rows per block
constexpr int SK_TL = 32;      // fine-grid points per block
constexpr int SK_TJ = 32;      // training rows per step
constexpr int SK_FLUSH = 8;    // steps between folds of the float-float sums into Y
constexpr int SK_THREADS = 256;

// acc += w (h + l) for two outputs (f32x2 halves) in float-float: w h by TwoProd (exact
// error through the FMA), the sum by TwoSum, the low-order terms gathered in acc_l; nw = -w.
__device__ __forceinline__ void ff_axpy_x2(f32x2& acc_h, f32x2& acc_l, f32x2 w, f32x2 nw, f32x2 h, f32x2 l) {
  const f32x2 ph = x2_mul(w, h);
  const f32x2 e1 = x2_fma(nw, h, ph);  // ph - w h, exact
  const f32x2 s = x2_add(acc_h, ph);
  const f32x2 bb = x2_sub(s, acc_h);
  const f32x2 e = x2_add(x2_sub(acc_h, x2_sub(s, bb)), x2_sub(ph, bb));
  acc_h = s;
  acc_l = x2_add(acc_l, x2_fma(w, l, x2_sub(e, e1)));
}

// Om: nt x ks FP32 (training row t's sketch coefficients contiguous); Y: ks x nf column-major
// FP64. Thread (ty, tx) owns sketch rows rb + 8 ty .. + 7 and fine points lb + 4 tx .. + 3.
template <int MODE>
__global__ void __launch_bounds__(SK_THREADS) sketch_kernel(int ks, int nf, const float* __restrict__ Om,
                                                            const double* __restrict__ xt,
                                                            const double* __restrict__ xf, int r0, int r1,
                                                            const float4* __restrict__ logtab,
                                                            double* __restrict__ Y) {
  __shared__ __align__(16) float Os[SK_TJ][SK_ROWS];
  __shared__ __align__(16) float Ah[SK_TJ][SK_TL];
  __shared__ __align__(16) float Al[SK_TJ][SK_TL];
  __shared__ float4 tab[kLogTable];
  for (int t = threadIdx.x; t < kLogTable; t += SK_THREADS) tab[t] = logtab[t];
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  const int rb = blockIdx.y * SK_ROWS, lb = blockIdx.x * SK_TL;
  f32x2 ah[8][2], al[8][2];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int c = 0; c < 2; ++c) ah[i][c] = al[i][c] = x2_splat(0.0f);
  int step = 0;
  for (int j0 = r0; j0 < r1; j0 += SK_TJ, ++step) {
    __syncthreads();
    for (int e = threadIdx.x; e < SK_TJ * SK_ROWS; e += SK_THREADS) {
      const int jj = e / SK_ROWS, rr = e - jj * SK_ROWS;
      const int t = j0 + jj, r = rb + rr;
      Os[jj][rr] = (t < r1 && r < ks) ? Om[(int64_t)t * ks + r] : 0.0f;
    }
    for (int e = threadIdx.x; e < SK_TJ * SK_TL; e += SK_THREADS) {
      const int jj = e / SK_TL, ll = e - jj * SK_TL;
      const int t = j0 + jj, l = lb + ll;
      f2 g{0.0f, 0.0f};
      if (t < r1 && l < nf) {
        const double dx = xt[3 * t] - xf[3 * l], dy = xt[3 * t + 1] - xf[3 * l + 1], dz = xt[3 * t + 2] - xf[3 * l + 2];
        g = green_f2<MODE>(f2_from_double(fma(dx, dx, fma(dy, dy, dz * dz))), tab);
      }
      Ah[jj][ll] = g.hi;
      Al[jj][ll] = g.lo;
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < SK_TJ; ++jj) {
      const float4 w0 = *reinterpret_cast<const float4*>(&Os[jj][8 * ty]);
      const float4 w1 = *reinterpret_cast<const float4*>(&Os[jj][8 * ty + 4]);
      const float4 h = *reinterpret_cast<const float4*>(&Ah[jj][4 * tx]);
      const float4 lo = *reinterpret_cast<const float4*>(&Al[jj][4 * tx]);
      const f32x2 H[2] = {x2_pack(h.x, h.y), x2_pack(h.z, h.w)};
      const f32x2 L[2] = {x2_pack(lo.x, lo.y), x2_pack(lo.z, lo.w)};
      const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const f32x2 W = x2_splat(w[i]), NW = x2_splat(-w[i]);
#pragma unroll
        for (int c = 0; c < 2; ++c) ff_axpy_x2(ah[i][c], al[i][c], W, NW, H[c], L[c]);
      }
    }
    if (step % SK_FLUSH == SK_FLUSH - 1 || j0 + SK_TJ >= r1) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = rb + 8 * ty + i;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          float h0, h1, l0, l1;
          x2_unpack(ah[i][c], h0, h1);
          x2_unpack(al[i][c], l0, l1);
          const int l = lb + 4 * tx + 2 * c;
          if (r < ks && l < nf) Y[(int64_t)l * ks + r] += (double)h0 + (double)l0;
          if (r < ks && l + 1 < nf) Y[(int64_t)(l + 1) * ks + r] += (double)h1 + (double)l1;
          ah[i][c] = al[i][c] = x2_splat(0.0f);
        }
      }
    }
  }
}

// The FP64 sketch, for ID tolerances below the float-float kernel entries' accuracy:
// each block owns a 64 x 64 tile of Y, evaluates its 32 x 64 kernel entries per step in
// FP64 and accumulates 4 x 4 register tiles per thread (Omega row-major, ks x nt).
constexpr int S64_TR = 64;   // FP64 sketch: sketch rows per block
constexpr int S64_TL = 64;   // fine-grid points per block
constexpr int S64_TJ = 32;   // training rows per step

// On-surface Green's function of the unit sphere from the chord d (eqs. Gextonsurface /
// Gintonsurface written with log(2/d)): exterior 2/d - log(2/d) - log(1 + d/2),
// interior 2/d + log(2/d) - log(1 + d/2).
__device__ __forceinline__ double g_surface(double d, double sgn) {
  return 2.0 / d + sgn * log(2.0 / d) - log1p(0.5 * d);
}

__global__ void __launch_bounds__(SK_THREADS) sketch64_kernel(int ks, int nt, int nf, double sgn,
                                                            const double* __restrict__ Om,
                                                            const double* __restrict__ xt,
                                                            const double* __restrict__ xf, int r0, int r1,
                                                            double* __restrict__ Y) {
  __shared__ double Os[S64_TJ][S64_TR + 1];
  __shared__ double As[S64_TJ][S64_TL + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int rb = blockIdx.y * S64_TR, lb = blockIdx.x * S64_TL;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[i][k] = 0.0;
  for (int j0 = r0; j0 < r1; j0 += S64_TJ) {
    __syncthreads();
    for (int e = threadIdx.x; e < S64_TJ * S64_TR; e += SK_THREADS) {
      const int rr = e / S64_TJ, jj = e - rr * S64_TJ;  // consecutive threads: consecutive j
      const int r = rb + rr, j = j0 + jj;
      Os[jj][rr] = (r < ks && j < r1) ? Om[(int64_t)r * nt + j] : 0.0;
    }
    for (int e = threadIdx.x; e < S64_TJ * S64_TL; e += SK_THREADS) {
      const int jj = e / S64_TL, ll = e - jj * S64_TL;
      const int j = j0 + jj, l = lb + ll;
      double v = 0.0;
      if (j < r1 && l < nf) {
        const double dx = xt[3 * j] - xf[3 * l], dy = xt[3 * j + 1] - xf[3 * l + 1], dz = xt[3 * j + 2] - xf[3 * l + 2];
        v = g_surface(sqrt(dx * dx + dy * dy + dz * dz), sgn);
      }
      As[jj][ll] = v;
    }
    __syncthreads();
    for (int jj = 0; jj < S64_TJ; ++jj) {
      double o[4], a[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) o[i] = Os[jj][ty * 4 + i];
#pragma unroll
      for (int k = 0; k < 4; ++k) a[k] = As[jj][tx * 4 + k];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[i][k] = fma(o[i], a[k], acc[i][k]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int r = rb + ty * 4 + i, l = lb + tx * 4 + k;
      if (r < ks && l < nf) Y[(int64_t)l * ks + r] += acc[i][k];
    }
}

constexpr int CP_THREADS = 1024;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum over CP_THREADS threads (all must call); result in every thread.
__device__ __forceinline__ double block_sum64(double v, double* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < CP_THREADS / 32; ++i) s += red[i];
  return s;
}

// Yc (kse x nf) = first kse rows of Y (ks x nf), column norms, identity order. One warp per column.
__global__ void cpqr_init_kernel(int ks, int kse, int nf, const double* __restrict__ Y, double* __restrict__ Yc,
                                 double* __restrict__ cn, double* __restrict__ cn0, int* __restrict__ piv) {
  const int l = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (l >= nf) return;
  double s = 0.0;
  for (int r = lane; r < kse; r += 32) {
    const double y = Y[(int64_t)l * ks + r];
    Yc[(int64_t)l * kse + r] = y;
    s += y * y;
  }
  s = warp_sum(s);
  if (lane == 0) {
    cn[l] = cn0[l] = s;
    piv[l] = l;
  }
}

// Step st, part 1 (one block): pivot column = largest remaining norm (lowest index on
// ties), swapped into place; Householder vector v of its rows st.. and R_st,st.
__global__ void __launch_bounds__(CP_THREADS) cpqr_pivot_kernel(int kse, int nf, int st, double tol,
                                                                double* __restrict__ Yc, double* __restrict__ cn,
                                                                double* __restrict__ cn0, int* __restrict__ piv,
                                                                double* __restrict__ v, CpqrStatus* __restrict__ S) {
  __shared__ double red[CP_THREADS / 32];
  __shared__ double bv[CP_THREADS / 32];
  __shared__ int bi[CP_THREADS / 32];
  __shared__ int best_s;
  if (S->done) return;
  double best = -1.0;
  int bidx = nf;
  for (int l = st + threadIdx.x; l < nf; l += CP_THREADS)
    if (cn[l] > best) {
      best = cn[l];
      bidx = l;
    }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    if (ob > best || (ob == best && oi < bidx)) {
      best = ob;
      bidx = oi;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    bv[threadIdx.x >> 5] = best;
    bi[threadIdx.x >> 5] = bidx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = bv[0];
    int i = bi[0];
    for (int w = 1; w < CP_THREADS / 32; ++w)
      if (bv[w] > b || (bv[w] == b && bi[w] < i)) {
        b = bv[w];
        i = bi[w];
      }
    best_s = i < nf ? i : st;
  }
  __syncthreads();
  const int bst = best_s;
  double* col = Yc + (int64_t)st * kse;
  if (bst != st) {
    double* other = Yc + (int64_t)bst * kse;
    for (int r = threadIdx.x; r < kse; r += CP_THREADS) {
      const double t = col[r];
      col[r] = other[r];
      other[r] = t;
    }
    if (threadIdx.x == 0) {
      double t = cn[st];
      cn[st] = cn[bst];
      cn[bst] = t;
      t = cn0[st];
      cn0[st] = cn0[bst];
      cn0[bst] = t;
      const int ti = piv[st];
      piv[st] = piv[bst];
      piv[bst] = ti;
    }
  }
  __syncthreads();
  double a = 0.0;
  for (int r = st + threadIdx.x; r < kse; r += CP_THREADS) a += col[r] * col[r];
  const double nrm = sqrt(block_sum64(a, red));
  const double c0 = col[st];
  const double rss = (c0 >= 0.0) ? -nrm : nrm;
  const double r00 = (st == 0) ? fabs(rss) : S->r00;
  __syncthreads();
  if (fabs(rss) < tol * r00 || nrm == 0.0) {
    if (threadIdx.x == 0) {
      S->done = 1;
      S->p = st;
      if (st == 0) S->r00 = r00;
    }
    return;
  }
  double b2 = 0.0;
  for (int r = threadIdx.x; r < kse; r += CP_THREADS) {
    const double vr = (r < st) ? 0.0 : (r == st ? col[r] - rss : col[r]);
    v[r] = vr;
    b2 += vr * vr;
  }
  const double vv = block_sum64(b2, red);
  for (int r = st + threadIdx.x; r < kse; r += CP_THREADS) col[r] = (r == st) ? rss : 0.0;
  if (threadIdx.x == 0) {
    S->vv = vv;
    S->r00 = r00;
    S->p = st + 1;
  }
}

// Step st, part 2: apply the reflector to the remaining columns and downdate their norms
// (recomputed after cancellation). One warp per column.
__global__ void cpqr_update_kernel(int kse, int nf, int st, double* __restrict__ Yc, double* __restrict__ cn,
                                   double* __restrict__ cn0, const double* __restrict__ v,
                                   const CpqrStatus* __restrict__ S) {
  if (S->done) return;
  const int l = st + 1 + (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (l >= nf) return;
  double* y = Yc + (int64_t)l * kse;
  double d = 0.0;
  for (int r = st + lane; r < kse; r += 32) d += v[r] * y[r];
  d = warp_sum(d);
  const double f = 2.0 * d / S->vv;
  for (int r = st + lane; r < kse; r += 32) y[r] -= f * v[r];
  __syncwarp();
  const double yst = y[st];
  double nn = cn[l] - yst * yst;
  if (nn < 1e-10 * cn0[l]) {
    double q = 0.0;
    for (int r = st + 1 + lane; r < kse; r += 32) q += y[r] * y[r];
    nn = warp_sum(q);
    if (lane == 0) cn0[l] = nn;
  }
  if (lane == 0) cn[l] = nn;
}

// X = R11^-1 R12 (p x nrest, row-major): one back-substitution per rest column.
__global__ void cpqr_solve_x_kernel(int kse, int p, int nf, const double* __restrict__ Yc, double* __restrict__ X) {
  const int nrest = nf - p;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nrest) return;
  const double* y = Yc + (int64_t)(p + c) * kse;
  for (int m = p - 1; m >= 0; --m) {
    double val = y[m];
    for (int q = m + 1; q < p; ++q) val -= Yc[(int64_t)q * kse + m] * X[(int64_t)q * nrest + c];
    X[(int64_t)m * nrest + c] = val / Yc[(int64_t)m * kse + m];
  }
}

// T[m][j] = WB[piv[m]][j] + sum_c X[m][c] WB[piv[p + c]][j] (eq. Tmap); one thread per entry.
__global__ void assemble_t_kernel(int p, int K, int nf, const int* __restrict__ piv, const double* __restrict__ X,
                                  const double* __restrict__ WB, double* __restrict__ T) {
  const int m = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= K) return;
  const int nrest = nf - p;
  const double* xm = X + (int64_t)m * nrest;
  double t0 = WB[(int64_t)piv[m] * K + j], t1 = 0.0, t2 = 0.0, t3 = 0.0;
  int c = 0;
  for (; c + 4 <= nrest; c += 4) {
    t0 = fma(xm[c], WB[(int64_t)piv[p + c] * K + j], t0);
    t1 = fma(xm[c + 1], WB[(int64_t)piv[p + c + 1] * K + j], t1);
    t2 = fma(xm[c + 2], WB[(int64_t)piv[p + c + 2] * K + j], t2);
    t3 = fma(xm[c + 3], WB[(int64_t)piv[p + c + 3] * K + j], t3);
  }
  for (; c < nrest; ++c) t0 = fma(xm[c], WB[(int64_t)piv[p + c] * K + j], t0);
  T[(int64_t)m * K + j] = (t0 + t1) + (t2 + t3);
}

}  // namespace

struct DeviceSketch {
  int ks = 0, nt = 0, nf = 0;
  int mode = 0;
  bool ff = true;         // float-float sketch (else FP64)
  float* Om = nullptr;    // float-float sketch: nt x ks (Omega transposed, FP32 values)
  double* Om64 = nullptr; // FP64 sketch: ks x nt
  float4* logtab = nullptr;
  double *xt = nullptr, *xf = nullptr, *Y = nullptr;
  // CPQR of the first kse rows and assembly of T
  int kse = 0, K = 0;
  double *Yc = nullptr, *cn = nullptr, *cn0 = nullptr, *v = nullptr, *X = nullptr, *WB = nullptr, *T = nullptr;
  int* piv = nullptr;
  CpqrStatus* st = nullptr;
  cudaStream_t stream = nullptr;
};

void sketch_destroy(DeviceSketch* s) {
  if (!s) return;
  cudaFree(s->Om);
  cudaFree(s->Om64);
  cudaFree(s->logtab);
  cudaFree(s->xt);
  cudaFree(s->xf);
  cudaFree(s->Y);
  cudaFree(s->Yc);
  cudaFree(s->cn);
  cudaFree(s->cn0);
  cudaFree(s->v);
  cudaFree(s->X);
  cudaFree(s->WB);
  cudaFree(s->T);
  cudaFree(s->piv);
  cudaFree(s->st);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

DeviceSketch* sketch_create(int ks, int nt, int nf, int mode, const double* Om, const double* xt,
                            const double* xf, bool ff) {
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();  // clear the error state of a machine without a device
    return nullptr;
  }
  DeviceSketch* s = new DeviceSketch();
  s->ks = ks;
  s->nt = nt;
  s->nf = nf;
  s->mode = mode;
  s->ff = ff;
  const size_t nOm = (size_t)ks * nt, nY = (size_t)ks * nf;
  // float-float sketch: Omega's values are FP32 numbers (the precompute draws them so),
  // transposed so that a training row's coefficients are contiguous
  std::vector<float> omt(ff ? nOm : 0);
  for (int r = 0; r < (ff ? ks : 0); ++r)
    for (int t = 0; t < nt; ++t) omt[(size_t)t * ks + r] = (float)Om[(size_t)r * nt + t];
  // float-float log table of green_f2: c_i = 1 + (i + 1/2)/64, (log c_i, 1/c_i) as hi, lo
  std::vector<float> lt(4 * kLogTable);
  for (int i = 0; i < kLogTable; ++i) {
    const double ci = 1.0 + (i + 0.5) / 64.0;
    const double L = std::log(ci), inv = 1.0 / ci;
    lt[4 * i + 0] = (float)L;
    lt[4 * i + 1] = (float)(L - (double)(float)L);
    lt[4 * i + 2] = (float)inv;
    lt[4 * i + 3] = (float)(inv - (double)(float)inv);
  }
  bool ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess &&
            (ff ? cudaMalloc(&s->Om, nOm * sizeof(float)) : cudaMalloc(&s->Om64, nOm * sizeof(double))) ==
                cudaSuccess &&
            cudaMalloc(&s->logtab, kLogTable * sizeof(float4)) == cudaSuccess &&
            cudaMalloc(&s->xt, 3 * (size_t)nt * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&s->xf, 3 * (size_t)nf * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&s->Y, nY * sizeof(double)) == cudaSuccess &&
            (ff ? cudaMemcpyAsync(s->Om, omt.data(), nOm * sizeof(float), cudaMemcpyHostToDevice, s->stream)
                : cudaMemcpyAsync(s->Om64, Om, nOm * sizeof(double), cudaMemcpyHostToDevice, s->stream)) ==
                cudaSuccess &&
            cudaMemcpyAsync(s->logtab, lt.data(), kLogTable * sizeof(float4), cudaMemcpyHostToDevice, s->stream) ==
                cudaSuccess &&
            cudaMemcpyAsync(s->xt, xt, 3 * (size_t)nt * sizeof(double), cudaMemcpyHostToDevice, s->stream) ==
                cudaSuccess &&
            cudaMemcpyAsync(s->xf, xf, 3 * (size_t)nf * sizeof(double), cudaMemcpyHostToDevice, s->stream) ==
                cudaSuccess &&
            cudaMemsetAsync(s->Y, 0, nY * sizeof(double), s->stream) == cudaSuccess &&
            cudaStreamSynchronize(s->stream) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    sketch_destroy(s);
    return nullptr;
  }
  return s;
}

bool sketch_add_rows(DeviceSketch* s, int r0, int r1) {
  if (r1 <= r0) return true;
  if (!s->ff) {
    dim3 grid((unsigned)((s->nf + S64_TL - 1) / S64_TL), (unsigned)((s->ks + S64_TR - 1) / S64_TR));
    count_launch(), sketch64_kernel<<<grid, SK_THREADS, 0, s->stream>>>(s->ks, s->nt, s->nf, s->mode == 0 ? -1.0 : 1.0,
                                                                        s->Om64, s->xt, s->xf, r0, r1, s->Y);
    return cudaGetLastError() == cudaSuccess;
  }
  dim3 grid((unsigned)((s->nf + SK_TL - 1) / SK_TL), (unsigned)((s->ks + SK_ROWS - 1) / SK_ROWS));
  if (s->mode == 0)
    count_launch(), sketch_kernel<0><<<grid, SK_THREADS, 0, s->stream>>>(s->ks, s->nf, s->Om, s->xt, s->xf, r0, r1,
                                                                          s->logtab, s->Y);
  else
    count_launch(), sketch_kernel<1><<<grid, SK_THREADS, 0, s->stream>>>(s->ks, s->nf, s->Om, s->xt, s->xf, r0, r1,
                                                                          s->logtab, s->Y);
  return cudaGetLastError() == cudaSuccess;
}

bool sketch_read(DeviceSketch* s, double* Y) {
  return cudaMemcpyAsync(Y, s->Y, (size_t)s->ks * s->nf * sizeof(double), cudaMemcpyDeviceToHost, s->stream) ==
             cudaSuccess &&
         cudaStreamSynchronize(s->stream) == cudaSuccess;
}

int sketch_cpqr(DeviceSketch* s, int kse, double tol, std::vector<int>& piv) {
  const int nf = s->nf;
  if (kse > s->ks || kse < 1) return -1;
  bool ok = true;
  if (!s->Yc) {
    ok = cudaMalloc(&s->Yc, (size_t)s->ks * nf * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&s->cn, (size_t)nf * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&s->cn0, (size_t)nf * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&s->v, (size_t)s->ks * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&s->piv, (size_t)nf * sizeof(int)) == cudaSuccess &&
         cudaMalloc(&s->st, sizeof(CpqrStatus)) == cudaSuccess;
    if (!ok) return -1;
  }
  s->kse = kse;
  const CpqrStatus zero{0, 0, 0.0, 1.0};
  if (cudaMemcpyAsync(s->st, &zero, sizeof(zero), cudaMemcpyHostToDevice, s->stream) != cudaSuccess) return -1;
  const unsigned wblocks = (unsigned)(((int64_t)nf * 32 + 255) / 256);
  count_launch(), cpqr_init_kernel<<<wblocks, 256, 0, s->stream>>>(s->ks, kse, nf, s->Y, s->Yc, s->cn, s->cn0,
                                                                   s->piv);
  if (cudaGetLastError() != cudaSuccess) return -1;
  CpqrStatus h{};
  for (int st = 0; st < kse; ++st) {
    count_launch(), cpqr_pivot_kernel<<<1, CP_THREADS, 0, s->stream>>>(kse, nf, st, tol, s->Yc, s->cn, s->cn0, s->piv,
                                                                       s->v, s->st);
    const int rest = nf - st - 1;
    if (rest > 0) {
      const unsigned ub = (unsigned)(((int64_t)rest * 32 + 255) / 256);
      count_launch(), cpqr_update_kernel<<<ub, 256, 0, s->stream>>>(kse, nf, st, s->Yc, s->cn, s->cn0, s->v, s->st);
    }
    if (cudaGetLastError() != cudaSuccess) return -1;
    if ((st & 15) == 15 || st == kse - 1) {
      if (cudaMemcpyAsync(&h, s->st, sizeof(h), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
          cudaStreamSynchronize(s->stream) != cudaSuccess)
        return -1;
      if (h.done) break;
    }
  }
  piv.resize(nf);
  if (cudaMemcpyAsync(piv.data(), s->piv, (size_t)nf * sizeof(int), cudaMemcpyDeviceToHost, s->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(&h, s->st, sizeof(h), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    return -1;
  return h.done ? h.p : kse;
}

bool sketch_set_wb(DeviceSketch* s, int K, const double* WB) {
  s->K = K;
  const size_t n = (size_t)s->nf * K;
  return (s->WB || cudaMalloc(&s->WB, n * sizeof(double)) == cudaSuccess) &&
         cudaMemcpyAsync(s->WB, WB, n * sizeof(double), cudaMemcpyHostToDevice, s->stream) == cudaSuccess &&
         cudaStreamSynchronize(s->stream) == cudaSuccess;
}

bool sketch_assemble(DeviceSketch* s, int p, std::vector<double>& T) {
  const int nf = s->nf, K = s->K, nrest = nf - p;
  if (!s->WB || p < 1 || p > s->kse || nrest < 0) return false;
  if (!s->X && cudaMalloc(&s->X, (size_t)s->ks * nf * sizeof(double)) != cudaSuccess) return false;
  if (!s->T && cudaMalloc(&s->T, (size_t)s->ks * K * sizeof(double)) != cudaSuccess) return false;
  if (nrest > 0) {
    count_launch(), cpqr_solve_x_kernel<<<(unsigned)((nrest + 127) / 128), 128, 0, s->stream>>>(s->kse, p, nf, s->Yc,
                                                                                                 s->X);
    if (cudaGetLastError() != cudaSuccess) return false;
  }
  dim3 grid((unsigned)((K + 127) / 128), (unsigned)p);
  count_launch(), assemble_t_kernel<<<grid, 128, 0, s->stream>>>(p, K, nf, s->piv, s->X, s->WB, s->T);
  if (cudaGetLastError() != cudaSuccess) return false;
  T.resize((size_t)p * K);
  return cudaMemcpyAsync(T.data(), s->T, T.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream) ==
             cudaSuccess &&
         cudaStreamSynchronize(s->stream) == cudaSuccess;
}


}  // namespace ncs
