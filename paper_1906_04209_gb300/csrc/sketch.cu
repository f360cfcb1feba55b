// Device accumulation of the ID sketch (see sketch.hpp): Y += Omega[:, r0:r1] A[r0:r1, :]
// in FP64, A_tl = G(|x_t - x_l|) evaluated on the fly. Each block owns a 64 x 64 tile of Y
// (sketch rows x fine points), stages 32 training rows of Omega and of A per step in shared
// memory and accumulates 4 x 4 register tiles per thread.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.hpp"
#include "sketch.hpp"

namespace ncs {

namespace {

constexpr int SK_TR = 64;   // sketch rows per block
constexpr int SK_TL = 64;   // fine-grid points per block
constexpr int SK_TJ = 32;   // training rows per step
constexpr int SK_THREADS = 256;

// On-surface Green's function of the unit sphere from the chord d (eqs. Gextonsurface /
// Gintonsurface written with log(2/d)): exterior 2/d - log(2/d) - log(1 + d/2),
// interior 2/d + log(2/d) - log(1 + d/2).
__device__ __forceinline__ double g_surface(double d, double sgn) {
  return 2.0 / d + sgn * log(2.0 / d) - log1p(0.5 * d);
}

__global__ void __launch_bounds__(SK_THREADS) sketch_kernel(int ks, int nt, int nf, double sgn,
                                                            const double* __restrict__ Om,
                                                            const double* __restrict__ xt,
                                                            const double* __restrict__ xf, int r0, int r1,
                                                            double* __restrict__ Y) {
  __shared__ double Os[SK_TJ][SK_TR + 1];
  __shared__ double As[SK_TJ][SK_TL + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int rb = blockIdx.y * SK_TR, lb = blockIdx.x * SK_TL;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[i][k] = 0.0;
  for (int j0 = r0; j0 < r1; j0 += SK_TJ) {
    __syncthreads();
    for (int e = threadIdx.x; e < SK_TJ * SK_TR; e += SK_THREADS) {
      const int rr = e / SK_TJ, jj = e - rr * SK_TJ;  // consecutive threads: consecutive j
      const int r = rb + rr, j = j0 + jj;
      Os[jj][rr] = (r < ks && j < r1) ? Om[(int64_t)r * nt + j] : 0.0;
    }
    for (int e = threadIdx.x; e < SK_TJ * SK_TL; e += SK_THREADS) {
      const int jj = e / SK_TL, ll = e - jj * SK_TL;
      const int j = j0 + jj, l = lb + ll;
      double v = 0.0;
      if (j < r1 && l < nf) {
        const double dx = xt[3 * j] - xf[3 * l], dy = xt[3 * j + 1] - xf[3 * l + 1], dz = xt[3 * j + 2] - xf[3 * l + 2];
        v = g_surface(sqrt(dx * dx + dy * dy + dz * dz), sgn);
      }
      As[jj][ll] = v;
    }
    __syncthreads();
    for (int jj = 0; jj < SK_TJ; ++jj) {
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

}  // namespace

struct DeviceSketch {
  int ks = 0, nt = 0, nf = 0;
  double sgn = 1.0;
  double *Om = nullptr, *xt = nullptr, *xf = nullptr, *Y = nullptr;
  cudaStream_t stream = nullptr;
};

void sketch_destroy(DeviceSketch* s) {
  if (!s) return;
  cudaFree(s->Om);
  cudaFree(s->xt);
  cudaFree(s->xf);
  cudaFree(s->Y);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

DeviceSketch* sketch_create(int ks, int nt, int nf, int mode, const double* Om, const double* xt,
                            const double* xf) {
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();  // clear the error state of a machine without a device
    return nullptr;
  }
  DeviceSketch* s = new DeviceSketch();
  s->ks = ks;
  s->nt = nt;
  s->nf = nf;
  s->sgn = (mode == 0) ? -1.0 : 1.0;
  const size_t nOm = (size_t)ks * nt, nY = (size_t)ks * nf;
  bool ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMalloc(&s->Om, nOm * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&s->xt, 3 * (size_t)nt * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&s->xf, 3 * (size_t)nf * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&s->Y, nY * sizeof(double)) == cudaSuccess &&
            cudaMemcpyAsync(s->Om, Om, nOm * sizeof(double), cudaMemcpyHostToDevice, s->stream) == cudaSuccess &&
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
  dim3 grid((unsigned)((s->nf + SK_TL - 1) / SK_TL), (unsigned)((s->ks + SK_TR - 1) / SK_TR));
  count_launch(), sketch_kernel<<<grid, SK_THREADS, 0, s->stream>>>(s->ks, s->nt, s->nf, s->sgn, s->Om, s->xt, s->xf,
                                                                     r0, r1, s->Y);
  return cudaGetLastError() == cudaSuccess;
}

bool sketch_read(DeviceSketch* s, double* Y) {
  return cudaMemcpyAsync(Y, s->Y, (size_t)s->ks * s->nf * sizeof(double), cudaMemcpyDeviceToHost, s->stream) ==
             cudaSuccess &&
         cudaStreamSynchronize(s->stream) == cudaSuccess;
}

}  // namespace ncs
