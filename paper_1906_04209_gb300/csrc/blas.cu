// Dense-vector kernels for GMRES on the device (FP64, deterministic reductions).
#include <cstdint>

#include "internal.hpp"

namespace ncs {

// partial[j * kDotChunks + c] = sum over chunk c of V_j . w
__global__ void __launch_bounds__(256) dots_partial_kernel(int64_t n, const double* __restrict__ V, int64_t ld,
                                                           const double* __restrict__ w,
                                                           double* __restrict__ partial) {
  __shared__ double red[256];
  const int c = blockIdx.x, j = blockIdx.y;
  const int64_t chunk = (n + kDotChunks - 1) / kDotChunks;
  const int64_t lo = c * chunk, hi = min(n, lo + chunk);
  const double* v = V + j * ld;
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc = fma(v[i], w[i], acc);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[j * kDotChunks + c] = red[0];
}

__global__ void dots_final_kernel(int k, const double* __restrict__ partial, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  double s = 0.0;
  for (int c = 0; c < kDotChunks; ++c) s += partial[j * kDotChunks + c];
  out[j] = s;
}

cudaError_t launch_dots(int64_t n, int k, const double* V, int64_t ld, const double* w, double* partial,
                        double* out, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  count_launch(), dots_partial_kernel<<<dim3(kDotChunks, k), 256, 0, s>>>(n, V, ld, w, partial);
  count_launch(), dots_final_kernel<<<(k + 127) / 128, 128, 0, s>>>(k, partial, out);
  return cudaGetLastError();
}

// w += sign * sum_j h_j V_j
__global__ void __launch_bounds__(256) sub_combination_kernel(int64_t n, int k, const double* __restrict__ V,
                                                              int64_t ld, const double* __restrict__ h,
                                                              double* __restrict__ w, double sign) {
  extern __shared__ double hs[];
  for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = h[j];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc = fma(hs[j], V[j * ld + i], acc);
    w[i] = fma(sign, acc, w[i]);
  }
}

cudaError_t launch_sub_combination(int64_t n, int k, const double* V, int64_t ld, const double* h, double* w,
                                   double sign, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
  count_launch(), sub_combination_kernel<<<(unsigned)blocks, 256, k * sizeof(double), s>>>(n, k, V, ld, h, w, sign);
  return cudaGetLastError();
}

__global__ void scale_copy_kernel(int64_t n, const double* __restrict__ w, double a, double* __restrict__ v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = a * w[i];
}

cudaError_t launch_scale_copy(int64_t n, const double* w, double a, double* v, cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
  count_launch(), scale_copy_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, w, a, v);
  return cudaGetLastError();
}

// y = a x + b y
__global__ void axpby_kernel(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], b * y[i]);
}

cudaError_t launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
  count_launch(), axpby_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, a, x, b, y);
  return cudaGetLastError();
}

__global__ void nonfinite_kernel(int64_t n, const double* __restrict__ x, int* __restrict__ out) {
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (bad) atomicOr(out, 1);
}

cudaError_t launch_nonfinite_count(int64_t n, const double* x, int* out, cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 4);
  count_launch(), nonfinite_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, x, out);
  return cudaGetLastError();
}

}  // namespace ncs

namespace ncs {

// partial[c] = sum over chunk c of x[i] * I[i mod K]  (I_sigma = I . sum_i f_i, eq. getI)
__global__ void __launch_bounds__(256) periodic_dot_kernel(int64_t n, int K, const double* __restrict__ x,
                                                           const double* __restrict__ I,
                                                           double* __restrict__ partial) {
  __shared__ double red[256];
  const int c = blockIdx.x;
  const int64_t chunk = (n + kDotChunks - 1) / kDotChunks;
  const int64_t lo = c * chunk, hi = min(n, lo + chunk);
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc = fma(x[i], I[i % K], acc);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[c] = red[0];
}

cudaError_t launch_periodic_dot(int64_t n, int K, const double* x, const double* I, double* partial,
                                double* out, cudaStream_t s) {
  count_launch(), periodic_dot_kernel<<<kDotChunks, 256, 0, s>>>(n, K, x, I, partial);
  count_launch(), dots_final_kernel<<<1, 128, 0, s>>>(1, partial, out);
  return cudaGetLastError();
}

}  // namespace ncs
