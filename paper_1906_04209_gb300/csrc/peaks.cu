// Arithmetic-pipe peaks of the device, measured by the library's own microkernel: the
// denominators for the FP64 and FP32 pair kernels' pipe fractions (no counterpart in the
// paper). Each thread runs 8 independent FMA chains (enough to hide the pipe latency),
// 152 x 8 blocks of 256 threads, timed with CUDA events on a private stream.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.hpp"

namespace ncs {

namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(int iters, T a, T b, T* __restrict__ sink) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == (T)-1.2345) sink[threadIdx.x] = s;  // keeps the chains alive; never true
}

}  // namespace

}  // namespace ncs

extern "C" int ncs_fma_peak(int precision, double* tflops) {
  if (!tflops || (precision != NCS_FP64 && precision != NCS_FP32)) return NCS_E_INPUT;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* sink = nullptr;
  int rc = NCS_OK;
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess || cudaMalloc(&sink, 256 * sizeof(double)) != cudaSuccess) {
    rc = NCS_E_CUDA;
  } else {
    const int blocks = sms * 8;
    const int iters = precision == NCS_FP64 ? 4096 : 65536;
    float best = 1e30f;
    for (int rep = 0; rep < 4 && rc == NCS_OK; ++rep) {  // the first launch warms up
      cudaEventRecord(e0, s);
      if (precision == NCS_FP64)
        ncs::count_launch(), ncs::fma_peak_kernel<double><<<blocks, 256, 0, s>>>(iters, 0.999999, 1e-7, (double*)sink);
      else
        ncs::count_launch(), ncs::fma_peak_kernel<float><<<blocks, 256, 0, s>>>(iters, 0.999f, 1e-3f, (float*)sink);
      cudaEventRecord(e1, s);
      float ms = 0.0f;
      if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        rc = NCS_E_CUDA;
      else if (rep > 0 && ms < best)
        best = ms;
    }
    if (rc == NCS_OK) *tflops = 2.0 * 8.0 * iters * (double)blocks * 256.0 / (best * 1e-3) / 1e12;
  }
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  return rc;
}
