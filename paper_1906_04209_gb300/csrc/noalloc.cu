// Allocation-free variant of the Arnoldi projection kernel (ncs_block_dots_noalloc).
//
// Some callers cannot call cudaMalloc: an application that hands the library a device
// whose memory it manages itself (a fixed budget carved out up front, a pool it owns),
// a real-time loop that must not block on the allocator, or code that records its
// work into a stream capture where allocation calls are not allowed. For them the
// partial sums of the two-stage reduction live in a file-scope device array sized for
// at most kNoAllocMaxVectors vectors; the caller passes only its inputs and outputs.
// The first call on a device looks the array's device address up (with that device
// current), so make that first call before any stream capture. Calls that overlap on
// the GPU share the array and race: serialise them (one stream, or events).
#include <cuda_runtime.h>

#include <mutex>

#include "internal.hpp"

namespace ncs {

constexpr int kNoAllocMaxVectors = 1024;  // 64 partial sums each: 512 KiB of scratch

// Scratch shared by every call on a device (each GPU that loads the library holds
// one copy until the process exits). Each call overwrites the partial sums it reads,
// so nothing has to be cleared between calls.
static __device__ __align__(256) double g_noalloc_partial[kDotChunks * kNoAllocMaxVectors];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch array for the current device, looked up once per
// device with that device current (the host-side symbol is only a stand-in).
double* scratch_for_current_device(int* rc) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *rc = NCS_E_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    double* p = nullptr;
    if (cudaGetSymbolAddress((void**)&p, g_noalloc_partial) != cudaSuccess || !p) {
      *rc = NCS_E_CUDA;
      return nullptr;
    }
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

}  // namespace

}  // namespace ncs

extern "C" int ncs_block_dots_noalloc(int64_t n, int k, const double* V, int64_t ld, const double* w, double* out,
                                      void* stream) {
  if (n < 0 || k < 0 || ld < n || (k > 0 && (!V || !w || !out))) return NCS_E_INPUT;
  if (k > ncs::kNoAllocMaxVectors) return NCS_E_INPUT;  // beyond the fixed scratch
  if (k == 0) return NCS_OK;
  // an error left by earlier, unrelated work on this thread would otherwise surface
  // after this call's launch as if the launch had failed: report it before launching
  if (cudaGetLastError() != cudaSuccess) return NCS_E_CUDA;
  int rc = NCS_OK;
  double* partial = ncs::scratch_for_current_device(&rc);
  if (!partial) return rc;
  if (ncs::launch_dots(n, k, V, ld, w, partial, out, (cudaStream_t)stream) != cudaSuccess) return NCS_E_CUDA;
  return NCS_OK;
}
