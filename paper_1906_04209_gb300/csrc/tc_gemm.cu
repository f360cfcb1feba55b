// Tensor-core (tcgen05, kind::tf32) GEMM for the per-patch operator contractions of the
// FP32 product (Kaye & Greengard, Section 7, Steps 3.1 and 3.5):
//     rho (N x p_total) = X (N x K) T_all^T          (outgoing coefficients, eq. Tmap)
//     y   (N x K)       = X + Z (N x K*) P^T         (Zernike transform P)
// D = A B^T with A (rows x Kd) and B (cols x Kd) both K-major in global memory (FP64 or
// FP32). Each CTA computes a 128-row x BN-column tile: the operands are converted to
// TF32 pairs (hi = tf32(v), lo = tf32(v - hi)) while being staged into shared memory in
// the canonical no-swizzle K-major layout (8-row x 16-byte core matrices), one thread
// issues tcgen05.mma for hi*hi + hi*lo + lo*hi (the "3xTF32" split, ~FP32 accuracy)
// accumulating in tensor memory, completion is signalled through an mbarrier, and the
// four warps read the accumulator back with tcgen05.ld. Every wait is bounded: on
// timeout the kernel records an error flag, skips its stores and still frees TMEM.
#include <cstdint>

#include "internal.hpp"

namespace ncs {

namespace {

constexpr int TC_BM = 128;   // rows per CTA (TMEM lanes)
constexpr int TC_KC = 32;    // K elements staged per chunk (4 MMA k-steps of 8)
constexpr int TC_THREADS = 128;
constexpr uint32_t kSpinLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t to_tf32(float v) {
  uint32_t r;
  asm volatile("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

// Shared-memory matrix descriptor (no swizzle, K-major): start >> 4 in bits 0-13,
// leading (K-direction) core-matrix stride >> 4 in bits 16-29, stride (M/N-direction)
// core-matrix stride >> 4 in bits 32-45, descriptor version 1 in bits 46-47.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor for kind::tf32: D = F32 (bits 4-5 = 1), A and B = TF32
// (bits 7-9 and 10-12 = 2), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok = 0;
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity));
    if (ok) return true;
  }
  return false;
}

// Offset (bytes) of element (r, k) of a rows x kc tile in the core-matrix layout:
// core matrix (r/8, k/4) at ((r/8) * (kc/4) + k/4) * 128, row r%8 at 16 * (r%8),
// element k%4 at 4 * (k%4). K-direction core stride (LBO) = 128 B, M/N-direction
// stride (SBO) = (kc/4) * 128 B.
__device__ __forceinline__ uint32_t tile_off(int r, int k, int kc) {
  return (uint32_t)((((r >> 3) * (kc >> 2) + (k >> 2)) << 7) + ((r & 7) << 4) + ((k & 3) << 2));
}

template <typename TA, typename TB, int BN>
__global__ void __launch_bounds__(TC_THREADS) tc_gemm_kernel(int64_t rows, int cols, int Kd, const TA* __restrict__ A,
                                                             int64_t lda, const TB* __restrict__ B, int64_t ldb,
                                                             float* __restrict__ D, int64_t ldd,
                                                             const double* __restrict__ addx, double* __restrict__ Dd,
                                                             int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char tc_smem_raw[];
  // [A hi | A lo | B hi | B lo], each TC_BM (or BN) rows x TC_KC tf32 words, 128-B aligned
  uint8_t* tc_smem = tc_smem_raw + ((128u - (smem_u32(tc_smem_raw) & 127u)) & 127u);
  uint8_t* Ahi = tc_smem;
  uint8_t* Alo = Ahi + TC_BM * TC_KC * 4;
  uint8_t* Bhi = Alo + TC_BM * TC_KC * 4;
  uint8_t* Blo = Bhi + BN * TC_KC * 4;
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = (int64_t)blockIdx.x * TC_BM;
  const int c0 = blockIdx.y * BN;
  constexpr uint32_t NCOL = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(NCOL));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = idesc_tf32(TC_BM, BN);
  uint32_t phase = 0;
  const int nchunk = (Kd + TC_KC - 1) / TC_KC;
  for (int ch = 0; ch < nchunk; ++ch) {
    const int k0 = ch * TC_KC;
    // stage A (TC_BM x TC_KC) and B (BN x TC_KC) as tf32 hi/lo, zero padded
    for (int idx = threadIdx.x; idx < TC_BM * TC_KC; idx += TC_THREADS) {
      const int r = idx / TC_KC, k = idx - r * TC_KC;
      float v = 0.0f;
      if (r0 + r < rows && k0 + k < Kd) v = (float)A[(r0 + r) * lda + k0 + k];
      const uint32_t h = to_tf32(v);
      const uint32_t l = to_tf32(v - __uint_as_float(h));
      const uint32_t o = tile_off(r, k, TC_KC);
      *reinterpret_cast<uint32_t*>(Ahi + o) = h;
      *reinterpret_cast<uint32_t*>(Alo + o) = l;
    }
    for (int idx = threadIdx.x; idx < BN * TC_KC; idx += TC_THREADS) {
      const int r = idx / TC_KC, k = idx - r * TC_KC;
      float v = 0.0f;
      if (c0 + r < cols && k0 + k < Kd) v = (float)B[(int64_t)(c0 + r) * ldb + k0 + k];
      const uint32_t h = to_tf32(v);
      const uint32_t l = to_tf32(v - __uint_as_float(h));
      const uint32_t o = tile_off(r, k, TC_KC);
      *reinterpret_cast<uint32_t*>(Bhi + o) = h;
      *reinterpret_cast<uint32_t*>(Blo + o) = l;
    }
    // make the generic-proxy smem writes visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t sboA = (TC_KC / 4) * 128, sboB = (TC_KC / 4) * 128;
      for (int ks = 0; ks < TC_KC / 8; ++ks) {
        const uint32_t koff = (uint32_t)ks * 2 * 128;  // two core matrices (8 tf32) per k-step
        const uint64_t ah = smem_desc(smem_u32(Ahi) + koff, 128, sboA);
        const uint64_t al = smem_desc(smem_u32(Alo) + koff, 128, sboA);
        const uint64_t bh = smem_desc(smem_u32(Bhi) + koff, 128, sboB);
        const uint64_t bl = smem_desc(smem_u32(Blo) + koff, 128, sboB);
        const uint32_t acc0 = (ch > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ah), "l"(bh), "r"(idesc), "r"(acc0));
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, 1, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ah), "l"(bl), "r"(idesc));
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, 1, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(al), "l"(bh), "r"(idesc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&bar)));
    }
    // all threads wait for the MMAs of this chunk before the staging buffers are reused
    if (!mbar_wait(&bar, phase)) failed = 1;
    phase ^= 1u;
    __syncthreads();
    if (failed) break;
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!failed) {
    // epilogue: warp w owns TMEM lanes 32w..32w+31 = tile rows; 32 columns per load
    const int64_t r = r0 + warp * 32 + lane;
    for (int cb = 0; cb < BN; cb += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
            "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
            "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (r < rows) {
        for (int j = 0; j < 32; ++j) {
          const int c = c0 + cb + j;
          if (c < cols && cb + j < BN) {
            const float val = __uint_as_float(v[j]);
            if (Dd)
              Dd[r * ldd + c] = addx[r * ldd + c] + (double)val;
            else
              D[r * ldd + c] = val;
          }
        }
      }
    }
  } else if (threadIdx.x == 0) {
    atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL));
}

template <typename TA, typename TB, int BN>
cudaError_t launch(int64_t rows, int cols, int Kd, const TA* A, int64_t lda, const TB* B, int64_t ldb, float* D,
                   int64_t ldd, const double* addx, double* Dd, int* err, cudaStream_t s) {
  const size_t smem = (size_t)(2 * TC_BM + 2 * BN) * TC_KC * 4 + 1024;
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<TA, TB, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((rows + TC_BM - 1) / TC_BM), (unsigned)((cols + BN - 1) / BN));
  count_launch(), tc_gemm_kernel<TA, TB, BN><<<grid, TC_THREADS, smem, s>>>(rows, cols, Kd, A, lda, B, ldb, D, ldd, addx, Dd, err);
  return cudaGetLastError();
}

}  // namespace

// rho32 = X T_all^T (FP32 result), X: N x K FP64, T_all: p_total x K FP32 (row-major).
cudaError_t launch_tc_outgoing(const DeviceData& d, const double* x, const float* T32, int* err, cudaStream_t s) {
  return launch<double, float, 128>(d.N, d.p, d.K, x, d.K, T32, d.K, d.rho32, d.p, nullptr, nullptr, err, s);
}

// y = x + Z P^T, Z: N x Kstar FP64, P: K x Kstar FP32 (row-major), y, x: N x K FP64.
cudaError_t launch_tc_apply_P(const DeviceData& d, const double* x, double* y, const float* P32, int* err,
                              cudaStream_t s) {
  if (d.K <= 64)
    return launch<double, float, 64>(d.N, d.K, d.Kstar, d.z, d.Kstar, P32, d.Kstar, nullptr, d.K, x, y, err, s);
  if (d.K <= 128)
    return launch<double, float, 128>(d.N, d.K, d.Kstar, d.z, d.Kstar, P32, d.Kstar, nullptr, d.K, x, y, err, s);
  if (d.K <= 144)
    return launch<double, float, 144>(d.N, d.K, d.Kstar, d.z, d.Kstar, P32, d.Kstar, nullptr, d.K, x, y, err, s);
  return launch<double, float, 256>(d.N, d.K, d.Kstar, d.z, d.Kstar, P32, d.Kstar, nullptr, d.K, x, y, err, s);
}

// Standalone D = A B^T (FP32 inputs and output) for tests.
cudaError_t launch_tc_gemm_f32(int64_t rows, int cols, int Kd, const float* A, const float* B, float* D, int* err,
                               cudaStream_t s) {
  return launch<float, float, 128>(rows, cols, Kd, A, Kd, B, Kd, D, cols, nullptr, nullptr, err, s);
}

}  // namespace ncs
