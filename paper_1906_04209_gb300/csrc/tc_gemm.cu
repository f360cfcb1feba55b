// Tensor-core (tcgen05, kind::tf32) GEMM for the per-patch operator contractions of the
// FP32 product (Kaye & Greengard, Section 7, Steps 3.1 and 3.5):
//     rho (N x p_total) = X (N x K) T_all^T          (outgoing coefficients, eq. Tmap)
//     y   (N x K)       = X + Z (N x K*) P^T         (Zernike transform P)
// D = A B^T with A (rows x Kd) K-major in global memory (FP64 or FP32) and B a constant
// operator. Accuracy: both operands are split into TF32 pairs (hi = tf32(v),
// lo = tf32(v - hi)) and the tensor cores accumulate hi*hi + hi*lo + lo*hi in FP32
// ("3xTF32", about FP32 accuracy).
//
// Data movement:
//   * B is split and laid out once (tc_pack_kernel) in the canonical no-swizzle K-major
//     shared-memory layout, one contiguous block per (column tile, K chunk); a CTA brings
//     each block in with one bulk TMA copy (cp.async.bulk) completing on an mbarrier;
//   * A is read by all threads, split and stored into the same layout (one 128-byte core
//     matrix per warp store);
//   * two stages: while the tensor cores work on chunk c, the threads stage chunk c + 1;
//   * one thread issues the MMAs; tcgen05.commit signals their completion on an
//     mbarrier; the accumulator (128 lanes x BN columns of TMEM) is read back with
//     tcgen05.ld and written out through shared memory with coalesced stores.
// Every wait is bounded: on timeout the kernel records an error flag, waits (bounded)
// for its own copies and MMAs in flight, skips its stores and still frees TMEM.
#include <algorithm>
#include <cstdint>

#include "internal.hpp"

namespace ncs {

namespace {

constexpr int TC_BM = 128;   // rows per CTA (TMEM lanes)
constexpr int TC_KC = 32;    // K elements per chunk (4 MMA k-steps of 8)
constexpr int TC_THREADS = 128;
constexpr uint32_t kSpinLimit = 1u << 26;
constexpr uint32_t kAStageBytes = TC_BM * TC_KC * 4;  // one TF32 plane of an A chunk

__host__ __device__ constexpr uint32_t b_block_bytes(int BN) { return 2u * BN * TC_KC * 4; }
__host__ __device__ constexpr uint32_t stage_bytes(int BN) { return 2 * kAStageBytes + b_block_bytes(BN); }

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

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok = 0;
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Bulk (non-tensor) TMA copy global -> shared completing on an mbarrier; both addresses
// 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Offset (bytes) of element (r, k) of a rows x TC_KC tile in the core-matrix layout:
// core matrix (r/8, k/4) at ((r/8) * (TC_KC/4) + k/4) * 128, row r%8 at 16 * (r%8),
// element k%4 at 4 * (k%4). K-direction core stride (LBO) = 128 B, M/N-direction
// stride (SBO) = (TC_KC/4) * 128 B.
__host__ __device__ __forceinline__ uint32_t tile_off(int r, int k) {
  return (uint32_t)((((r >> 3) * (TC_KC >> 2) + (k >> 2)) << 7) + ((r & 7) << 4) + ((k & 3) << 2));
}

// Packs B (cols x Kd, row-major FP32, leading dimension ldb) into TF32 hi/lo blocks:
// block (t, c) = [hi tile | lo tile] of columns t*BN.. and K range c*TC_KC.., each tile
// BN x TC_KC words at tile_off positions, zero beyond cols and Kd.
__global__ void tc_pack_kernel(const float* __restrict__ B, int cols, int Kd, int64_t ldb, int BN, int nch,
                               int ntile, uint32_t* __restrict__ out) {
  const int64_t per = (int64_t)BN * TC_KC;
  const int64_t total = (int64_t)ntile * nch * per;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = i / per;
    const int e = (int)(i - blk * per);
    const int r = e / TC_KC, k = e - r * TC_KC;
    const int t = (int)(blk / nch), c = (int)(blk - (int64_t)t * nch);
    const int col = t * BN + r, kk = c * TC_KC + k;
    const float v = (col < cols && kk < Kd) ? B[(int64_t)col * ldb + kk] : 0.0f;
    const uint32_t h = to_tf32(v);
    const uint32_t l = to_tf32(v - __uint_as_float(h));
    uint32_t* base = out + blk * 2 * per;
    base[tile_off(r, k) >> 2] = h;
    base[per + (tile_off(r, k) >> 2)] = l;
  }
}

// Stages an A chunk (TC_BM rows x TC_KC columns from k0) as TF32 hi/lo planes; each
// warp store writes one 128-byte core matrix (8 rows x 4 elements).
template <typename TA>
__device__ __forceinline__ void stage_a(const TA* __restrict__ A, int64_t lda, int64_t rows, int Kd, int64_t r0,
                                        int k0, uint8_t* hi, uint8_t* lo) {
#pragma unroll 8
  for (int it = 0; it < (TC_BM * TC_KC) / TC_THREADS; ++it) {
    const int idx = it * TC_THREADS + threadIdx.x;
    const int ln = idx & 31, rest = idx >> 5;
    const int rr = ln >> 2, kk = ln & 3, rg = rest >> 3, kg = rest & 7;
    const int r = rg * 8 + rr, k = kg * 4 + kk;
    float v = 0.0f;
    if (r0 + r < rows && k0 + k < Kd) v = (float)A[(r0 + r) * lda + k0 + k];
    const uint32_t h = to_tf32(v);
    const uint32_t l = to_tf32(v - __uint_as_float(h));
    const uint32_t o = ((uint32_t)(rg * 8 + kg) << 7) + ((uint32_t)rr << 4) + ((uint32_t)kk << 2);
    *reinterpret_cast<uint32_t*>(hi + o) = h;
    *reinterpret_cast<uint32_t*>(lo + o) = l;
  }
}

template <typename TA, int BN>
__global__ void __launch_bounds__(TC_THREADS) tc_gemm_kernel(int64_t rows, int cols, int Kd,
                                                             const TA* __restrict__ A, int64_t lda,
                                                             const uint32_t* __restrict__ Bpack, float* __restrict__ D,
                                                             int64_t ldd, const double* __restrict__ addx,
                                                             double* __restrict__ Dd, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char tc_smem_raw[];
  uint8_t* sm = tc_smem_raw + ((1024u - (smem_u32(tc_smem_raw) & 1023u)) & 1023u);
  __shared__ uint64_t full[2], done[2];
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  constexpr uint32_t SB = stage_bytes(BN);
  constexpr uint32_t NCOL = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  constexpr uint32_t idesc = idesc_tf32(TC_BM, BN);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ct = blockIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * TC_BM;
  const int c0 = ct * BN;
  const int nch = (Kd + TC_KC - 1) / TC_KC;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(NCOL));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&done[s], 1);
    }
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  // thread 0's record of asynchronous work in flight (for the bounded clean-up)
  int copy_pending = -1, commit_last = -1;
  for (int ch = 0; ch < nch; ++ch) {
    const int s = ch & 1;
    uint8_t* Ahi = sm + s * SB;
    uint8_t* Alo = Ahi + kAStageBytes;
    uint8_t* Bs = Alo + kAStageBytes;
    __syncthreads();  // publishes thread 0's `failed`
    if (failed) break;
    // stage s is free again once the MMAs of chunk ch - 2 have completed
    if (ch >= 2 && threadIdx.x == 0 && !mbar_wait(&done[s], ((ch >> 1) - 1) & 1)) failed = 1;
    __syncthreads();
    if (failed) break;
    if (threadIdx.x == 0) {
      mbar_expect_tx(&full[s], b_block_bytes(BN));
      bulk_g2s(Bs, Bpack + ((int64_t)ct * nch + ch) * (b_block_bytes(BN) / 4), b_block_bytes(BN), &full[s]);
      copy_pending = ch;
    }
    stage_a<TA>(A, lda, rows, Kd, r0, ch * TC_KC, Ahi, Alo);
    // make the generic-proxy smem writes visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (threadIdx.x == 0) {
      if (!mbar_wait(&full[s], (ch >> 1) & 1)) {
        failed = 1;
      } else {
        copy_pending = -1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        constexpr uint32_t sbo = (TC_KC / 4) * 128;
        const uint32_t ah0 = smem_u32(Ahi), al0 = smem_u32(Alo), bh0 = smem_u32(Bs);
        const uint32_t bl0 = bh0 + (uint32_t)BN * TC_KC * 4;
        for (int ks = 0; ks < TC_KC / 8; ++ks) {
          const uint32_t koff = (uint32_t)ks * 2 * 128;  // two core matrices (8 tf32) per k-step
          const uint64_t ah = smem_desc(ah0 + koff, 128, sbo), al = smem_desc(al0 + koff, 128, sbo);
          const uint64_t bh = smem_desc(bh0 + koff, 128, sbo), bl = smem_desc(bl0 + koff, 128, sbo);
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
            smem_u32(&done[s])));
        commit_last = ch;
      }
    }
  }
  __syncthreads();
  if (!failed) {
    // the last commit completes when every MMA issued before it has completed
    const int L = nch - 1;
    if (threadIdx.x == 0 && !mbar_wait(&done[L & 1], (L >> 1) & 1)) failed = 1;
    __syncthreads();
  }
  if (failed) {
    if (threadIdx.x == 0) {
      // bounded clean-up: let the bulk copy and the MMAs already issued land
      if (copy_pending >= 0) mbar_wait(&full[copy_pending & 1], (copy_pending >> 1) & 1);
      if (commit_last >= 0) mbar_wait(&done[commit_last & 1], (commit_last >> 1) & 1);
      atomicExch(err, 1);
    }
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;");
    // epilogue: warp w owns TMEM lanes (tile rows) 32w..32w+31; each 32-column slice is
    // transposed through shared memory so that one warp store covers a row segment
    float* tile = reinterpret_cast<float*>(sm) + warp * 32 * 33;
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
#pragma unroll
      for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = __uint_as_float(v[j]);
      __syncwarp();
      const int c = c0 + cb + lane;
      const bool cok = (cb + lane < BN) && (c < cols);
      for (int rr = 0; rr < 32; ++rr) {
        const int64_t r = r0 + warp * 32 + rr;
        if (cok && r < rows) {
          const float val = tile[rr * 33 + lane];
          if (Dd)
            Dd[r * ldd + c] = addx[r * ldd + c] + (double)val;
          else
            D[r * ldd + c] = val;
        }
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL));
}

template <typename TA, int BN>
cudaError_t launch(int64_t rows, int cols, int Kd, const TA* A, int64_t lda, const uint32_t* Bpack, float* D,
                   int64_t ldd, const double* addx, double* Dd, int* err, cudaStream_t s) {
  const size_t smem = (size_t)2 * stage_bytes(BN) + 1024;
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<TA, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t rt = (rows + TC_BM - 1) / TC_BM;
  if (rt > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)((cols + BN - 1) / BN), (unsigned)rt);
  count_launch(), tc_gemm_kernel<TA, BN><<<grid, TC_THREADS, smem, s>>>(rows, cols, Kd, A, lda, Bpack, D, ldd, addx,
                                                                        Dd, err);
  return cudaGetLastError();
}

template <typename TA>
cudaError_t launch_bn(int BN, int64_t rows, int cols, int Kd, const TA* A, int64_t lda, const uint32_t* Bpack,
                      float* D, int64_t ldd, const double* addx, double* Dd, int* err, cudaStream_t s) {
  switch (BN) {
    case 64: return launch<TA, 64>(rows, cols, Kd, A, lda, Bpack, D, ldd, addx, Dd, err, s);
    case 128: return launch<TA, 128>(rows, cols, Kd, A, lda, Bpack, D, ldd, addx, Dd, err, s);
    case 144: return launch<TA, 144>(rows, cols, Kd, A, lda, Bpack, D, ldd, addx, Dd, err, s);
    case 256: return launch<TA, 256>(rows, cols, Kd, A, lda, Bpack, D, ldd, addx, Dd, err, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int tc_block_cols(int cols) {
  return cols <= 64 ? 64 : (cols <= 128 ? 128 : (cols <= 144 ? 144 : (cols <= 256 ? 256 : 128)));
}

int64_t tc_pack_words(int cols, int Kd) {
  const int BN = tc_block_cols(cols);
  const int64_t ntile = (cols + BN - 1) / BN, nch = (Kd + TC_KC - 1) / TC_KC;
  return ntile * nch * 2 * (int64_t)BN * TC_KC;
}

cudaError_t launch_tc_pack(const float* B, int cols, int Kd, uint32_t* out, cudaStream_t s) {
  const int BN = tc_block_cols(cols);
  const int ntile = (cols + BN - 1) / BN, nch = (Kd + TC_KC - 1) / TC_KC;
  const int64_t total = (int64_t)ntile * nch * BN * TC_KC;
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 8));
  count_launch(), tc_pack_kernel<<<blocks, 256, 0, s>>>(B, cols, Kd, Kd, BN, nch, ntile, out);
  return cudaGetLastError();
}

// rho32 = X T_all^T (FP32 result), X: N x K FP64, T_all packed (p_total columns).
cudaError_t launch_tc_outgoing(const DeviceData& d, const double* x, int* err, cudaStream_t s) {
  return launch_bn<double>(tc_block_cols(d.p), d.N, d.p, d.K, x, d.K, d.Tpack, d.rho32, d.p, nullptr, nullptr, err,
                           s);
}

// y = x + Z P^T, Z: N x Kstar FP64, P packed (K columns), y, x: N x K FP64.
cudaError_t launch_tc_apply_P(const DeviceData& d, const double* x, double* y, int* err, cudaStream_t s) {
  return launch_bn<double>(tc_block_cols(d.K), d.N, d.K, d.Kstar, d.z, d.Kstar, d.Ppack, nullptr, d.K, x, y, err,
                           s);
}

// D = A B^T with FP32 A (rows x Kd) and B packed by launch_tc_pack (cols columns).
cudaError_t launch_tc_gemm_f32(int64_t rows, int cols, int Kd, const float* A, const uint32_t* Bpack, float* D,
                               int* err, cudaStream_t s) {
  return launch_bn<float>(tc_block_cols(cols), rows, cols, Kd, A, Kd, Bpack, D, cols, nullptr, nullptr, err, s);
}

}  // namespace ncs
