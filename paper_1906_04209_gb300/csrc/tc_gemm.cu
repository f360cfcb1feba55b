// Tensor-core (tcgen05, kind::tf32) GEMM for the per-patch operator contractions of the
// FP32 product (Kaye & Greengard, Section 7, Steps 3.1 and 3.5):
//     rho (N x p_total) = X (N x K) T_all^T          (outgoing coefficients, eq. Tmap)
//     y   (N x K)       = X + Z (N x K*) P^T         (Zernike transform P)
// D = A B^T with A (rows x Kd) and B (cols x Kd), both K-major. Accuracy: both operands
// are split into TF32 pairs (hi = tf32(v), lo = tf32(v - hi)) and the tensor cores
// accumulate hi*hi + hi*lo + lo*hi in FP32 ("3xTF32", about FP32 accuracy).
//
// Data movement (all operand traffic by TMA):
//   * tc_pack_kernel splits an operand and lays it out in the canonical no-swizzle K-major
//     shared-memory layout (8-row x 16-byte core matrices), one contiguous block per
//     (128- or BN-row tile, 32-wide K chunk): once for the constant operators, once per
//     product for X or Z (a streaming, HBM-bound pass);
//   * one thread runs an S-stage pipeline: a bulk TMA copy (cp.async.bulk) per operand
//     block completing on the stage's mbarrier (transaction count), then the MMAs of
//     that chunk and a tcgen05.commit that frees the stage;
//   * the accumulator (128 lanes x BN columns of TMEM) is read back with tcgen05.ld and
//     written out through shared memory with coalesced stores.
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

__host__ __device__ constexpr uint32_t b_block_bytes(int BN) { return 2u * BN * TC_KC * 4; }

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

// Packs a row-major operand (nrows x Kd, leading dimension ld, FP32 or FP64) into TF32
// hi/lo blocks: block (t, c) = [hi tile | lo tile] of rows t*H.. and K range c*TC_KC..,
// each tile H x TC_KC words at tile_off positions, zero beyond nrows and Kd. Lanes map to
// (8 rows x 4 columns) so that each warp reads 32-byte row segments and writes one
// 128-byte core matrix.
template <typename T>
__global__ void tc_pack_kernel(const T* __restrict__ src, int64_t nrows, int Kd, int64_t ld, int H, int nch,
                               int64_t ntile, uint32_t* __restrict__ out) {
  const int64_t per = (int64_t)H * TC_KC;
  const int64_t total = ntile * nch * per;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = i / per;
    const int e = (int)(i - blk * per);
    const int ln = e & 31, rest = e >> 5;
    const int rr = ln >> 2, kk = ln & 3, rg = rest >> 3, kg = rest & 7;
    const int r = rg * 8 + rr, k = kg * 4 + kk;
    const int64_t t = blk / nch;
    const int c = (int)(blk - t * nch);
    const int64_t row = t * H + r;
    const int col = c * TC_KC + k;
    const float v = (row < nrows && col < Kd) ? (float)src[row * ld + col] : 0.0f;
    const uint32_t h = to_tf32(v);
    const uint32_t l = to_tf32(v - __uint_as_float(h));
    const uint32_t o = tile_off(r, k) >> 2;
    uint32_t* base = out + blk * 2 * per;
    base[o] = h;
    base[per + o] = l;
  }
}

constexpr uint32_t kABlockBytes = 2u * TC_BM * TC_KC * 4;  // hi + lo tiles of a 128-row block

// Pipeline depth for a given tile width: as many stages as fit in 200 KB.
__host__ __device__ constexpr int tc_stages(int BN) {
  return (int)((200u * 1024u) / (kABlockBytes + b_block_bytes(BN))) < 4
             ? (int)((200u * 1024u) / (kABlockBytes + b_block_bytes(BN)))
             : 4;
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS) tc_gemm_kernel(int64_t rows, int cols, int nch,
                                                             const uint32_t* __restrict__ Apack,
                                                             const uint32_t* __restrict__ Bpack, float* __restrict__ D,
                                                             int64_t ldd, const double* __restrict__ addx,
                                                             double* __restrict__ Dd, int* __restrict__ err) {
  constexpr int S = tc_stages(BN);
  constexpr uint32_t SB = kABlockBytes + b_block_bytes(BN);
  constexpr uint32_t NCOL = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  constexpr uint32_t idesc = idesc_tf32(TC_BM, BN);
  extern __shared__ __align__(128) unsigned char tc_smem_raw[];
  uint8_t* sm = tc_smem_raw + ((1024u - (smem_u32(tc_smem_raw) & 1023u)) & 1023u);
  __shared__ uint64_t full[S], done[S];
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ct = blockIdx.x;
  const int64_t rt = blockIdx.y;
  const int64_t r0 = rt * TC_BM;
  const int c0 = ct * BN;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(NCOL));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
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
  if (threadIdx.x == 0) {
    // producer and MMA issuer: copies for up to S chunks in flight
    int issued = 0, waited_copy = 0, committed = 0, waited_mma = 0;
    auto issue = [&](int ch) {
      const int s = ch % S;
      uint8_t* st = sm + s * SB;
      mbar_expect_tx(&full[s], SB);
      bulk_g2s(st, Apack + (rt * nch + ch) * (int64_t)(kABlockBytes / 4), kABlockBytes, &full[s]);
      bulk_g2s(st + kABlockBytes, Bpack + ((int64_t)ct * nch + ch) * (b_block_bytes(BN) / 4), b_block_bytes(BN),
               &full[s]);
    };
    for (; issued < S && issued < nch; ++issued) issue(issued);
    constexpr uint32_t sbo = (TC_KC / 4) * 128;
    for (int ch = 0; ch < nch; ++ch) {
      const int s = ch % S;
      const uint32_t par = (uint32_t)(ch / S) & 1u;
      if (!mbar_wait(&full[s], par)) {
        failed = 1;
        break;
      }
      waited_copy = ch + 1;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t ah0 = smem_u32(sm + s * SB);
      const uint32_t al0 = ah0 + kABlockBytes / 2;
      const uint32_t bh0 = ah0 + kABlockBytes;
      const uint32_t bl0 = bh0 + b_block_bytes(BN) / 2;
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
      committed = ch + 1;
      if (issued < nch) {
        // stage s is refilled once the MMAs just issued from it have completed
        if (!mbar_wait(&done[s], par)) {
          failed = 1;
          break;
        }
        waited_mma = ch + 1;
        issue(issued++);
      }
    }
    if (!failed && committed > waited_mma) {
      // the last commit completes when every MMA issued before it has completed
      const int L = committed - 1;
      if (!mbar_wait(&done[L % S], (uint32_t)(L / S) & 1u)) failed = 1;
      else waited_mma = committed;
    }
    if (failed) {
      // bounded clean-up: let the copies and MMAs already issued land
      for (int ch = waited_copy; ch < issued; ++ch) mbar_wait(&full[ch % S], (uint32_t)(ch / S) & 1u);
      if (committed > waited_mma) {
        const int L = committed - 1;
        mbar_wait(&done[L % S], (uint32_t)(L / S) & 1u);
      }
      atomicExch(err, 1);
    }
  }
  __syncthreads();
  if (!failed) {
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

template <int BN>
cudaError_t launch(int64_t rows, int cols, int Kd, const uint32_t* Apack, const uint32_t* Bpack, float* D,
                   int64_t ldd, const double* addx, double* Dd, int* err, cudaStream_t s) {
  const size_t smem = (size_t)tc_stages(BN) * (kABlockBytes + b_block_bytes(BN)) + 1024;
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t rt = (rows + TC_BM - 1) / TC_BM;
  if (rt > 65535) return cudaErrorInvalidConfiguration;
  const int nch = (Kd + TC_KC - 1) / TC_KC;
  dim3 grid((unsigned)((cols + BN - 1) / BN), (unsigned)rt);
  count_launch(), tc_gemm_kernel<BN><<<grid, TC_THREADS, smem, s>>>(rows, cols, nch, Apack, Bpack, D, ldd, addx, Dd,
                                                                    err);
  return cudaGetLastError();
}

cudaError_t launch_bn(int BN, int64_t rows, int cols, int Kd, const uint32_t* Apack, const uint32_t* Bpack,
                      float* D, int64_t ldd, const double* addx, double* Dd, int* err, cudaStream_t s) {
  switch (BN) {
    case 64: return launch<64>(rows, cols, Kd, Apack, Bpack, D, ldd, addx, Dd, err, s);
    case 128: return launch<128>(rows, cols, Kd, Apack, Bpack, D, ldd, addx, Dd, err, s);
    case 144: return launch<144>(rows, cols, Kd, Apack, Bpack, D, ldd, addx, Dd, err, s);
    case 256: return launch<256>(rows, cols, Kd, Apack, Bpack, D, ldd, addx, Dd, err, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t pack(const T* src, int64_t nrows, int Kd, int64_t ld, int H, uint32_t* out, cudaStream_t s) {
  const int64_t ntile = (nrows + H - 1) / H;
  const int nch = (Kd + TC_KC - 1) / TC_KC;
  const int64_t total = ntile * nch * (int64_t)H * TC_KC;
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
  count_launch(), tc_pack_kernel<T><<<blocks, 256, 0, s>>>(src, nrows, Kd, ld, H, nch, ntile, out);
  return cudaGetLastError();
}

}  // namespace

int tc_block_cols(int cols) {
  return cols <= 64 ? 64 : (cols <= 128 ? 128 : (cols <= 144 ? 144 : (cols <= 256 ? 256 : 128)));
}

int64_t tc_pack_words(int64_t nrows, int Kd, int H) {
  const int64_t ntile = (nrows + H - 1) / H, nch = (Kd + TC_KC - 1) / TC_KC;
  return ntile * nch * 2 * (int64_t)H * TC_KC;
}

cudaError_t launch_tc_pack_b(const float* B, int cols, int Kd, uint32_t* out, cudaStream_t s) {
  return pack<float>(B, cols, Kd, Kd, tc_block_cols(cols), out, s);
}

// rho32 = X T_all^T (FP32 result), X: N x K FP64 (packed into Apack), T_all packed.
cudaError_t launch_tc_outgoing(const DeviceData& d, const double* x, int* err, cudaStream_t s) {
  cudaError_t e = pack<double>(x, d.N, d.K, d.K, TC_BM, d.Apack, s);
  if (e != cudaSuccess) return e;
  return launch_bn(tc_block_cols(d.p), d.N, d.p, d.K, d.Apack, d.Tpack, d.rho32, d.p, nullptr, nullptr, err, s);
}

// y = x + Z P^T, Z: N x Kstar FP64 (packed into Apack), P packed, y, x: N x K FP64.
cudaError_t launch_tc_apply_P(const DeviceData& d, const double* x, double* y, int* err, cudaStream_t s) {
  cudaError_t e = pack<double>(d.z, d.N, d.Kstar, d.Kstar, TC_BM, d.Apack, s);
  if (e != cudaSuccess) return e;
  return launch_bn(tc_block_cols(d.K), d.N, d.K, d.Kstar, d.Apack, d.Ppack, nullptr, d.K, x, y, err, s);
}

// D = A B^T with FP32 A (rows x Kd, packed here into Apack) and B packed by
// launch_tc_pack_b (cols columns).
cudaError_t launch_tc_gemm_f32(int64_t rows, int cols, int Kd, const float* A, uint32_t* Apack,
                               const uint32_t* Bpack, float* D, int* err, cudaStream_t s) {
  cudaError_t e = pack<float>(A, rows, Kd, Kd, TC_BM, Apack, s);
  if (e != cudaSuccess) return e;
  return launch_bn(tc_block_cols(cols), rows, cols, Kd, Apack, Bpack, D, cols, nullptr, nullptr, err, s);
}

}  // namespace ncs
