// The modal collocation matrices of the one-patch solve on the device (see onepatch.hpp),
// FP64 throughout. One block per (row i, panel j), four warps; each warp takes its
// quadrature nodes 32 at a time:
//   * every lane forms one node's G^(1) + s G^(2) modes (elliptic integrals and the
//     three-term recurrence, the serial part) and its Lagrange values;
//   * then, node by node, the warp sums G^(3)_n = sum over the theta rule of
//     log(1 + d/2) cos(n theta) w / pi with the theta nodes spread over the lanes and the
//     modes in registers, reduces across the lanes, and adds wt L_k G_n into its
//     (mode, column) accumulators in shared memory;
//   * the four warps' accumulators are summed and written to the block's nord columns of
//     row i of every A_n (each entry written once, no atomics).
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "internal.hpp"
#include "modal.hpp"
#include "onepatch.hpp"

namespace ncs {

namespace {

constexpr int CO_WARPS = 4;
constexpr int CO_THREADS = 32 * CO_WARPS;
constexpr int CO_MAXORD = kCollocMaxOrd;

struct CollocArgs {
  int nr, npan, nord, nmodes, nth;
  double sgn;
  const double* tr;
  const double* colscale;
  const double* lag_nodes;
  const double* lag_bw;
  const int* qoff;
  const double* tq;
  const double* wt;
  const double* ls;
  const double* hs2;
  const double* cw;
  double* A;
};

// per warp: accumulators NM x CO_MAXORD, node modes 32 x NM, Lagrange values 32 x CO_MAXORD,
// node (t', weight) 32 x 2
template <int NM>
constexpr int colloc_warp_doubles() {
  return NM * CO_MAXORD + 32 * NM + 32 * CO_MAXORD + 64;
}

template <int NM>
__global__ void __launch_bounds__(CO_THREADS) colloc_kernel(CollocArgs a) {
  extern __shared__ double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m1 = a.nmodes, nord = a.nord, ne = m1 * nord;
  double* sacc = sm + warp * (NM * CO_MAXORD);
  double* sg = sm + CO_WARPS * (NM * CO_MAXORD) + warp * (32 * NM);
  double* sl = sm + CO_WARPS * (NM * CO_MAXORD + 32 * NM) + warp * (32 * CO_MAXORD);
  double* sq = sm + CO_WARPS * (NM * CO_MAXORD + 32 * NM + 32 * CO_MAXORD) + warp * 64;
  const int b = blockIdx.x, i = b / a.npan, j = b - i * a.npan;
  const bool jac = (j == a.npan - 1);
  const double ti = a.tr[i], sti = sin(ti);
  const double* xn = a.lag_nodes + (jac ? nord : 0);
  const double* bw = a.lag_bw + (jac ? nord : 0);
  const double* cs = a.colscale + j * nord;
  for (int e = lane; e < ne; e += 32) sacc[e] = 0.0;
  const int qa = a.qoff[b], qb = a.qoff[b + 1];
  for (int q0 = qa + 32 * warp; q0 < qb; q0 += 32 * CO_WARPS) {
    const int cnt = min(32, qb - q0);
    if (lane < cnt) {
      const int q = q0 + lane;
      const double tq = a.tq[q];
      double* g = sg + lane * NM;
      modal::coulomb_modes<NM>(ti, tq, m1 - 1, g);
      modal::log_modes_add(ti, tq, m1 - 1, a.sgn, g);
      double* L = sl + lane * CO_MAXORD;
      const double s = a.ls[q];
      int hit = -1;
      for (int k = 0; k < nord; ++k)
        if (s == xn[k]) hit = k;
      if (hit >= 0) {
        for (int k = 0; k < nord; ++k) L[k] = (k == hit) ? cs[k] : 0.0;
      } else {
        double den = 0.0;
        for (int k = 0; k < nord; ++k) {
          L[k] = bw[k] / (s - xn[k]);
          den += L[k];
        }
        for (int k = 0; k < nord; ++k) L[k] = L[k] / den * cs[k];
      }
      sq[2 * lane] = tq;
      sq[2 * lane + 1] = a.wt[q];
    }
    __syncwarp();
    for (int u = 0; u < cnt; ++u) {
      const double tq = sq[2 * u];
      const double sh = sin(0.5 * (ti - tq));
      const double A4 = 4.0 * sh * sh, B4 = 4.0 * sti * sin(tq);
      double part[NM];
#pragma unroll
      for (int n = 0; n < NM; ++n) part[n] = 0.0;
      for (int it = lane; it < a.nth; it += 32) {
        const double gq = log1p(0.5 * sqrt(A4 + B4 * a.hs2[it]));
        const double* c = a.cw + (size_t)it * m1;
#pragma unroll
        for (int n = 0; n < NM; ++n)
          if (n < m1) part[n] = fma(gq, c[n], part[n]);
      }
#pragma unroll
      for (int n = 0; n < NM; ++n) {
        if (n < m1) {
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) part[n] += __shfl_xor_sync(0xffffffffu, part[n], off);
        }
      }
      double* g = sg + u * NM;
      if (lane == 0) {
#pragma unroll
        for (int n = 0; n < NM; ++n)
          if (n < m1) g[n] -= part[n];
      }
      __syncwarp();
      const double w = sq[2 * u + 1];
      const double* L = sl + u * CO_MAXORD;
      for (int e = lane; e < ne; e += 32) {
        const int n = e / nord, k = e - n * nord;
        sacc[e] = fma(w * L[k], g[n], sacc[e]);
      }
    }
    __syncwarp();
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ne; e += CO_THREADS) {
    double v = 0.0;
    for (int w = 0; w < CO_WARPS; ++w) v += sm[w * (NM * CO_MAXORD) + e];
    const int n = e / nord, k = e - n * nord;
    a.A[((size_t)n * a.nr + i) * a.nr + j * nord + k] = v;
  }
}

template <int NM>
cudaError_t launch_colloc(const CollocArgs& a, int nblocks, cudaStream_t s) {
  const size_t smem = sizeof(double) * CO_WARPS * (size_t)colloc_warp_doubles<NM>();
  cudaError_t e = cudaFuncSetAttribute(colloc_kernel<NM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launch(), colloc_kernel<NM><<<nblocks, CO_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

int colloc_assemble_device(const CollocProblem& p, std::vector<double>& A, std::string* err) {
  if (p.nord < 1 || p.nord > CO_MAXORD || p.nmodes < 1 || p.nmodes > kCollocMaxModes || p.nr != p.npan * p.nord)
    return 0;
  const int nb = p.nr * p.npan;
  if ((int)p.qoff.size() != nb + 1 || (int)p.tr.size() != p.nr || (int)p.colscale.size() != p.nr ||
      (int)p.lag_nodes.size() != 2 * p.nord || (int)p.lag_bw.size() != 2 * p.nord)
    return 0;
  const int nq = p.qoff[nb], nth = (int)p.hs2.size();
  if ((int)p.tq.size() != nq || (int)p.wt.size() != nq || (int)p.ls.size() != nq ||
      p.cw.size() != (size_t)nth * p.nmodes || nth < 1)
    return 0;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();  // clear the error state of a machine without a device
    return 0;
  }
  // one allocation: the doubles, then A, then the offsets
  const size_t nin = (size_t)p.nr * 2 + 4 * (size_t)p.nord + 3 * (size_t)nq + nth + p.cw.size();
  const size_t nA = (size_t)p.nmodes * p.nr * p.nr;
  const size_t bytes = (nin + nA) * sizeof(double) + (size_t)(nb + 1) * sizeof(int);
  cudaStream_t s = nullptr;
  char* buf = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaMalloc(&buf, bytes) != cudaSuccess) {
    // no room or no usable device: the host loop forms the matrices, as for the ID sketch
    if (s) cudaStreamDestroy(s);
    cudaGetLastError();
    return 0;
  }
  cudaError_t e = cudaSuccess;
  double* d = reinterpret_cast<double*>(buf);
  CollocArgs a{};
  {
    size_t off = 0;
    auto put = [&](const std::vector<double>& v) -> const double* {
      double* dst = d + off;
      off += v.size();
      if (e == cudaSuccess && !v.empty())
        e = cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice, s);
      return dst;
    };
    a.nr = p.nr;
    a.npan = p.npan;
    a.nord = p.nord;
    a.nmodes = p.nmodes;
    a.nth = nth;
    a.sgn = (p.mode == 0) ? -1.0 : 1.0;
    a.tr = put(p.tr);
    a.colscale = put(p.colscale);
    a.lag_nodes = put(p.lag_nodes);
    a.lag_bw = put(p.lag_bw);
    a.tq = put(p.tq);
    a.wt = put(p.wt);
    a.ls = put(p.ls);
    a.hs2 = put(p.hs2);
    a.cw = put(p.cw);
    a.A = d + nin;
    int* qo = reinterpret_cast<int*>(d + nin + nA);
    a.qoff = qo;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(qo, p.qoff.data(), (size_t)(nb + 1) * sizeof(int), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) {
    if (p.nmodes <= 16)
      e = launch_colloc<16>(a, nb, s);
    else if (p.nmodes <= 32)
      e = launch_colloc<32>(a, nb, s);
    else
      e = launch_colloc<64>(a, nb, s);
  }
  if (e == cudaSuccess) {
    A.resize(nA);
    e = cudaMemcpyAsync(A.data(), a.A, nA * sizeof(double), cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (buf) cudaFree(buf);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) {
    if (err) *err = std::string("collocation matrices on the device: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return -1;
  }
  return 1;
}

}  // namespace ncs
