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

// Non-negative doubles order like their bit patterns, so atomicMax on the bits is a max.
__global__ void maxabs_diff_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                   unsigned long long* __restrict__ out) {
  double d = 0.0, m = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    d = fmax(d, fabs(a[i] - b[i]));
    m = fmax(m, fabs(b[i]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    d = fmax(d, __shfl_down_sync(0xffffffffu, d, o));
    m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  }
  if ((threadIdx.x & 31) == 0) {
    // a NaN difference is reported as +Inf (the largest bit pattern atomicMax keeps)
    atomicMax(out, (unsigned long long)__double_as_longlong(d == d ? d : INFINITY));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(m));
  }
}

cudaError_t launch_maxabs_diff(int64_t n, const double* a, const double* b, double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 4);
  count_launch(), maxabs_diff_kernel<<<(unsigned)std::max<int64_t>(1, blocks), 256, 0, s>>>(
      n, a, b, reinterpret_cast<unsigned long long*>(out));
  return cudaGetLastError();
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

// ---- GMRES with its whole state on the device (Section 7, Step 3: the Krylov solve
// of the second-kind system). One Arnoldi step is a fixed sequence of launches whose
// arguments never change: the column index lives in GmresState::m, the product reads a
// fixed copy `vk` of the newest basis vector, so the step can be captured once as a CUDA
// graph and replayed. Classical Gram-Schmidt is applied twice; the Givens rotations, the
// residual estimate and the back substitution run on the device in FP64.
namespace ncs {

// partial[j * kDotChunks + c] = chunk c of V_j . w for j <= m (the column in progress)
__global__ void __launch_bounds__(256) arnoldi_dots_kernel(int64_t n, const double* __restrict__ V, int64_t ld,
                                                           const double* __restrict__ w,
                                                           const GmresState* __restrict__ st,
                                                           double* __restrict__ partial) {
  if (st->done) return;
  const int k = st->m;
  __shared__ double red[256];
  const int c = blockIdx.x;
  const int64_t chunk = (n + kDotChunks - 1) / kDotChunks;
  const int64_t lo = c * chunk, hi = min(n, lo + chunk);
  for (int j = blockIdx.y; j <= k; j += gridDim.y) {
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
    __syncthreads();
  }
}

// h_j = sum_c partial[j, c] (kept in hout by block 0), w -= sum_j h_j V_j, and per block
// the partial sum of the updated |w_i|^2 (pnorm[blockIdx.x]); fixed grid, fixed order.
__global__ void __launch_bounds__(256) arnoldi_update_kernel(int64_t n, const double* __restrict__ V, int64_t ld,
                                                             double* __restrict__ w,
                                                             const GmresState* __restrict__ st,
                                                             const double* __restrict__ partial,
                                                             double* __restrict__ hout, double* __restrict__ pnorm) {
  if (st->done) return;
  const int k = st->m;
  extern __shared__ double hs[];
  __shared__ double red[256];
  for (int j = threadIdx.x; j <= k; j += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < kDotChunks; ++c) s += partial[j * kDotChunks + c];
    hs[j] = s;
    if (blockIdx.x == 0) hout[j] = s;
  }
  __syncthreads();
  double nrm = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j <= k; ++j) acc = fma(hs[j], V[j * ld + i], acc);
    const double wi = w[i] - acc;
    w[i] = wi;
    nrm = fma(wi, wi, nrm);
  }
  red[threadIdx.x] = nrm;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) pnorm[blockIdx.x] = red[0];
}

// Column m of the Hessenberg matrix (h1 + h2 from the two Gram-Schmidt passes, the norm
// of the new vector), the previous rotations applied to it, a new rotation zeroing its
// subdiagonal, the rotated right-hand side g and the residual estimate |g_{m+1}| / beta.
// One warp; lane 0 runs the (inherently sequential) rotations.
__global__ void givens_kernel(GmresState* __restrict__ st, double* __restrict__ H, int ldh, double* __restrict__ cs,
                              double* __restrict__ sn, double* __restrict__ g, const double* __restrict__ h1,
                              const double* __restrict__ h2, const double* __restrict__ pnorm, int nb) {
  if (st->done) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) s += pnorm[b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x != 0) return;
  const int k = st->m;
  const double hn = sqrt(s);
  double* col = H + (int64_t)k * ldh;
  bool finite = isfinite(hn);
  for (int j = 0; j <= k; ++j) {
    col[j] = h1[j] + h2[j];
    finite = finite && isfinite(col[j]);
  }
  if (k == 0) g[0] = st->beta;
  for (int j = 0; j < k; ++j) {
    const double a = col[j], b = col[j + 1];
    col[j] = cs[j] * a + sn[j] * b;
    col[j + 1] = -sn[j] * a + cs[j] * b;
  }
  const double a = col[k], b = hn;
  const double rr = hypot(a, b);
  st->hn = hn;
  st->m = k + 1;
  if (!finite || !(rr > 0.0)) {
    // a non-finite column, or a zero column (the operator maps the basis vector to 0)
    st->flag = finite ? kGmresBreakdown : kGmresNonFinite;
    st->done = 1;
    st->m = k;  // the column is not usable
    return;
  }
  cs[k] = a / rr;
  sn[k] = b / rr;
  col[k] = rr;
  col[k + 1] = 0.0;
  g[k + 1] = -sn[k] * g[k];
  g[k] = cs[k] * g[k];
  const double res = fabs(g[k + 1]) / st->beta;
  st->res = res;
  if (res <= st->tol) {
    st->flag = kGmresConverged;
    st->done = 1;
  } else if (hn == 0.0) {
    st->flag = kGmresHappy;  // the Krylov space is invariant: the iterate is exact
    st->done = 1;
  } else if (k + 1 >= st->maxit) {
    st->done = 1;
  }
}

// V_{m} = w / hn and the product's input copy vk = V_{m} (m already advanced).
__global__ void arnoldi_normalize_kernel(int64_t n, const double* __restrict__ w, double* __restrict__ V, int64_t ld,
                                         double* __restrict__ vk, const GmresState* __restrict__ st) {
  if (st->done) return;
  const double a = 1.0 / st->hn;
  double* v = V + (int64_t)st->m * ld;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = a * w[i];
    v[i] = x;
    vk[i] = x;
  }
}

// y = R^-1 g for the m x m upper triangle R of the rotated Hessenberg matrix.
__global__ void gmres_backsolve_kernel(const GmresState* __restrict__ st, const double* __restrict__ H, int ldh,
                                       const double* __restrict__ g, double* __restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int m = st->m;
  for (int i = m - 1; i >= 0; --i) {
    double t = g[i];
    for (int j = i + 1; j < m; ++j) t -= H[(int64_t)j * ldh + i] * y[j];
    y[i] = t / H[(int64_t)i * ldh + i];
  }
}

int gmres_update_blocks(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 8); }

cudaError_t launch_arnoldi_orthogonalize(int64_t n, const double* V, double* w, const GmresDev& gd,
                                         cudaStream_t s) {
  const int jg = std::min(gd.maxit + 1, 16);
  const int nb = gmres_update_blocks(n);
  const size_t hsm = (size_t)(gd.maxit + 1) * sizeof(double);
  for (int pass = 0; pass < 2; ++pass) {
    count_launch(), arnoldi_dots_kernel<<<dim3(kDotChunks, jg), 256, 0, s>>>(n, V, n, w, gd.st, gd.partial);
    count_launch(), arnoldi_update_kernel<<<nb, 256, hsm, s>>>(n, V, n, w, gd.st, gd.partial,
                                                                pass == 0 ? gd.h1 : gd.h2, gd.pnorm);
  }
  count_launch(), givens_kernel<<<1, 32, 0, s>>>(gd.st, gd.H, gd.maxit + 1, gd.cs, gd.sn, gd.g, gd.h1, gd.h2,
                                                 gd.pnorm, nb);
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
  count_launch(), arnoldi_normalize_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, w, const_cast<double*>(V), n,
                                                                            gd.vk, gd.st);
  return cudaGetLastError();
}

cudaError_t launch_gmres_backsolve(const GmresDev& gd, cudaStream_t s) {
  count_launch(), gmres_backsolve_kernel<<<1, 32, 0, s>>>(gd.st, gd.H, gd.maxit + 1, gd.g, gd.y);
  return cudaGetLastError();
}

}  // namespace ncs
