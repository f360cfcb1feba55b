// Single-layer potential of one patch at a target close to it (Kaye & Greengard, Section 2,
// eqs. urep and intBVPansatz with the off-surface Green's functions eqs. Gextoffsurface /
// Gintoffsurface): the targets of the paper's mean-first-passage-time maps on the sphere of
// radius 1 - eps/5 (Section 9.2) lie within 2 eps of patches, where the skeleton (far-field)
// representation of Section 7.1 does not hold.
//
// For patch j (centre c, frame e1, e2) with density sigma(t, theta) = sum_k f_k beta_k(t)
// trig(m_k theta) (the one-patch solution of Section 8) and a target x at local polar
// position (t0, theta0) and radius r:
//   S sigma(x) = int_0^eps sum_k f_k beta_k(t) [int_{-pi}^{pi} G(x, y(t, theta0 + phi))
//                trig(m_k (theta0 + phi)) dphi] sin t dt.
// G depends on phi only through cos phi, since
//   |x - y|^2 = (r - 1)^2 + 4 r [sin^2((t0 - t)/2) + sin t0 sin t sin^2(phi/2)]
// (every term non-negative: no cancellation as x approaches the patch), so the inner
// integral is trig(m theta0) C_m(t) with C_m(t) = 2 int_0^pi G cos(m phi) dphi (the odd part
// vanishes on the symmetric rule). The kernel is written through d and r alone,
//   exterior: G_E = 2/d + log((d + r - 1)/(d + r + 1)),
//   interior: G_I = 2/d + log(4/((d + 1 - r)(d + 1 + r))),
// which equal the printed forms and stay accurate as x approaches y.
//
// Quadrature (FP64): in t, the one-patch radial panels, each with a composite Gauss rule
// graded toward the target's t0 (split there when t0 lies inside the panel) down to the
// target's distance from the sphere; on the last panel the density is g / sqrt(eps - t)
// with g polynomial, integrated in u = sqrt(eps - t). beta_k between the panel nodes by
// barycentric Lagrange interpolation. In phi, a composite 12-point Gauss rule graded toward
// phi = 0 with a depth set by the target's distance to the circle t (tables built once
// per context).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "internal.hpp"
#include "numerics.hpp"

namespace ncs {

namespace {

constexpr int kNearThreads = 128;
constexpr int kNearWarps = kNearThreads / 32;
constexpr int kMaxRadNodes = 2048;

// The radial quadrature of one (target, patch) pair, built in shared memory: nodes t,
// weights (with sin t and, on the last panel, the substitution's factor) and panel index.
struct RadialRule {
  double* tq;
  double* wq;
  int* pan;
  int n;
  int overflow;
};

// Appends a composite rule on [a, b] made of ng-point Gauss pieces (nodes gx, weights gw on
// [-1, 1]), graded dyadically toward the endpoint `toward_a ? a : b` with nlev levels; on
// the last panel [a, b] is an interval of u = sqrt(eps - t).
__device__ void add_pieces(RadialRule& R, double a, double b, bool toward_a, int nlev, const double* gx,
                           const double* gw, int ng, int panel, bool jacobi, double eps) {
  const double L = b - a;
  for (int k = 0; k <= nlev; ++k) {
    // piece k spans [L 2^-(nlev-k+1), L 2^-(nlev-k)] from the graded end (piece 0 starts at it)
    const double u0 = (k == 0) ? 0.0 : L * ldexp(1.0, -(nlev - k + 1));
    const double u1 = L * ldexp(1.0, -(nlev - k));
    const double lo = toward_a ? a + u0 : b - u1, hi = toward_a ? a + u1 : b - u0;
    const double h = 0.5 * (hi - lo), m = 0.5 * (hi + lo);
    for (int i = 0; i < ng; ++i) {
      if (R.n >= kMaxRadNodes) {
        R.overflow = 1;
        return;
      }
      const double s = m + h * gx[i], w = h * gw[i];
      if (jacobi) {  // s is u = sqrt(eps - t): t = eps - u^2, dt / sqrt(eps - t) = 2 du
        const double t = eps - s * s;
        R.tq[R.n] = t;
        R.wq[R.n] = 2.0 * w * sin(t);
      } else {
        R.tq[R.n] = s;
        R.wq[R.n] = w * sin(s);
      }
      R.pan[R.n] = panel;
      ++R.n;
    }
  }
}

// The rule of one panel [a, b] (in t, or in u on the Jacobi panel) for a near-singularity
// at s (inside or outside the panel) at distance delta off the real axis.
__device__ void panel_rule(RadialRule& R, double a, double b, double s, double delta, const double* g10,
                           const double* w10, const double* g20, const double* w20, int panel, bool jacobi,
                           double eps) {
  const double L = b - a;
  const double floor_ = fmax(delta, 1e-13 * fmax(fabs(b), fabs(s)));
  if (a < s && s < b) {
    const int n1 = (int)fmin(40.0, fmax(1.0, ceil(log2((s - a) / floor_)) + 2.0));
    const int n2 = (int)fmin(40.0, fmax(1.0, ceil(log2((b - s) / floor_)) + 2.0));
    add_pieces(R, a, s, false, n1, g10, w10, 10, panel, jacobi, eps);
    add_pieces(R, s, b, true, n2, g10, w10, 10, panel, jacobi, eps);
    return;
  }
  const double dist = (s <= a) ? a - s : s - b;
  const double eff = sqrt(dist * dist + delta * delta);
  if (eff >= L) {
    add_pieces(R, a, b, true, 0, g20, w20, 20, panel, jacobi, eps);
    return;
  }
  const int nlev = (int)fmin(40.0, fmax(1.0, ceil(log2(L / fmax(eff, floor_))) + 2.0));
  add_pieces(R, a, b, s <= a, nlev, g10, w10, 10, panel, jacobi, eps);
}

template <int MODE>
__device__ __forceinline__ double green_near(double d, double r) {
  if (MODE == 0) return 2.0 / d + log((d + (r - 1.0)) / (d + r + 1.0));
  return 2.0 / d + log(4.0 / ((d + (1.0 - r)) * (d + 1.0 + r)));
}

// One block per (target, near patch) pair. MMAX bounds the angular orders (M <= MMAX).
template <int MODE, int MMAX>
__global__ void __launch_bounds__(kNearThreads) near_eval_kernel(NearEvalArgs a) {
  __shared__ double tq[kMaxRadNodes], wq[kMaxRadNodes];
  __shared__ int pan[kMaxRadNodes];
  __shared__ double sh[8];  // t0, theta0, r, delta, sin t0
  __shared__ double ctrig[MMAX + 1], strig[MMAX + 1];
  __shared__ double Cw[kNearWarps][MMAX + 1];
  __shared__ double red[kNearThreads];
  __shared__ int nq_s, over_s;
  const int64_t pr = blockIdx.x;
  const int64_t t = a.pair_target[pr];
  const int j = a.pair_patch[pr];
  const int K = a.K, M = a.M, nord = a.nord;
  const double eps = a.eps;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    // the target in the patch's polar frame: e1 = z x c / |z x c| (x at the poles), e2 = c x e1
    const double cx = a.centres[3 * j], cy = a.centres[3 * j + 1], cz = a.centres[3 * j + 2];
    double e1[3] = {-cy, cx, 0.0};
    const double na2 = e1[0] * e1[0] + e1[1] * e1[1];
    if (na2 >= 1e-24) {
      const double inv = 1.0 / sqrt(na2);
      e1[0] *= inv;
      e1[1] *= inv;
    } else {
      e1[0] = 1.0;
      e1[1] = 0.0;
    }
    const double e2[3] = {cy * e1[2] - cz * e1[1], cz * e1[0] - cx * e1[2], cx * e1[1] - cy * e1[0]};
    const double x0 = a.targets[3 * t], x1 = a.targets[3 * t + 1], x2 = a.targets[3 * t + 2];
    const double r = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
    const double p1 = (x0 * e1[0] + x1 * e1[1] + x2 * e1[2]) / r, p2 = (x0 * e2[0] + x1 * e2[1] + x2 * e2[2]) / r,
                 p3 = (x0 * cx + x1 * cy + x2 * cz) / r;
    const double t0 = atan2(sqrt(p1 * p1 + p2 * p2), p3);
    sh[0] = t0;
    sh[1] = atan2(p2, p1);
    sh[2] = r;
    sh[3] = fabs(r - 1.0);
    sh[4] = sin(t0);
    // the radial rule: every panel graded toward t0 (in u = sqrt(eps - t) on the last one)
    RadialRule R{tq, wq, pan, 0, 0};
    const int npan = a.npan;
    for (int p = 0; p < npan; ++p) {
      const double lo = a.edges[p], hi = a.edges[p + 1];
      if (p < npan - 1) {
        panel_rule(R, lo, hi, t0, sh[3], a.g10, a.w10, a.g20, a.w20, p, false, eps);
      } else {
        const double U = sqrt(eps - lo);
        // t0 maps to u = sqrt(eps - t0) (beyond the patch edge: to the imaginary axis, at
        // distance sqrt(t0 - eps) from u = 0); the off-sphere distance becomes
        // min(sqrt(delta), delta / (2 u0)) in u
        const double su = t0 <= eps ? sqrt(eps - t0) : -sqrt(t0 - eps);
        const double du = fmin(sqrt(sh[3]), su > 0.0 ? sh[3] / (2.0 * su) : sqrt(sh[3]));
        panel_rule(R, 0.0, U, su, du, a.g10, a.w10, a.g20, a.w20, p, true, eps);
      }
    }
    nq_s = R.n;
    over_s = R.overflow;
  }
  __syncthreads();
  if (over_s) {
    if (threadIdx.x == 0) atomicOr(a.err, 1);
    return;
  }
  for (int m = threadIdx.x; m <= M; m += blockDim.x) sincos((double)m * sh[1], &strig[m], &ctrig[m]);
  __syncthreads();
  const double t0 = sh[0], r = sh[2], delta = sh[3], st0 = sh[4];
  const double* fj = a.fhat + (int64_t)j * K;
  double acc = 0.0;
  for (int q = warp; q < nq_s; q += kNearWarps) {
    const double tt = tq[q], wt = wq[q];
    const int p = pan[q];
    const bool jac = (p == a.npan - 1);
    // theta rule depth for this circle: down to the target's distance from it
    const double stt = sin(tt);
    const double dt = tt - t0;
    const double scale = sqrt(delta * delta + dt * dt) / fmax(stt, 1e-300);
    const int nlev =
        (int)fmin((double)kNearMaxLevels, fmax(1.0, ceil(log2(3.141592653589793 / fmax(scale, 1e-300))) + 3.0));
    const double* T = a.phi_tab + 3 * (int64_t)a.phi_off[nlev];
    const int nphi = a.phi_off[nlev + 1] - a.phi_off[nlev];
    const double s2 = sin(0.5 * dt);
    const double base = delta * delta + 4.0 * r * s2 * s2, coef = 4.0 * r * st0 * stt;
    double C[MMAX + 1];
#pragma unroll
    for (int m = 0; m <= MMAX; ++m) C[m] = 0.0;
    for (int i = lane; i < nphi; i += 32) {
      const double w = T[3 * i], h = T[3 * i + 1], cphi = T[3 * i + 2];
      const double d = sqrt(fma(coef, h, base));
      const double g = 2.0 * w * green_near<MODE>(d, r);
      double cm1 = 1.0, cm = cphi;  // cos(0 phi), cos(phi)
      C[0] += g;
#pragma unroll
      for (int m = 1; m <= MMAX; ++m) {
        if (m > M) break;
        C[m] = fma(g, cm, C[m]);
        const double nx = 2.0 * cphi * cm - cm1;
        cm1 = cm;
        cm = nx;
      }
    }
#pragma unroll
    for (int m = 0; m <= MMAX; ++m) {
      if (m > M) break;
      double v = C[m];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) Cw[warp][m] = v;
    }
    __syncwarp();
    // g_k(tt) by barycentric interpolation on panel p (normalised nodes), times f_k
    const double lo = a.edges[p], hi = a.edges[p + 1];
    const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
    const double x = (tt - mid) / half;
    const double* xn = a.xnode + p * nord;
    const double* bw = a.bary + p * nord;
    int exact = -1;
    double den = 0.0;
    for (int l = 0; l < nord; ++l) {
      if (x == xn[l]) exact = l;
      den += bw[l] / (x - xn[l]);
    }
    for (int k = lane; k < K; k += 32) {
      double v;
      const double* bk = a.beta + (int64_t)p * nord * K + k;  // beta[(p nord + l) K + k]
      if (exact >= 0) {
        v = bk[(int64_t)exact * K] * (jac ? sqrt(eps - a.trad[p * nord + exact]) : 1.0);
      } else {
        double num = 0.0;
        for (int l = 0; l < nord; ++l) {
          const double gl = bk[(int64_t)l * K] * (jac ? a.sqrt_gap[p * nord + l] : 1.0);
          num += bw[l] / (x - xn[l]) * gl;
        }
        v = num / den;
      }
      const int m = a.bm[k];
      const double trig = a.bc[k] ? strig[m] : ctrig[m];
      acc = fma(wt * v * fj[k], Cw[warp][m] * trig, acc);
    }
    __syncwarp();
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kNearThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(&a.out[t], red[0]);
}

}  // namespace

// Tables of the phi rules: for nlev = 1..kNearMaxLevels, composite 12-point Gauss pieces on
// (0, pi) graded toward 0 (edges 0, pi 2^-nlev, ..., pi/2, pi; pieces longer than pi/8
// split evenly), each node as (weight, sin^2(phi/2), cos phi); off[nlev] = first node.
void near_phi_tables(std::vector<double>& tab, std::vector<int>& off) {
  std::vector<double> gx, gw;
  gauss_legendre(12, gx, gw);
  tab.clear();
  off.assign(kNearMaxLevels + 2, 0);
  for (int nlev = 0; nlev <= kNearMaxLevels; ++nlev) {
    off[nlev] = (int)(tab.size() / 3);
    if (nlev == 0) continue;  // unused level
    std::vector<double> e{0.0};
    for (int k = nlev; k >= 1; --k) e.push_back(kPi * std::ldexp(1.0, -k));
    e.push_back(kPi);
    std::vector<double> edges{0.0};
    for (size_t i = 1; i < e.size(); ++i) {
      const int parts = std::max(1, (int)std::ceil((e[i] - e[i - 1]) / (kPi / 8.0) - 1e-12));
      for (int q = 1; q <= parts; ++q) edges.push_back(e[i - 1] + (e[i] - e[i - 1]) * q / parts);
    }
    for (size_t i = 1; i < edges.size(); ++i) {
      const double h = 0.5 * (edges[i] - edges[i - 1]), m = 0.5 * (edges[i] + edges[i - 1]);
      for (int q = 0; q < 12; ++q) {
        const double phi = m + h * gx[q];
        const double sh = std::sin(0.5 * phi);
        tab.push_back(h * gw[q]);
        tab.push_back(sh * sh);
        tab.push_back(std::cos(phi));
      }
    }
  }
  off[kNearMaxLevels + 1] = (int)(tab.size() / 3);
}

cudaError_t launch_near_eval(const NearEvalArgs& a, int mode, int64_t npairs, cudaStream_t s) {
  if (npairs == 0) return cudaSuccess;
  if (a.M > 31) return cudaErrorInvalidValue;
  const bool small = a.M <= 17;
  if (mode == 0) {
    if (small)
      count_launch(), near_eval_kernel<0, 17><<<(unsigned)npairs, kNearThreads, 0, s>>>(a);
    else
      count_launch(), near_eval_kernel<0, 31><<<(unsigned)npairs, kNearThreads, 0, s>>>(a);
  } else {
    if (small)
      count_launch(), near_eval_kernel<1, 17><<<(unsigned)npairs, kNearThreads, 0, s>>>(a);
    else
      count_launch(), near_eval_kernel<1, 31><<<(unsigned)npairs, kNearThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace ncs
