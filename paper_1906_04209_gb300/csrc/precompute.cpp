// One-patch precompute for the narrow capture / escape solver (Kaye & Greengard):
//   * Zernike basis, sampling nodes and the discrete transform P (Section 4, Section 6);
//   * modal reduction of the one-patch equation (Section 8, eq. modalinteqn), with the
//     modal kernel split as G_n = G^(1) + s G^(2) - G^(3), s = -1 exterior, +1 interior
//     (from the on-surface forms eqs. Gextonsurface / Gintonsurface);
//       G^(1): Coulomb kernel, written through the Legendre function of half-integer
//              degree Q_{n-1/2}(chi) (toroidal function), evaluated from complete elliptic
//              integrals and the three-term recurrence (forward near chi = 1, Miller's
//              backward recurrence otherwise);
//       G^(2): the closed form printed in Section 8.1;
//       G^(3): graded Gauss quadrature in theta;
//   * dyadic panels refined toward t = eps with a Gauss-Jacobi (alpha=-1/2, beta=0) last
//     panel, collocation, one LU per mode (Section 8.2);
//   * fine grid, weights w, B and I = w^T B (Section 5, eq. getI);
//   * interpolative decomposition of the far field by a Gaussian sketch followed by
//     column-pivoted Householder QR, T = Pi W B (Section 7.1, eq. Tmap).
#include "precompute.hpp"
#include "sketch.hpp"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <stdexcept>

#include "modal.hpp"
#include "numerics.hpp"
#include "onepatch.hpp"
#ifdef _OPENMP
#include <omp.h>
#endif

namespace ncs {

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

double jacobi_value(int n, double a, double b, double x) {
  double p0 = 1.0, p1 = 0.5 * (a - b + (a + b + 2.0) * x);
  if (n == 0) return 1.0;
  for (int k = 2; k <= n; ++k) {
    double s = 2.0 * k + a + b;
    double c1 = 2.0 * k * (k + a + b) * (s - 2.0);
    double c2 = (s - 1.0) * (s * (s - 2.0) * x + a * a - b * b);
    double c3 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * s;
    double p2 = (c2 * p1 - c3 * p0) / c1;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// Composite rule on [a,b]: n-point Gauss-Legendre pieces graded dyadically (nlev levels)
// toward the endpoint `toward_a ? a : b`; pieces longer than hmax (if > 0) are split.
void graded(double a, double b, bool toward_a, int nlev, int n, std::vector<double>& x,
            std::vector<double>& w, double hmax = 0.0) {
  static thread_local std::vector<double> gx, gw;
  static thread_local int gn = -1;
  if (gn != n) {
    gauss_legendre(n, gx, gw);
    gn = n;
  }
  double L = b - a;
  double lo = 0.0;
  for (int k = nlev; k >= 0; --k) {
    double hi = (k == 0) ? L : L * std::ldexp(1.0, -k);
    const int split = (hmax > 0.0) ? std::max(1, (int)std::ceil((hi - lo) / hmax)) : 1;
    for (int sp = 0; sp < split; ++sp) {
      double u0 = lo + (hi - lo) * sp / split, u1 = lo + (hi - lo) * (sp + 1) / split;
      double c = 0.5 * (u0 + u1), h = 0.5 * (u1 - u0);
      for (int q = 0; q < n; ++q) {
        double u = c + h * gx[q];
        x.push_back(toward_a ? a + u : b - u);
        w.push_back(h * gw[q]);
      }
    }
    lo = hi;
  }
}

// Rule on [a,b] for an integrand with a (log-type) singularity at the real point s.
// Interior singular points are graded toward until the innermost piece would be shorter
// than hmin (hmin <= 0: 2e-13 max|a,b,s|), so that no node rounds onto s.
void singular_rule(double a, double b, double s, std::vector<double>& x, std::vector<double>& w,
                   double hmin = 0.0) {
  const int n_far = 20, n_grad = 10, nlev_sing = 40;
  x.clear();
  w.clear();
  if (s > a && s < b) {
    const double fl =
        hmin > 0.0 ? hmin : 2e-13 * std::max(std::fabs(s), std::max(std::fabs(a), std::fabs(b)));
    const int n1 = std::min(nlev_sing, std::max(1, (int)std::floor(std::log2((s - a) / fl))));
    const int n2 = std::min(nlev_sing, std::max(1, (int)std::floor(std::log2((b - s) / fl))));
    graded(a, s, false, n1, n_grad, x, w);
    graded(s, b, true, n2, n_grad, x, w);
    return;
  }
  double L = b - a;
  double delta = (s <= a) ? a - s : s - b;
  if (delta >= L) {
    std::vector<double> gx, gw;
    gauss_legendre(n_far, gx, gw);
    for (int q = 0; q < n_far; ++q) {
      x.push_back(0.5 * (a + b) + 0.5 * L * gx[q]);
      w.push_back(0.5 * L * gw[q]);
    }
    return;
  }
  int nlev = (delta <= 0.0) ? nlev_sing : (int)std::ceil(std::log2(L / delta)) + 1;
  graded(a, b, s <= a, nlev, n_grad, x, w);
}

struct ThetaRule {
  std::vector<double> th, w, half_sin2;  // half_sin2 = sin^2(th/2)
  int nmax = -1;
  std::vector<double> cosn;             // (nth) x (nmax+1), weights/pi folded in
  void build(int nmax_) {
    // graded toward 0 (40 levels, 8 nodes), pieces split to at most pi/32 so that
    // cos(n theta) stays resolved
    th.clear();
    w.clear();
    graded(0.0, kPi, true, 40, 8, th, w, kPi / 32.0);
    half_sin2.resize(th.size());
    for (size_t i = 0; i < th.size(); ++i) {
      double s = std::sin(0.5 * th[i]);
      half_sin2[i] = s * s;
    }
    nmax = nmax_;
    cosn.assign(th.size() * (nmax + 1), 0.0);
    for (size_t i = 0; i < th.size(); ++i)
      for (int n = 0; n <= nmax; ++n) cosn[i * (nmax + 1) + n] = std::cos(n * th[i]) * w[i] / kPi;
  }
};

const ThetaRule& theta_rule(int nmax) {
  static thread_local ThetaRule r;
  if (r.nmax < nmax) r.build(std::max(nmax, 32));
  return r;
}

}  // namespace

void zernike_basis(int K, std::vector<int>& bn, std::vector<int>& bm, std::vector<int>& bc) {
  bn.clear();
  bm.clear();
  bc.clear();
  for (int n = 0; (int)bn.size() < K; ++n)
    for (int m = n % 2; m <= n && (int)bn.size() < K; m += 2) {
      bn.push_back(n);
      bm.push_back(m);
      bc.push_back(0);
      if (m > 0 && (int)bn.size() < K) {
        bn.push_back(n);
        bm.push_back(m);
        bc.push_back(1);
      }
    }
}

double zernike_radial(int n, int m, double r) {
  int k = (n - m) / 2;
  double v = std::pow(r, m) * jacobi_value(k, (double)m, 0.0, 1.0 - 2.0 * r * r);
  return (k & 1) ? -v : v;
}

static double zernike_norm2(int n, int m) {
  return (m == 0 ? 2.0 : 1.0) * kPi / (2.0 * n + 2.0);
}

void local_offset(double t, double th, double* o) {
  double st = std::sin(t), sh = std::sin(0.5 * t);
  o[0] = st * std::cos(th);
  o[1] = st * std::sin(th);
  o[2] = -2.0 * sh * sh;
}

void modal_coulomb(double t, double tp, int nmax, double* out) {
  if (!modal::coulomb_modes<512>(t, tp, nmax, out)) throw std::runtime_error("modal_coulomb: nmax too large");
}

void modal_log(double t, double tp, int nmax, double* out) {
  for (int n = 0; n <= nmax; ++n) out[n] = 0.0;
  modal::log_modes_add(t, tp, nmax, 1.0, out);
}

void modal_log1p(double t, double tp, int nmax, double* out) {
  const ThetaRule& R = theta_rule(nmax);
  const double sh = std::sin(0.5 * (t - tp));
  const double A = 4.0 * sh * sh, B = 4.0 * std::sin(t) * std::sin(tp);
  for (int n = 0; n <= nmax; ++n) out[n] = 0.0;
  const int stride = R.nmax + 1;
  for (size_t i = 0; i < R.th.size(); ++i) {
    double d = std::sqrt(A + B * R.half_sin2[i]);
    double g = std::log1p(0.5 * d);
    const double* c = &R.cosn[i * stride];
    for (int n = 0; n <= nmax; ++n) out[n] += g * c[n];
  }
}

void modal_kernels(double t, double tp, int nmax, int mode, double* out) {
  double g1[512], g2[512], g3[512];
  modal_coulomb(t, tp, nmax, g1);
  modal_log(t, tp, nmax, g2);
  modal_log1p(t, tp, nmax, g3);
  const double s = (mode == 0) ? -1.0 : 1.0;
  for (int n = 0; n <= nmax; ++n) out[n] = g1[n] + s * g2[n] - g3[n];
}

void precompute_zernike(double eps, int K, Precomputed& out) {
  out.eps = eps;
  out.K = K;
  zernike_basis(K, out.bn, out.bm, out.bc);
  out.M = *std::max_element(out.bn.begin(), out.bn.end());
  const int M = out.M, nth = 2 * M + 1;
  std::vector<double> gx, gw;
  gauss_legendre(M + 1, gx, gw);
  out.Kstar = (M + 1) * nth;
  out.zr.resize(out.Kstar);
  out.zth.resize(out.Kstar);
  out.zloc.resize(3 * (size_t)out.Kstar);
  out.P.assign((size_t)K * out.Kstar, 0.0);
  for (int a = 0; a <= M; ++a)
    for (int b = 0; b < nth; ++b) {
      int q = a * nth + b;
      double r = 0.5 * (gx[a] + 1.0), th = 2.0 * kPi * b / nth;
      double wq = 0.5 * gw[a] * r * 2.0 * kPi / nth;
      out.zr[q] = r;
      out.zth[q] = th;
      local_offset(eps * r, th, &out.zloc[3 * (size_t)q]);
      for (int j = 0; j < K; ++j) {
        double trig = out.bc[j] ? std::sin(out.bm[j] * th) : std::cos(out.bm[j] * th);
        double qj = zernike_radial(out.bn[j], out.bm[j], r) * trig /
                    std::sqrt(zernike_norm2(out.bn[j], out.bm[j]));
        out.P[(size_t)j * out.Kstar + q] = wq * qj;
      }
    }
}

void precompute(double eps, int mode, int K, const PrecomputeOptions& opt, Precomputed& out) {
  if (!(eps > 0.0 && eps < 1.0)) throw std::runtime_error("precompute: eps must be in (0, 1)");
  if (K < 1 || K > 2000) throw std::runtime_error("precompute: K out of range");
  if (mode != 0 && mode != 1) throw std::runtime_error("precompute: mode must be 0 or 1");
#ifdef _OPENMP
  // the thread count is an ICV of the calling host thread: set it on every call, so that a
  // single-threaded precompute does not leave the next one on this thread single-threaded
  omp_set_num_threads(opt.threads > 0 ? opt.threads : omp_get_num_procs());
#endif
  const double t0 = now_s();
  precompute_zernike(eps, K, out);
  out.mode = mode;
  const int M = out.M;
  int mmax = 0;
  for (int j = 0; j < K; ++j) mmax = std::max(mmax, out.bm[j]);

  // ---- radial panels and collocation nodes (Section 8.2)
  const int npan = opt.npan, nord = opt.nord, nr = npan * nord;
  std::vector<double> edges(npan + 1);
  edges[0] = 0.0;
  for (int j = 1; j < npan; ++j) edges[j] = (1.0 - std::ldexp(1.0, -j)) * eps;
  edges[npan] = eps;
  std::vector<double> gx, gw, jx, jw;
  gauss_legendre(nord, gx, gw);
  gauss_jacobi(nord, -0.5, 0.0, jx, jw);  // weight (1-x)^(-1/2): singular end at t = eps
  std::vector<double> tr(nr), wsig(nr), pnorm(nr);
  for (int j = 0; j < npan; ++j) {
    double a = edges[j], b = edges[j + 1], h = b - a;
    for (int k = 0; k < nord; ++k) {
      int i = j * nord + k;
      if (j < npan - 1) {
        tr[i] = a + 0.5 * (gx[k] + 1.0) * h;
        wsig[i] = 0.5 * h * gw[k];
        pnorm[i] = gx[k];
      } else {
        tr[i] = a + 0.5 * (jx[k] + 1.0) * h;
        // int phi (eps-t)^(-1/2) dt = sqrt(h/2) sum w_k phi(t_k); sigma stored pointwise
        wsig[i] = std::sqrt(0.5 * h) * jw[k] * std::sqrt(eps - tr[i]);
        pnorm[i] = jx[k];
      }
    }
  }
  std::vector<double> nodes_gl(gx), nodes_gj(jx);
  const Lagrange lag_gl(nodes_gl), lag_gj(nodes_gj);

  // ---- collocation matrices A_n (n = 0..mmax), row-major nr x nr each. Row i against
  // panel j integrates G_n(t_i, t') times the panel's Lagrange basis with a rule graded
  // toward t' = t_i; on the Gauss-Jacobi panel the rule is taken in u = sqrt(eps - t').
  auto colloc_rule = [&](int i, int j, std::vector<double>& xq, std::vector<double>& wq) {
    const double a = edges[j], ti = tr[i];
    if (j < npan - 1) {
      singular_rule(a, edges[j + 1], ti, xq, wq);
      return;
    }
    // t' = eps - u^2 on u in [0, sqrt(eps - a)]: (eps - t')^(-1/2) dt' = 2 du
    const double U = std::sqrt(eps - a), su = std::sqrt(std::max(eps - ti, 0.0));
    // dt'/du = -2u: keep t' >= ~30 ulp away from t_i near u = su
    const double hu = su > 0.0 ? std::max(2e-13 * U, 2e-13 * eps / su) : 0.0;
    singular_rule(0.0, U, su, xq, wq, hu);
    for (size_t q = 0; q < xq.size(); ++q) {
      double u = xq[q];
      xq[q] = eps - u * u;
      wq[q] *= 2.0;
    }
  };
  // column factors: the Jacobi panel's unknowns are g(t_k) = sigma(t_k) sqrt(eps - t_k)
  std::vector<double> colscale(nr, 1.0);
  for (int k = 0; k < nord; ++k) colscale[(npan - 1) * nord + k] = std::sqrt(eps - tr[(npan - 1) * nord + k]);
  const double tc0 = now_s();
  std::vector<double> A;
  out.colloc_on_device = false;
  if (opt.device_colloc && nord <= kCollocMaxOrd && mmax < kCollocMaxModes) {
    CollocProblem pr;
    pr.nr = nr;
    pr.npan = npan;
    pr.nord = nord;
    pr.nmodes = mmax + 1;
    pr.mode = mode;
    pr.tr = tr;
    pr.colscale = colscale;
    pr.lag_nodes = gx;
    pr.lag_nodes.insert(pr.lag_nodes.end(), jx.begin(), jx.end());
    pr.lag_bw = lag_gl.bw;
    pr.lag_bw.insert(pr.lag_bw.end(), lag_gj.bw.begin(), lag_gj.bw.end());
    // every (row, panel) rule, built per row in parallel and concatenated in (i, j) order
    std::vector<std::vector<double>> rows(nr);
    std::vector<int> cnt((size_t)nr * npan);
#pragma omp parallel
    {
      std::vector<double> xq, wq;
#pragma omp for schedule(dynamic, 4)
      for (int i = 0; i < nr; ++i) {
        std::vector<double>& r = rows[i];
        for (int j = 0; j < npan; ++j) {
          colloc_rule(i, j, xq, wq);
          const double mid = 0.5 * (edges[j] + edges[j + 1]), half = 0.5 * (edges[j + 1] - edges[j]);
          for (size_t q = 0; q < xq.size(); ++q) {
            r.push_back(xq[q]);
            r.push_back(2.0 * kPi * wq[q] * std::sin(xq[q]));
            r.push_back((xq[q] - mid) / half);
          }
          cnt[(size_t)i * npan + j] = (int)xq.size();
        }
      }
    }
    pr.qoff.assign((size_t)nr * npan + 1, 0);
    for (size_t b = 0; b < cnt.size(); ++b) pr.qoff[b + 1] = pr.qoff[b] + cnt[b];
    const size_t nq = (size_t)pr.qoff.back();
    pr.tq.reserve(nq);
    pr.wt.reserve(nq);
    pr.ls.reserve(nq);
    for (int i = 0; i < nr; ++i)
      for (size_t q = 0; q < rows[i].size(); q += 3) {
        pr.tq.push_back(rows[i][q]);
        pr.wt.push_back(rows[i][q + 1]);
        pr.ls.push_back(rows[i][q + 2]);
      }
    const ThetaRule& R = theta_rule(mmax);
    pr.hs2 = R.half_sin2;
    pr.cw.resize(R.th.size() * (size_t)(mmax + 1));
    for (size_t it = 0; it < R.th.size(); ++it)
      for (int n = 0; n <= mmax; ++n) pr.cw[it * (mmax + 1) + n] = R.cosn[it * (R.nmax + 1) + n];
    std::string err;
    const int rc = colloc_assemble_device(pr, A, &err);
    if (rc < 0) throw std::runtime_error(err);
    out.colloc_on_device = rc > 0;
  }
  if (!out.colloc_on_device) {
    A.assign((size_t)(mmax + 1) * nr * nr, 0.0);
#pragma omp parallel
    {
      std::vector<double> xq, wq, Gn(mmax + 1), L(nord);
#pragma omp for schedule(dynamic, 1)
      for (int i = 0; i < nr; ++i) {
        const double ti = tr[i];
        for (int j = 0; j < npan; ++j) {
          const double mid = 0.5 * (edges[j] + edges[j + 1]), half = 0.5 * (edges[j + 1] - edges[j]);
          const bool jac = (j == npan - 1);
          colloc_rule(i, j, xq, wq);
          for (size_t q = 0; q < xq.size(); ++q) {
            const double tq = xq[q];
            modal_kernels(ti, tq, mmax, mode, Gn.data());
            (jac ? lag_gj : lag_gl).eval((tq - mid) / half, L.data());
            const double wt = 2.0 * kPi * wq[q] * std::sin(tq);
            for (int k = 0; k < nord; ++k) {
              const double c = wt * (L[k] * colscale[j * nord + k]);
              for (int n = 0; n <= mmax; ++n) A[((size_t)n * nr + i) * nr + j * nord + k] += c * Gn[n];
            }
          }
        }
      }
    }
  }
  const double tc1 = now_s();
  out.seconds_colloc = tc1 - tc0;

  // ---- one LU per mode; beta_j solves the mode-m_j system with rhs c_j R(t/eps)
  if (opt.keep_collocation) out.colloc = A;
  std::vector<LU> lus(mmax + 1);
#pragma omp parallel for schedule(dynamic, 1)
  for (int n = 0; n <= mmax; ++n) lus[n].factor(&A[(size_t)n * nr * nr], nr);
  out.nrad = nr;
  out.trad = tr;
  out.beta.assign((size_t)nr * K, 0.0);
  {
    std::vector<double> rhs(nr);
    for (int j = 0; j < K; ++j) {
      const double c = 1.0 / std::sqrt(zernike_norm2(out.bn[j], out.bm[j]));
      for (int i = 0; i < nr; ++i) rhs[i] = c * zernike_radial(out.bn[j], out.bm[j], tr[i] / eps);
      lus[out.bm[j]].solve(rhs.data());
      for (int i = 0; i < nr; ++i) out.beta[(size_t)i * K + j] = rhs[i];
    }
  }
  out.seconds_lu = now_s() - tc1;

  // ---- fine grid, weights and I = w^T B
  int nth = opt.ntheta_fine > 0 ? opt.ntheta_fine : M + 40;
  nth += nth % 2;
  out.ntheta = nth;
  const int nf = nr * nth;
  out.nf = nf;
  out.w.resize(nf);
  std::vector<double> thf(nth);
  for (int a = 0; a < nth; ++a) thf[a] = 2.0 * kPi * a / nth;
  for (int r = 0; r < nr; ++r)
    for (int a = 0; a < nth; ++a) out.w[(size_t)r * nth + a] = wsig[r] * std::sin(tr[r]) * 2.0 * kPi / nth;
  std::vector<double> trig((size_t)nth * K);
  for (int a = 0; a < nth; ++a)
    for (int j = 0; j < K; ++j)
      trig[(size_t)a * K + j] = out.bc[j] ? std::sin(out.bm[j] * thf[a]) : std::cos(out.bm[j] * thf[a]);
  // WB(l, j) = w_l beta_j(t_r) trig_j(theta_a), l = r*nth + a
  auto WB = [&](int l, double* row) {
    const int r = l / nth, a = l % nth;
    const double wl = out.w[l];
    for (int j = 0; j < K; ++j) row[j] = wl * out.beta[(size_t)r * K + j] * trig[(size_t)a * K + j];
  };
  out.I.assign(K, 0.0);
  {
    std::vector<double> row(K);
    for (int l = 0; l < nf; ++l) {
      WB(l, row.data());
      for (int j = 0; j < K; ++j) out.I[j] += row[j];
    }
  }
  // W B rows of every fine-grid point (nf x K), used by every representation's T
  std::vector<double> WBall((size_t)nf * K);
#pragma omp parallel for schedule(static)
  for (int l = 0; l < nf; ++l) WB(l, &WBall[(size_t)l * K]);
  const double t1 = now_s();
  out.seconds_onepatch = t1 - t0;

  // ---- interpolative decompositions of the far field (Section 7.1), one per far-field
  // radius of a ladder rho_min = 2, 2.52, 3.17, 4, 5.04, ... eps (the per-level recompression
  // of "Optimizations and parallelization": a source seen from farther away needs fewer
  // skeleton points). The training grid on {rho > rho_min} is made of radial panels whose
  // lower edges are the ladder radii (then doubling up to pi), with Gauss-Legendre nodes
  // and an azimuthal count from the (eps/rho)^m decay of fields generated in the patch.
  std::vector<double> ladder;
  {
    double r = opt.id_rho_min;
    ladder.push_back(r);
    if (opt.multilevel) {
      for (int it = 0; it < 64; ++it) {
        r *= 1.2599210498948732;  // 2^(1/3): three rungs per doubling of the radius
        if (r * eps > opt.id_ladder_max) break;
        ladder.push_back(r);
      }
    }
  }
  std::vector<double> pedges;
  for (double l : ladder) pedges.push_back(l * eps);
  while (pedges.back() * 2.0 < kPi) pedges.push_back(pedges.back() * 2.0);
  pedges.push_back(kPi);
  const int npanel = (int)pedges.size() - 1;
  std::vector<double> xt;
  std::vector<int> prow(npanel + 1, 0);
  {
    std::vector<double> px, pw;
    gauss_legendre(opt.id_nper, px, pw);
    for (int s = 0; s < npanel; ++s) {
      const double a = pedges[s], b = pedges[s + 1];
      int m = (int)std::ceil(std::log(opt.id_tol / 10.0) / std::log(eps / a));
      m = std::max(m, 8);
      const int nphi = 2 * m + 1;
      for (int q = 0; q < opt.id_nper; ++q) {
        const double rho = 0.5 * (a + b) + 0.5 * (b - a) * px[q];
        for (int f = 0; f < nphi; ++f) {
          const double phi = 2.0 * kPi * f / nphi;
          xt.push_back(std::sin(rho) * std::cos(phi));
          xt.push_back(std::sin(rho) * std::sin(phi));
          xt.push_back(std::cos(rho));
        }
      }
      prow[s + 1] = (int)(xt.size() / 3);
    }
  }
  const int nt = (int)(xt.size() / 3);
  std::vector<double> xf(3 * (size_t)nf);
  for (int r = 0; r < nr; ++r)
    for (int a = 0; a < nth; ++a) {
      size_t l = (size_t)r * nth + a;
      xf[3 * l + 0] = std::sin(tr[r]) * std::cos(thf[a]);
      xf[3 * l + 1] = std::sin(tr[r]) * std::sin(thf[a]);
      xf[3 * l + 2] = std::cos(tr[r]);
    }
  const double sgn = (mode == 0) ? -1.0 : 1.0;
  auto Gsurf = [sgn](double d) { return 2.0 / d + sgn * std::log(2.0 / d) - std::log1p(0.5 * d); };

  // Column-pivoted Householder QR of a sketch Y (column-major ks x nf, destroyed),
  // stopped at |R_kk| < tol |R_00|. Returns the rank; piv and the R factor stay in Y.
  auto cpqr = [&](std::vector<double>& Y, int ks, std::vector<int>& piv) {
    piv.resize(nf);
    for (int l = 0; l < nf; ++l) piv[l] = l;
    std::vector<double> cn(nf), cn0(nf);
    for (int l = 0; l < nf; ++l) {
      double v = 0.0;
      for (int r = 0; r < ks; ++r) v += Y[(size_t)l * ks + r] * Y[(size_t)l * ks + r];
      cn[l] = cn0[l] = v;
    }
    double r00 = 0.0;
    int p = 0;
    std::vector<double> v(ks);
    for (int st = 0; st < ks; ++st) {
      int best = st;
      for (int l = st + 1; l < nf; ++l)
        if (cn[l] > cn[best]) best = l;
      if (best != st) {
        std::swap(piv[st], piv[best]);
        std::swap(cn[st], cn[best]);
        std::swap(cn0[st], cn0[best]);
        std::swap_ranges(&Y[(size_t)st * ks], &Y[(size_t)st * ks] + ks, &Y[(size_t)best * ks]);
      }
      double* col = &Y[(size_t)st * ks];
      double nrm = 0.0;
      for (int r = st; r < ks; ++r) nrm += col[r] * col[r];
      nrm = std::sqrt(nrm);
      const double rss = (col[st] >= 0.0) ? -nrm : nrm;
      if (st == 0) r00 = std::fabs(rss);
      if (std::fabs(rss) < opt.id_tol * r00 || nrm == 0.0) return st;
      for (int r = st; r < ks; ++r) v[r] = col[r];
      v[st] -= rss;
      double vv = 0.0;
      for (int r = st; r < ks; ++r) vv += v[r] * v[r];
      col[st] = rss;
      for (int r = st + 1; r < ks; ++r) col[r] = 0.0;
#pragma omp parallel for schedule(static)
      for (int l = st + 1; l < nf; ++l) {
        double* y = &Y[(size_t)l * ks];
        double dot = 0.0;
        for (int r = st; r < ks; ++r) dot += v[r] * y[r];
        const double f = 2.0 * dot / vv;
        for (int r = st; r < ks; ++r) y[r] -= f * v[r];
        double nn = cn[l] - y[st] * y[st];
        if (nn < 1e-10 * cn0[l]) {  // recompute after cancellation
          nn = 0.0;
          for (int r = st + 1; r < ks; ++r) nn += y[r] * y[r];
          cn0[l] = nn;
        }
        cn[l] = nn;
      }
      p = st + 1;
    }
    return p;
  };

  // Skeleton coordinates of a representation from its pivot order.
  auto set_skeleton = [&](const std::vector<int>& piv, int p, double rho_min, OutRep& rep) {
    rep.rho_min = rho_min;
    rep.p = p;
    rep.st.resize(p);
    rep.sth.resize(p);
    rep.sloc.resize(3 * (size_t)p);
    for (int m = 0; m < p; ++m) {
      const int l = piv[m];
      rep.st[m] = tr[l / nth];
      rep.sth[m] = thf[l % nth];
      local_offset(rep.st[m], rep.sth[m], &rep.sloc[3 * (size_t)m]);
    }
  };

  // Pi = [I, R11^-1 R12] in pivoted order; T = Pi W B; skeleton coordinates.
  auto finish_level = [&](const std::vector<double>& Y, int ks, const std::vector<int>& piv, int p,
                          double rho_min, OutRep& rep) {
    const int nrest = nf - p;
    std::vector<double> X((size_t)p * nrest);
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nrest; ++c) {
      const double* y = &Y[(size_t)(p + c) * ks];
      std::vector<double> xcol(p);
      for (int m = p - 1; m >= 0; --m) {
        double v = y[m];
        for (int q = m + 1; q < p; ++q) v -= Y[(size_t)q * ks + m] * xcol[q];
        xcol[m] = v / Y[(size_t)m * ks + m];
      }
      for (int m = 0; m < p; ++m) X[(size_t)m * nrest + c] = xcol[m];
    }
    rep.rho_min = rho_min;
    rep.p = p;
    rep.T.assign((size_t)p * K, 0.0);
    // T = W B[skeleton] + X W B[rest] (eq. Tmap), as a product blocked over the rest
    // columns: each block of WB rows is gathered once and applied to all rows of T
    for (int m = 0; m < p; ++m)
      std::copy(&WBall[(size_t)piv[m] * K], &WBall[(size_t)piv[m] * K] + K, &rep.T[(size_t)m * K]);
    constexpr int CBL = 64;
    std::vector<double> blk((size_t)CBL * K);
    for (int c0 = 0; c0 < nrest; c0 += CBL) {
      const int nc = std::min(CBL, nrest - c0);
      for (int c = 0; c < nc; ++c)
        std::copy(&WBall[(size_t)piv[p + c0 + c] * K], &WBall[(size_t)piv[p + c0 + c] * K] + K, &blk[(size_t)c * K]);
#pragma omp parallel for schedule(static)
      for (int m = 0; m < p; ++m) {
        double* Tm = &rep.T[(size_t)m * K];
        const double* xm = &X[(size_t)m * nrest + c0];
        for (int c = 0; c < nc; ++c) {
          const double x = xm[c];
          const double* b = &blk[(size_t)c * K];
          for (int j = 0; j < K; ++j) Tm[j] += x * b[j];
        }
      }
    }
    set_skeleton(piv, p, rho_min, rep);
  };

  const int nlev = (int)ladder.size();
  int ks = std::min(256, nt);
  for (;;) {
    out.reps.assign(nlev, OutRep());
    // Gaussian sketch Omega (ks x nt, counter-based, each value rounded to FP32 so that the
    // device forms its products exactly in float-float); panels are added from the outside
    // in, so after adding panel k the running sum is the sketch of the training rows
    // of {rho > ladder[k] eps}.
    std::vector<double> Om((size_t)ks * nt);
    for (int r = 0; r < ks; ++r)
      for (int j = 0; j < nt; ++j)
        Om[(size_t)r * nt + j] = (double)(float)normal_variate(((uint64_t)r << 32) + j + 0x5eedull);
    std::vector<double> Yrun((size_t)ks * nf, 0.0), Yc;
    bool enlarge = false;
    int kse_start = nlev == 1 ? 256 : 64;
    const int CB = 32;
    // the sketch products on the device when one is available (same Omega, FP64)
    // float-float sketch products unless the ID tolerance is within reach of their accuracy
    DeviceSketch* dsk = opt.device_sketch ? sketch_create(ks, nt, nf, mode, Om.data(), xt.data(), xf.data(),
                                                          opt.id_tol >= 1e-12)
                                          : nullptr;
    if (dsk && !sketch_set_wb(dsk, K, WBall.data())) {
      sketch_destroy(dsk);
      dsk = nullptr;
    }
    out.sketch_on_device = dsk != nullptr;
    for (int pan = npanel - 1; pan >= 0 && !enlarge; --pan) {
      const int r0 = prow[pan], r1 = prow[pan + 1], nrw = r1 - r0;
      const double ts0 = now_s();
      if (dsk) {
        if (!sketch_add_rows(dsk, r0, r1)) {
          sketch_destroy(dsk);
          throw std::runtime_error("precompute: device sketch failed");
        }
      } else
#pragma omp parallel
      {
        std::vector<double> Ab((size_t)nrw * CB);
#pragma omp for schedule(dynamic, 1)
        for (int cb = 0; cb < (nf + CB - 1) / CB; ++cb) {
          const int l0 = cb * CB, nl = std::min(CB, nf - l0);
          // kernel block stored column by column (Ab[c][j]) so that the sketch update
          // below runs over contiguous rows of Omega and of the block
          for (int c = 0; c < nl; ++c) {
            const double* bp = &xf[3 * (size_t)(l0 + c)];
            double* ac = &Ab[(size_t)c * nrw];
            for (int j = 0; j < nrw; ++j) {
              const double* a = &xt[3 * (size_t)(r0 + j)];
              const double dx = a[0] - bp[0], dy = a[1] - bp[1], dz = a[2] - bp[2];
              ac[j] = Gsurf(std::sqrt(dx * dx + dy * dy + dz * dz));
            }
          }
          for (int c = 0; c < nl; ++c) {
            double* ycol = &Yrun[(size_t)(l0 + c) * ks];
            const double* ac = &Ab[(size_t)c * nrw];
            for (int r = 0; r < ks; ++r) {
              const double* om = &Om[(size_t)r * nt + r0];
              double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
              int j = 0;
              for (; j + 4 <= nrw; j += 4) {
                v0 += om[j] * ac[j];
                v1 += om[j + 1] * ac[j + 1];
                v2 += om[j + 2] * ac[j + 2];
                v3 += om[j + 3] * ac[j + 3];
              }
              for (; j < nrw; ++j) v0 += om[j] * ac[j];
              ycol[r] += (v0 + v1) + (v2 + v3);
            }
          }
        }
      }
      out.seconds_sketch += now_s() - ts0;
      if (pan < nlev) {
        const double tc0 = now_s();
        // CPQR on the first kse rows of the sketch (itself a Gaussian sketch), doubling from
        // 64 rows until at least 16 rows of oversampling remain past the rank: the outer
        // levels of the ladder have small ranks. Levels are processed from the outside in,
        // so ranks grow from one level to the next: each level starts at the row count the
        // doubling reached for the previous one (the same final count as starting from 64,
        // without the restarts). A lone level at 2 eps starts at 256 rows: its rank at the
        // ID tolerances in use exceeds 112, where the doubling from 64 ends there as well.
        std::vector<int> piv;
        int kse = std::min(ks, kse_start), p = 0;
        for (;;) {
          if (dsk) {
            p = sketch_cpqr(dsk, kse, opt.id_tol, piv);
            if (p < 0) {
              sketch_destroy(dsk);
              throw std::runtime_error("precompute: device CPQR failed");
            }
          } else {
            Yc.resize((size_t)kse * nf);
            for (int l = 0; l < nf; ++l)
              std::copy(&Yrun[(size_t)l * ks], &Yrun[(size_t)l * ks] + kse, &Yc[(size_t)l * kse]);
            p = cpqr(Yc, kse, piv);
          }
          if (p >= kse - 16 && kse < ks) {
            kse = std::min(2 * kse, ks);
            continue;
          }
          break;
        }
        if (p >= ks - 16 && ks < nt) {
          enlarge = true;
          break;
        }
        kse_start = kse;
        if (p < 1) {
          sketch_destroy(dsk);
          throw std::runtime_error("precompute: ID rank is zero");
        }
        const double tc1 = now_s();
        out.seconds_cpqr += tc1 - tc0;
        if (dsk) {
          if (!sketch_assemble(dsk, p, out.reps[pan].T)) {
            sketch_destroy(dsk);
            throw std::runtime_error("precompute: device assembly failed");
          }
          set_skeleton(piv, p, ladder[pan] * eps, out.reps[pan]);
        } else {
          finish_level(Yc, kse, piv, p, ladder[pan] * eps, out.reps[pan]);
        }
        out.seconds_assemble += now_s() - tc1;
      }
    }
    sketch_destroy(dsk);
    if (!enlarge) break;
    ks = std::min(2 * ks, nt);  // rank not revealed by the sketch: enlarge it
  }
  // the finest representation (far field beyond id_rho_min eps) doubles as the
  // single-level operator
  out.p = out.reps[0].p;
  out.T = out.reps[0].T;
  out.st = out.reps[0].st;
  out.sth = out.reps[0].sth;
  out.sloc = out.reps[0].sloc;
  out.seconds_id = now_s() - t1;
}

}  // namespace ncs
