// Host FP64 numerics used by the one-patch precompute: Gauss rules (Golub-Welsch
// with Newton polish), Jacobi polynomials, Lagrange interpolation, LU with partial
// pivoting, complete elliptic integrals by the arithmetic-geometric mean.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>
#include <stdexcept>
#include <vector>

namespace ncs {

constexpr double kPi = 3.14159265358979323846264338327950288;

// Symmetric tridiagonal eigenproblem by implicit QL with Wilkinson shifts.
// d: diagonal (n), e: sub-diagonal (e[1..n-1] used, e[0] ignored). On exit d holds
// the eigenvalues and z0 the first component of each normalised eigenvector.
inline void tridiag_ql(std::vector<double>& d, std::vector<double> e, std::vector<double>& z0) {
  const int n = (int)d.size();
  std::vector<double> Z((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
  for (int i = 1; i < n; ++i) e[i - 1] = e[i];
  e[n - 1] = 0.0;
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    int m;
    do {
      for (m = l; m < n - 1; ++m) {
        double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (std::fabs(e[m]) <= 1e-300 + 2.2e-16 * dd) break;
      }
      if (m != l) {
        if (++iter > 200) throw std::runtime_error("tridiag_ql: no convergence");
        double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
        double r = std::hypot(g, 1.0);
        g = d[m] - d[l] + e[l] / (g + (g >= 0 ? std::fabs(r) : -std::fabs(r)));
        double s = 1.0, c = 1.0, p = 0.0;
        int i;
        for (i = m - 1; i >= l; --i) {
          double f = s * e[i], b = c * e[i];
          r = std::hypot(f, g);
          e[i + 1] = r;
          if (r == 0.0) {
            d[i + 1] -= p;
            e[m] = 0.0;
            break;
          }
          s = f / r;
          c = g / r;
          g = d[i + 1] - p;
          r = (d[i] - g) * s + 2.0 * c * b;
          p = s * r;
          d[i + 1] = g + p;
          g = c * r - b;
          for (int k = 0; k < n; ++k) {
            double zk1 = Z[(size_t)k * n + i + 1];
            double zk = Z[(size_t)k * n + i];
            Z[(size_t)k * n + i + 1] = s * zk + c * zk1;
            Z[(size_t)k * n + i] = c * zk - s * zk1;
          }
        }
        if (r == 0.0 && i >= l) continue;
        d[l] -= p;
        e[l] = g;
        e[m] = 0.0;
      }
    } while (m != l);
  }
  z0.assign(n, 0.0);
  for (int j = 0; j < n; ++j) z0[j] = Z[j];  // row 0 = first components
}

// Jacobi polynomial P_n^{(a,b)}(x) and its derivative by the three-term recurrence.
inline void jacobi_pd(int n, double a, double b, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = 0.5 * (a - b + (a + b + 2.0) * x);
  if (n == 0) {
    *p = 1.0;
    *dp = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    double s = 2.0 * k + a + b;
    double c1 = 2.0 * k * (k + a + b) * (s - 2.0);
    double c2 = (s - 1.0) * (s * (s - 2.0) * x + a * a - b * b);
    double c3 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * s;
    double p2 = (c2 * p1 - c3 * p0) / c1;
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  // derivative: d/dx P_n^{(a,b)} = (n+a+b+1)/2 P_{n-1}^{(a+1,b+1)}
  double q0 = 1.0, q1 = 0.5 * (a - b + (a + b + 4.0) * x);
  double aa = a + 1.0, bb = b + 1.0;
  if (n - 1 == 0) {
    *dp = 0.5 * (n + a + b + 1.0);
    return;
  }
  for (int k = 2; k <= n - 1; ++k) {
    double s = 2.0 * k + aa + bb;
    double c1 = 2.0 * k * (k + aa + bb) * (s - 2.0);
    double c2 = (s - 1.0) * (s * (s - 2.0) * x + aa * aa - bb * bb);
    double c3 = 2.0 * (k + aa - 1.0) * (k + bb - 1.0) * s;
    double q2 = (c2 * q1 - c3 * q0) / c1;
    q0 = q1;
    q1 = q2;
  }
  *dp = 0.5 * (n + a + b + 1.0) * q1;
}

// n-point Gauss-Jacobi rule on [-1,1] for weight (1-x)^a (1+x)^b, ascending nodes.
inline void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
  std::vector<double> d(n), e(n, 0.0), z0;
  for (int k = 0; k < n; ++k) {
    double s = 2.0 * k + a + b;
    d[k] = (k == 0) ? (b - a) / (a + b + 2.0) : (b * b - a * a) / (s * (s + 2.0));
    if (k >= 1) {
      double num = 4.0 * k * (k + a) * (k + b) * (k + a + b);
      double den = s * s * (s + 1.0) * (s - 1.0);
      e[k] = std::sqrt(num / den);
    }
  }
  tridiag_ql(d, e, z0);
  double mu0 = std::pow(2.0, a + b + 1.0) * std::tgamma(a + 1.0) * std::tgamma(b + 1.0) /
               std::tgamma(a + b + 2.0);
  std::vector<std::pair<double, double>> xw(n);
  for (int i = 0; i < n; ++i) xw[i] = {d[i], mu0 * z0[i] * z0[i]};
  // sort ascending
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && xw[j].first < xw[j - 1].first; --j) std::swap(xw[j], xw[j - 1]);
  x.resize(n);
  w.resize(n);
  // Newton polish of the nodes; weights from the derivative formula
  // w_i = C / ((1 - x_i^2) P_n'(x_i)^2).
  double lc = (a + b + 1.0) * std::log(2.0) + std::lgamma(n + a + 1.0) + std::lgamma(n + b + 1.0) -
              std::lgamma(n + a + b + 1.0) - std::lgamma(n + 1.0);
  for (int i = 0; i < n; ++i) {
    double xi = xw[i].first, p, dp;
    for (int it = 0; it < 3; ++it) {
      jacobi_pd(n, a, b, xi, &p, &dp);
      xi -= p / dp;
    }
    jacobi_pd(n, a, b, xi, &p, &dp);
    x[i] = xi;
    w[i] = std::exp(lc) / ((1.0 - xi * xi) * dp * dp);
  }
}

inline void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  gauss_jacobi(n, 0.0, 0.0, x, w);
}

// Lagrange cardinal functions on nodes (barycentric form), evaluated at s.
struct Lagrange {
  std::vector<double> nodes, bw;
  explicit Lagrange(const std::vector<double>& xn) : nodes(xn), bw(xn.size(), 1.0) {
    const size_t n = xn.size();
    for (size_t j = 0; j < n; ++j) {
      double p = 1.0;
      for (size_t k = 0; k < n; ++k)
        if (k != j) p *= (xn[j] - xn[k]);
      bw[j] = 1.0 / p;
    }
  }
  void eval(double s, double* out) const {
    const size_t n = nodes.size();
    for (size_t j = 0; j < n; ++j)
      if (s == nodes[j]) {
        for (size_t k = 0; k < n; ++k) out[k] = (k == j) ? 1.0 : 0.0;
        return;
      }
    double den = 0.0;
    for (size_t j = 0; j < n; ++j) {
      out[j] = bw[j] / (s - nodes[j]);
      den += out[j];
    }
    for (size_t j = 0; j < n; ++j) out[j] /= den;
  }
};

// LU with partial pivoting (row-major n x n, in place).
struct LU {
  int n = 0;
  std::vector<double> a;
  std::vector<int> piv;
  void factor(const double* A, int n_) {
    n = n_;
    a.assign(A, A + (size_t)n * n);
    piv.resize(n);
    for (int k = 0; k < n; ++k) {
      int p = k;
      double mx = std::fabs(a[(size_t)k * n + k]);
      for (int i = k + 1; i < n; ++i)
        if (std::fabs(a[(size_t)i * n + k]) > mx) {
          mx = std::fabs(a[(size_t)i * n + k]);
          p = i;
        }
      piv[k] = p;
      if (mx == 0.0) throw std::runtime_error("LU: singular matrix");
      if (p != k)
        for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)p * n + j]);
      double inv = 1.0 / a[(size_t)k * n + k];
      for (int i = k + 1; i < n; ++i) {
        double f = (a[(size_t)i * n + k] *= inv);
        if (f != 0.0) {
          const double* rk = &a[(size_t)k * n];
          double* ri = &a[(size_t)i * n];
          for (int j = k + 1; j < n; ++j) ri[j] -= f * rk[j];
        }
      }
    }
  }
  void solve(double* b) const {
    // rows were swapped whole during factorisation: permute b first, then L y = Pb
    for (int k = 0; k < n; ++k)
      if (piv[k] != k) std::swap(b[k], b[piv[k]]);
    for (int i = 1; i < n; ++i) {
      double s = b[i];
      const double* ri = &a[(size_t)i * n];
      for (int j = 0; j < i; ++j) s -= ri[j] * b[j];
      b[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = b[i];
      for (int j = i + 1; j < n; ++j) s -= a[(size_t)i * n + j] * b[j];
      b[i] = s / a[(size_t)i * n + i];
    }
  }
};

// Counter-based standard normal variates (splitmix64 + Box-Muller).
inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
inline double unit_uniform(uint64_t key) {
  return ((splitmix64(key) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}
inline double normal_variate(uint64_t key) {
  double u1 = unit_uniform(2 * key), u2 = unit_uniform(2 * key + 1);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * kPi * u2);
}

}  // namespace ncs
