// Modal parts of the on-surface Green's function of the unit sphere (Kaye & Greengard,
// Section 8.1), shared by the host precompute and the device collocation kernel.
//
// For two circles t, t' (geodesic distance from the patch centre) the azimuthal Fourier
// modes of G split as G_n = G^(1)_n + s G^(2)_n - G^(3)_n with s = -1 exterior, +1 interior
// (eqs. Gextonsurface / Gintonsurface):
//   G^(1): the Coulomb part 2/d, written through Q_{n-1/2}(chi), the Legendre function of
//          half-integer degree (toroidal function) at chi = 1 + 2 sin^2((t-t')/2) / (sin t sin t');
//   G^(2): the log(2/d) part in the closed form of Section 8.1;
//   G^(3): the log(1 + d/2) part, by quadrature in theta (host loop or device warp).
// Every function is written for both compilers: host C++ and CUDA device code.
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define NCS_HD __host__ __device__ __forceinline__
#else
#define NCS_HD inline
#endif

namespace ncs {
namespace modal {

constexpr double kPiM = 3.14159265358979323846;

// Complete elliptic integrals K(k), E(k) from k^2 and k'^2 = 1 - k^2 (k'^2 passed separately
// so that it keeps its relative accuracy near k = 1), by the arithmetic-geometric mean:
// K = pi / (2 AGM(1, k')), E = K (1 - sum 2^(j-1) c_j^2) with c_0 = k.
NCS_HD void ellipke(double k2, double kp2, double* K, double* E) {
  double a = 1.0, b = sqrt(kp2), c = sqrt(k2);
  double sum = 0.5 * c * c, pw = 0.5;
  for (int it = 0; it < 60; ++it) {
    const double an = 0.5 * (a + b), bn = sqrt(a * b), cn = 0.5 * (a - b);
    a = an;
    b = bn;
    pw *= 2.0;
    sum += pw * cn * cn;
    if (fabs(cn) <= 1e-17 * a) break;
  }
  *K = kPiM / (2.0 * a);
  *E = *K * (1.0 - sum);
}

// G^(1)_n(t, t'), n = 0..nmax, into out[0..nmax]. Q_{-1/2}(chi) = k K(k) and
// Q_{1/2}(chi) = chi k K(k) - 2 E(k) / k with k^2 = 2 / (1 + chi); higher degrees by the
// three-term recurrence (n + 1/2) Q_{n+1/2} = 2 n chi Q_{n-1/2} - (n - 1/2) Q_{n-3/2}, run
// forward while it grows by less than two digits over the modes and otherwise backward
// (Miller), normalised by Q_{-1/2}. The mode factor is 2 / (pi sqrt(sin t sin t')).
// Returns false (out untouched) if nmax >= CAP.
template <int CAP>
NCS_HD bool coulomb_modes(double t, double tp, int nmax, double* out) {
  if (nmax >= CAP) return false;
  const double st = sin(t) * sin(tp);
  const double sh = sin(0.5 * (t - tp));
  const double chim1 = 2.0 * sh * sh / st;  // chi - 1, accurate for t ~ t'
  const double chi = 1.0 + chim1;
  const double k2 = 2.0 / (2.0 + chim1), kp2 = chim1 / (2.0 + chim1);
  double K, E;
  ellipke(k2, kp2, &K, &E);
  const double k = sqrt(k2);
  const double Q0 = k * K;
  const double pref = 2.0 / (kPiM * sqrt(st));
  out[0] = pref * Q0;
  if (nmax == 0) return true;
  const double lnal = log(chi + sqrt(chim1 * (2.0 + chim1)));  // arccosh(chi)
  if (2.0 * nmax * lnal < 4.605170185988091) {                // growth below 100
    double qm = Q0, q = chi * k * K - 2.0 * E / k;
    out[1] = pref * q;
    for (int n = 1; n < nmax; ++n) {
      const double qn = (2.0 * n * chi * q - (n - 0.5) * qm) / (n + 0.5);
      qm = q;
      q = qn;
      out[n + 1] = pref * q;
    }
    return true;
  }
  // backward from degree N - 1/2, far enough that the start's error has decayed below
  // 1e-8 relative (the minimal solution falls like exp(-lnal) per degree); out[] holds the
  // unnormalised values until the end
  const int N = nmax + (int)ceil(18.5 / lnal) + 10;
  double qp = 0.0, q = 1.0;
  for (int n = N; n >= 1; --n) {
    const double qm = (2.0 * n * chi * q - (n + 0.5) * qp) / (n - 0.5);
    qp = q;
    q = qm;
    if (n - 1 <= nmax) out[n - 1] = q;
    if (n <= nmax) out[n] = qp;
    if (fabs(q) > 1e250) {
      q *= 1e-250;
      qp *= 1e-250;
      for (int j = n - 1; j <= nmax; ++j) out[j] *= 1e-250;
    }
  }
  const double scale = pref * Q0 / out[0];
  for (int n = 0; n <= nmax; ++n) out[n] *= scale;
  return true;
}

// G^(2)_n(t, t') (the log(2/d) part), n = 0..nmax, in the closed form of Section 8.1:
// G^(2)_0 = -log(cos(t_</2) sin(t_>/2)), G^(2)_n = (tan(t_</2) / tan(t_>/2))^n / (2n).
// Adds s G^(2)_n to out[n].
NCS_HD void log_modes_add(double t, double tp, int nmax, double s, double* out) {
  const double t1 = t < tp ? t : tp, t2 = t < tp ? tp : t;
  out[0] += s * -log(cos(0.5 * t1) * sin(0.5 * t2));
  const double ratio = tan(0.5 * t1) / tan(0.5 * t2);
  double pw = 1.0;
  for (int n = 1; n <= nmax; ++n) {
    pw *= ratio;
    out[n] += s * (pw / (2.0 * n));
  }
}

}  // namespace modal
}  // namespace ncs
