// One-patch precompute (Step 1 of Kaye & Greengard, Section 7): Zernike basis and
// transform P (Section 4), modal one-patch solve giving B, fine-grid weights w and
// I = w^T B (Sections 5, 6, 8), interpolative decomposition and T = Pi W B (Section 7.1).
#pragma once
#include <string>
#include <vector>

namespace ncs {

struct PrecomputeOptions {
  int npan = 13;            // radial panels, dyadically refined toward the patch edge
  int nord = 20;            // nodes per panel
  int ntheta_fine = 0;      // fine-grid azimuths (0: M + 40 rounded up to even)
  double id_tol = 1e-11;    // ID tolerance
  int id_nper = 10;         // training-grid Gauss nodes per radial panel
  int threads = 0;          // host threads (0: all)
  double id_rho_min = 2.0;  // far region starts at id_rho_min * eps
  bool multilevel = true;   // also compress against farther regions (ladder x 2^(1/3))
  double id_ladder_max = 1.0;  // largest far-field radius of the ladder (radians)
  bool device_sketch = false;  // form the ID sketch on the current CUDA device when one exists
  bool device_colloc = false;  // form the modal collocation matrices on the current CUDA device
  bool keep_collocation = false;  // keep the modal collocation matrices (diagnostics)
};

// Outgoing representation valid for targets farther than rho_min (geodesic) from
// the patch centre: rho = T f on p skeleton points (Section 7.1, eq. Tmap).
struct OutRep {
  double rho_min = 0.0;
  int p = 0;
  std::vector<double> T;        // p x K
  std::vector<double> st, sth;  // skeleton (t, theta)
  std::vector<double> sloc;     // p x 3 offsets in the patch frame
};

struct Precomputed {
  double eps = 0;
  int mode = 0;             // 0 exterior (G_E), 1 interior (G_I)
  int K = 0, M = 0, Kstar = 0, p = 0, nf = 0, nrad = 0, ntheta = 0;
  std::vector<int> bn, bm, bc;       // basis (n, m, cos=0/sin=1)
  std::vector<double> P;             // K x Kstar, row-major
  std::vector<double> zr, zth;       // sampling nodes on the unit disk
  std::vector<double> zloc;          // Kstar x 3 offsets from the centre in the patch frame
  std::vector<double> T;             // p x K
  std::vector<double> st, sth;       // skeleton (t, theta)
  std::vector<double> sloc;          // p x 3 offsets in the patch frame
  std::vector<double> I;             // K
  std::vector<OutRep> reps;          // increasing rho_min; reps[0] equals (T, st, sth, sloc)
  bool sketch_on_device = false;     // the ID sketch was formed on a CUDA device
  bool colloc_on_device = false;     // the collocation matrices were formed on a CUDA device
  std::vector<double> trad;          // radial collocation nodes
  std::vector<double> beta;          // nrad x K radial profiles
  std::vector<double> w;             // nf fine-grid weights
  std::vector<double> colloc;        // (mmax+1) x nrad x nrad when kept
  double seconds_onepatch = 0, seconds_id = 0;
  double seconds_sketch = 0, seconds_cpqr = 0, seconds_assemble = 0;  // parts of seconds_id
  double seconds_colloc = 0, seconds_lu = 0;  // parts of seconds_onepatch: matrices, LUs + solves
};

// Basis ordering: n ascending, then m ascending, cos before sin; first K kept.
void zernike_basis(int K, std::vector<int>& n, std::vector<int>& m, std::vector<int>& c);
double zernike_radial(int n, int m, double r);

// Modal kernels G_n(t, t'), n = 0..nmax, for the on-surface Green's function of the
// given mode (split into Coulomb, log(2/d) and log(1 + d/2) parts, Section 8.1).
void modal_kernels(double t, double tp, int nmax, int mode, double* out);
void modal_coulomb(double t, double tp, int nmax, double* out);   // G^(1)
void modal_log(double t, double tp, int nmax, double* out);       // G^(2)
void modal_log1p(double t, double tp, int nmax, double* out);     // G^(3)

// Runs the full precompute. Throws std::runtime_error on failure.
void precompute(double eps, int mode, int K, const PrecomputeOptions& opt, Precomputed& out);

// Fills P, zr, zth, zloc and the basis only (no one-patch solve); used when the
// outgoing operator is supplied by the caller.
void precompute_zernike(double eps, int K, Precomputed& out);

// Offsets (x - c) in the patch frame for local polar coordinates (t, theta):
// (sin t cos th, sin t sin th, cos t - 1).
void local_offset(double t, double th, double* o);

}  // namespace ncs
