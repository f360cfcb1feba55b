// The modal collocation matrices of the one-patch solve (Kaye & Greengard, Section 8.2,
// eq. modalinteqn) on the device. Host-only interface (no CUDA types).
//
// Row i, panel j, mode n: A_n(i, j*nord + k) = sum_q wt_q L_k(s_q) G_n(t_i, t'_q), where
// t'_q runs over the quadrature nodes of (i, j) (graded toward t_i, and toward the patch
// edge on the Gauss-Jacobi panel), wt_q = 2 pi w_q sin t'_q, L_k is panel j's Lagrange
// basis at the panel coordinate s_q, already multiplied by colscale (sqrt(eps - t_k) on
// the Jacobi panel, whose unknowns are g = sigma sqrt(eps - t)), and
// G_n = G^(1)_n + s G^(2)_n - G^(3)_n with G^(3)_n from the theta rule.
#pragma once

#include <string>
#include <vector>

namespace ncs {

struct CollocProblem {
  int nr = 0, npan = 0, nord = 0;  // collocation nodes = npan * nord
  int nmodes = 0;                  // modes n = 0..nmodes-1
  int mode = 0;                    // 0 exterior (s = -1), 1 interior (s = +1)
  std::vector<double> tr;          // nr collocation nodes
  std::vector<double> colscale;    // nr column factors
  std::vector<double> lag_nodes;   // 2 x nord: Gauss-Legendre then Gauss-Jacobi nodes on [-1, 1]
  std::vector<double> lag_bw;      // 2 x nord barycentric weights of those node sets
  std::vector<int> qoff;           // nr * npan + 1 offsets of the (i, j) node ranges, (i, j) row-major
  std::vector<double> tq, wt, ls;  // per quadrature node: t', 2 pi w sin t', panel coordinate
  std::vector<double> hs2;         // theta rule: sin^2(theta / 2), nth values
  std::vector<double> cw;          // theta rule: cos(n theta) w / pi, nth x nmodes row-major
};

// Largest nord and nmodes the device kernel takes (the host path covers the rest).
constexpr int kCollocMaxOrd = 32;
constexpr int kCollocMaxModes = 64;

// Fills A (nmodes x nr x nr, row-major per mode) on the current CUDA device. Returns 1 on
// success, 0 if no device is usable, its buffers cannot be allocated or the sizes exceed
// the kernel's limits (A untouched), -1 on a CUDA error after that (message in *err).
int colloc_assemble_device(const CollocProblem& p, std::vector<double>& A, std::string* err);

}  // namespace ncs
