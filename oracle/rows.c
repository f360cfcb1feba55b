/*
 * Plain-C FP64 compressed sums at sampled target nodes, for large N.
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle (see oracle/__init__.py); the
 * product path never links or calls it.
 *
 * For each requested (patch i, node k) it evaluates, with no tree and no
 * blocking beyond a loop over source patches,
 *     z_i(k) = sum_{j != i} sum_m G(x^z_{i,k}, x_{j,pi(m)}) rho_{j,m},   rho_j = T f_j
 * (Kaye & Greengard, Section 7.1, eq. Tmap and eq. outgoingcompressed), with the
 * on-surface Green's functions of Section 2.1 (eqs. Gextonsurface / Gintonsurface)
 * written as 2/d -+ log(2/d) - log(1 + d/2).
 *
 * Patch frame for centre c: e1 = (z x c)/|z x c| (x-axis at the poles), e2 = c x e1;
 * local (t, theta) -> cos t c + sin t (cos theta e1 + sin theta e2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static void frame(const double *c, double *e1, double *e2) {
  double ax = -c[1], ay = c[0], na2 = ax * ax + ay * ay;
  if (na2 >= 1e-24) {
    double na = sqrt(na2);
    e1[0] = ax / na;
    e1[1] = ay / na;
    e1[2] = 0.0;
  } else {
    e1[0] = 1.0;
    e1[1] = 0.0;
    e1[2] = 0.0;
  }
  e2[0] = c[1] * e1[2] - c[2] * e1[1];
  e2[1] = c[2] * e1[0] - c[0] * e1[2];
  e2[2] = c[0] * e1[1] - c[1] * e1[0];
}

static void local_point(const double *c, double t, double th, double *x) {
  double e1[3], e2[3];
  frame(c, e1, e2);
  double ct = cos(t), st = sin(t), cth = cos(th), sth = sin(th);
  for (int a = 0; a < 3; ++a) x[a] = ct * c[a] + st * (cth * e1[a] + sth * e2[a]);
}

static double green(double d, int mode) {
  double s = (mode == 0) ? -1.0 : 1.0;
  return 2.0 / d + s * log(2.0 / d) - log1p(0.5 * d);
}

/*
 * N, K, p, mode; centres (N*3); T (p*K row-major); skel_t, skel_th (p);
 * x (N*K); eps; targets: ntarget pairs (patch, node) with node (r, theta) on the
 * unit disk given in node_r, node_th (per target); out: ntarget values.
 */
int ncs_oracle_rows(int64_t N, int K, int p, int mode, const double *centres, const double *T,
                    const double *skel_t, const double *skel_th, const double *x, double eps,
                    int64_t ntarget, const int64_t *tpatch, const double *node_r, const double *node_th,
                    double *out) {
  double *rho = (double *)malloc(sizeof(double) * (size_t)N * p);
  double *src = (double *)malloc(sizeof(double) * (size_t)N * p * 3);
  if (!rho || !src) {
    free(rho);
    free(src);
    return -1;
  }
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < N; ++j) {
    for (int m = 0; m < p; ++m) {
      double s = 0.0;
      for (int k = 0; k < K; ++k) s += T[(size_t)m * K + k] * x[(size_t)j * K + k];
      rho[(size_t)j * p + m] = s;
      local_point(&centres[3 * j], skel_t[m], skel_th[m], &src[3 * ((size_t)j * p + m)]);
    }
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < ntarget; ++q) {
    const int64_t i = tpatch[q];
    double xt[3];
    local_point(&centres[3 * i], eps * node_r[q], node_th[q], xt);
    double acc = 0.0;
    for (int64_t j = 0; j < N; ++j) {
      if (j == i) continue;
      const double *sj = &src[3 * (size_t)j * p];
      const double *rj = &rho[(size_t)j * p];
      for (int m = 0; m < p; ++m) {
        double dx = xt[0] - sj[3 * m], dy = xt[1] - sj[3 * m + 1], dz = xt[2] - sj[3 * m + 2];
        acc += green(sqrt(dx * dx + dy * dy + dz * dz), mode) * rj[m];
      }
    }
    out[q] = acc;
  }
  free(rho);
  free(src);
  return 0;
}
