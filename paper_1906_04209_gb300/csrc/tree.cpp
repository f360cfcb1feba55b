// Host construction of the cube-sphere quadtree (Kaye & Greengard, Section 7.2),
// interaction lists, bounding circles and incoming-grid sizes (Section 7.3 and the
// adaptive sizing of "Optimizations and parallelization"), flattened into work lists
// for the device (Step 2 of Section 7).
//
// Levels 0..L: level 0 has the six cube faces, level l has 2^l x 2^l boxes per face,
// and L is the first level at which no box holds more than one patch (empty boxes are
// dropped). Neighbours are the boxes sharing an edge or a corner, wrapping across
// cube edges (a box at a cube corner has seven). The interaction list of a box is the
// set of non-neighbour children of its parent's neighbours (and of its parent); at
// level 0 it is the set of non-neighbour faces. Each ordered pair of distinct patches
// is then accounted for exactly once: in the interaction list of the target's group at
// one level, or as leaf-level neighbours.
//
// For a group whose incoming field is cheaper to keep on a polar grid than to evaluate
// at its members' Zernike nodes, sources are summed onto the grid (P2L) and the grid is
// interpolated at the nodes (L2P); otherwise, and for leaf neighbours, the sources are
// evaluated directly at the Zernike nodes.
#include "tree.hpp"

#include <algorithm>
#include <cmath>
#include <stdexcept>
#include <unordered_map>

#include "numerics.hpp"

namespace ncs {

namespace {

struct BoxId {
  int face, ix, iy;
};

inline uint64_t box_key(int face, int ix, int iy) {
  return ((uint64_t)face << 48) | ((uint64_t)(uint32_t)ix << 24) | (uint64_t)(uint32_t)iy;
}

// Face of a point: axis of largest |coordinate| (lowest axis on ties), sign; the
// face coordinates (u, v) are the other two coordinates (axes a+1, a+2) over |p_a|.
inline void face_coords(const double* p, int* face, double* u, double* v) {
  int a = 0;
  if (std::fabs(p[1]) > std::fabs(p[a])) a = 1;
  if (std::fabs(p[2]) > std::fabs(p[a])) a = 2;
  const double pa = p[a];
  *face = 2 * a + (pa < 0.0 ? 1 : 0);
  const double inv = 1.0 / std::fabs(pa);
  *u = p[(a + 1) % 3] * inv;
  *v = p[(a + 2) % 3] * inv;
}

inline int cell_index(double u, int n) {
  int i = (int)std::floor(0.5 * (u + 1.0) * n);
  return std::min(n - 1, std::max(0, i));
}

// Neighbour of box (face, ix, iy) at level with n = 2^level cells per side, offset
// (dx, dy); false if it falls across a cube corner (no such box).
bool neighbour_box(int face, int ix, int iy, int n, int dx, int dy, BoxId* out) {
  const int jx = ix + dx, jy = iy + dy;
  if (jx >= 0 && jx < n && jy >= 0 && jy < n) {
    *out = {face, jx, jy};
    return true;
  }
  const double u = -1.0 + (jx + 0.5) * 2.0 / n, v = -1.0 + (jy + 0.5) * 2.0 / n;
  if (std::fabs(u) > 1.0 && std::fabs(v) > 1.0) return false;
  const int a = face / 2, b = (a + 1) % 3, c = (a + 2) % 3;
  const double s = (face % 2) ? -1.0 : 1.0;
  double p[3];
  if (std::fabs(u) > 1.0) {  // fold across the edge u = +-1 onto the face normal to e_b
    const double delta = std::fabs(u) - 1.0;
    p[b] = (u > 0) ? 1.0 : -1.0;
    p[a] = s * (1.0 - delta);
    p[c] = v;
  } else {  // fold across v = +-1 onto the face normal to e_c
    const double delta = std::fabs(v) - 1.0;
    p[c] = (v > 0) ? 1.0 : -1.0;
    p[a] = s * (1.0 - delta);
    p[b] = u;
  }
  int f2;
  double u2, v2;
  face_coords(p, &f2, &u2, &v2);
  *out = {f2, cell_index(u2, n), cell_index(v2, n)};
  return true;
}

// Coarsest outgoing representation whose far field starts at or before `dist`.
int select_rep(const Precomputed& pc, double dist) {
  // the last representation whose far region starts at or before dist (radii increase
  // along the ladder), else the first
  int lo = 0, hi = (int)pc.reps.size() - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (pc.reps[mid].rho_min <= dist)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

int rep_p(const Precomputed& pc, int k) { return pc.reps.empty() ? pc.p : pc.reps[k].p; }

double geodesic(const double* a, const double* b) {
  const double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
  return std::atan2(std::sqrt(cx * cx + cy * cy + cz * cz), a[0] * b[0] + a[1] * b[1] + a[2] * b[2]);
}

// Smallest circle enclosing the points p (2-D), randomised incremental algorithm
// (Welzl); returns centre (cx, cy) and radius.
void min_circle(std::vector<std::pair<double, double>>& p, double* cx, double* cy, double* r) {
  // deterministic shuffle
  uint64_t st = 0x9E3779B97F4A7C15ull;
  for (size_t i = p.size(); i > 1; --i) {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    std::swap(p[i - 1], p[(st >> 33) % i]);
  }
  auto inside = [&](double x, double y, double ccx, double ccy, double rr) {
    return (x - ccx) * (x - ccx) + (y - ccy) * (y - ccy) <= rr * rr * (1.0 + 1e-12) + 1e-300;
  };
  double X = p[0].first, Y = p[0].second, Rr = 0.0;
  for (size_t i = 1; i < p.size(); ++i) {
    if (inside(p[i].first, p[i].second, X, Y, Rr)) continue;
    X = p[i].first;
    Y = p[i].second;
    Rr = 0.0;
    for (size_t j = 0; j < i; ++j) {
      if (inside(p[j].first, p[j].second, X, Y, Rr)) continue;
      X = 0.5 * (p[i].first + p[j].first);
      Y = 0.5 * (p[i].second + p[j].second);
      Rr = 0.5 * std::hypot(p[i].first - p[j].first, p[i].second - p[j].second);
      for (size_t k = 0; k < j; ++k) {
        if (inside(p[k].first, p[k].second, X, Y, Rr)) continue;
        // circumcircle of i, j, k
        const double ax = p[i].first, ay = p[i].second, bx = p[j].first, by = p[j].second, qx = p[k].first,
                     qy = p[k].second;
        const double d = 2.0 * (ax * (by - qy) + bx * (qy - ay) + qx * (ay - by));
        if (std::fabs(d) < 1e-300) continue;
        const double a2 = ax * ax + ay * ay, b2 = bx * bx + by * by, q2 = qx * qx + qy * qy;
        X = (a2 * (by - qy) + b2 * (qy - ay) + q2 * (ay - by)) / d;
        Y = (a2 * (qx - bx) + b2 * (ax - qx) + q2 * (bx - ax)) / d;
        Rr = std::hypot(ax - X, ay - Y);
      }
    }
  }
  *cx = X;
  *cy = Y;
  *r = Rr;
}

// Centre of a small enclosing circle of the patch centres `mem` on the sphere: the
// smallest enclosing circle in the gnomonic plane at the mean direction, mapped back.
// Returns the geodesic radius to the farthest member (exact for the returned centre).
double bounding_circle(const std::vector<double>& centres, const std::vector<int>& mem, double* c) {
  double m[3] = {0, 0, 0};
  for (int i : mem)
    for (int a = 0; a < 3; ++a) m[a] += centres[3 * i + a];
  const double nm = std::sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  for (int a = 0; a < 3; ++a) m[a] /= nm;
  for (int a = 0; a < 3; ++a) c[a] = m[a];
  if (mem.size() > 1) {
    double e1[3], e2[3];
    const double ax = -m[1], ay = m[0], na2 = ax * ax + ay * ay;
    if (na2 >= 1e-24) {
      e1[0] = ax / std::sqrt(na2);
      e1[1] = ay / std::sqrt(na2);
      e1[2] = 0.0;
    } else {
      e1[0] = 1.0;
      e1[1] = e1[2] = 0.0;
    }
    e2[0] = m[1] * e1[2] - m[2] * e1[1];
    e2[1] = m[2] * e1[0] - m[0] * e1[2];
    e2[2] = m[0] * e1[1] - m[1] * e1[0];
    std::vector<std::pair<double, double>> pts;
    bool ok = true;
    for (int i : mem) {
      const double* x = &centres[3 * i];
      const double h = x[0] * m[0] + x[1] * m[1] + x[2] * m[2];
      if (h < 0.2) {
        ok = false;
        break;
      }
      pts.push_back({(x[0] * e1[0] + x[1] * e1[1] + x[2] * e1[2]) / h, (x[0] * e2[0] + x[1] * e2[1] + x[2] * e2[2]) / h});
    }
    if (ok) {
      double X, Y, r;
      min_circle(pts, &X, &Y, &r);
      double cc[3];
      for (int a = 0; a < 3; ++a) cc[a] = m[a] + X * e1[a] + Y * e2[a];
      const double nc = std::sqrt(cc[0] * cc[0] + cc[1] * cc[1] + cc[2] * cc[2]);
      double R1 = 0.0, R0 = 0.0;
      for (int a = 0; a < 3; ++a) cc[a] /= nc;
      for (int i : mem) {
        R1 = std::max(R1, geodesic(cc, &centres[3 * i]));
        R0 = std::max(R0, geodesic(m, &centres[3 * i]));
      }
      if (R1 < R0)
        for (int a = 0; a < 3; ++a) c[a] = cc[a];
    }
  }
  double R = 0.0;
  for (int i : mem) R = std::max(R, geodesic(c, &centres[3 * i]));
  return R;
}

struct Level {
  int n = 1;
  std::vector<uint64_t> keys;                   // sorted nonempty box keys
  std::unordered_map<uint64_t, int> index;      // key -> group
  std::vector<std::vector<int>> members;        // patches per group
  std::vector<int> group_of;                    // per patch
  std::vector<std::vector<int>> nbrs;           // neighbour groups (same level)
  std::vector<std::vector<int>> il;             // interaction-list groups (same level)
};

struct Structure {
  std::vector<Level> lv;
};

void build_structure(const std::vector<double>& centres, const TreeOptions& opt, Structure& S) {
  const int N = (int)(centres.size() / 3);
  std::vector<int> face(N);
  std::vector<double> U(N), V(N);
  for (int i = 0; i < N; ++i) face_coords(&centres[3 * i], &face[i], &U[i], &V[i]);
  S.lv.clear();
  for (int l = 0;; ++l) {
    if (l > opt.max_level) throw std::runtime_error("tree: patches too close for the maximum depth");
    Level L;
    L.n = 1 << l;
    L.group_of.resize(N);
    std::vector<std::pair<uint64_t, int>> kp(N);
    for (int i = 0; i < N; ++i) kp[i] = {box_key(face[i], cell_index(U[i], L.n), cell_index(V[i], L.n)), i};
    std::sort(kp.begin(), kp.end());
    size_t maxocc = 0;
    for (size_t s = 0; s < kp.size();) {
      size_t e = s;
      while (e < kp.size() && kp[e].first == kp[s].first) ++e;
      const int g = (int)L.keys.size();
      L.keys.push_back(kp[s].first);
      L.index[kp[s].first] = g;
      L.members.emplace_back();
      for (size_t q = s; q < e; ++q) {
        L.members.back().push_back(kp[q].second);
        L.group_of[kp[q].second] = g;
      }
      maxocc = std::max(maxocc, e - s);
      s = e;
    }
    S.lv.push_back(std::move(L));
    if (maxocc <= 1) break;
  }
  const int nl = (int)S.lv.size();
  // neighbours (each group's list written by one thread; the box index is only read)
  for (int l = 0; l < nl; ++l) {
    Level& L = S.lv[l];
    L.nbrs.resize(L.keys.size());
    const int64_t ng = (int64_t)L.keys.size();
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t g = 0; g < ng; ++g) {
      const uint64_t k = L.keys[g];
      const int f = (int)(k >> 48), ix = (int)((k >> 24) & 0xffffff), iy = (int)(k & 0xffffff);
      for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy) {
          if (!dx && !dy) continue;
          BoxId b;
          if (!neighbour_box(f, ix, iy, L.n, dx, dy, &b)) continue;
          auto it = L.index.find(box_key(b.face, b.ix, b.iy));
          if (it != L.index.end()) L.nbrs[g].push_back(it->second);
        }
      std::sort(L.nbrs[g].begin(), L.nbrs[g].end());
      L.nbrs[g].erase(std::unique(L.nbrs[g].begin(), L.nbrs[g].end()), L.nbrs[g].end());
    }
  }
  // interaction lists
  for (int l = 0; l < nl; ++l) {
    Level& L = S.lv[l];
    L.il.resize(L.keys.size());
    const int64_t ng = (int64_t)L.keys.size();
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t g = 0; g < ng; ++g) {
      std::vector<int> cand;
      if (l == 0) {
        for (size_t h = 0; h < L.keys.size(); ++h) cand.push_back((int)h);
      } else {
        const Level& P = S.lv[l - 1];
        const uint64_t k = L.keys[g];
        const int f = (int)(k >> 48), ix = (int)((k >> 24) & 0xffffff), iy = (int)(k & 0xffffff);
        const int pg = P.index.at(box_key(f, ix / 2, iy / 2));
        std::vector<int> pset = P.nbrs[pg];
        pset.push_back(pg);
        for (int q : pset) {
          const uint64_t pk = P.keys[q];
          const int pf = (int)(pk >> 48), px = (int)((pk >> 24) & 0xffffff), py = (int)(pk & 0xffffff);
          for (int cx = 0; cx < 2; ++cx)
            for (int cy = 0; cy < 2; ++cy) {
              auto it = L.index.find(box_key(pf, 2 * px + cx, 2 * py + cy));
              if (it != L.index.end()) cand.push_back(it->second);
            }
        }
      }
      std::sort(cand.begin(), cand.end());
      cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
      for (int h : cand)
        if (h != (int)g && !std::binary_search(L.nbrs[g].begin(), L.nbrs[g].end(), h)) L.il[g].push_back(h);
    }
  }
}

// Incoming-grid size for a group of radius R whose nearest source is at geodesic
// distance D from the centre: the angular Fourier coefficients of a point source there
// decay like (R/D)^m and its radial parity-restricted Chebyshev coefficients like
// rho_B^-k with rho_B = rho + sqrt(rho^2 - 1), rho = D/R. The grid keeps the modes and
// degrees up to the first trailing coefficient below tol (Section 7.3).
GridShape grid_size(double R, double D, double tol) {
  const double rho = D / R;
  const double lt = std::log(1.0 / tol);
  const int m = (int)std::ceil(lt / std::log(rho));
  int nth = 2 * m + 2;
  nth = (nth + 3) / 4 * 4;
  const double rb = rho + std::sqrt(rho * rho - 1.0);
  const int d = (int)std::ceil(lt / std::log(rb));
  int nr = (d + 2) / 2;
  GridShape s;
  s.nr = std::min(64, std::max(2, nr));
  s.nth = std::min(512, std::max(8, nth));
  return s;
}

}  // namespace

void tree_build(const std::vector<double>& centres, const Precomputed& pc, const TreeOptions& opt, TreeHost& t) {
  const int N = (int)(centres.size() / 3);
  Structure S;
  build_structure(centres, opt, S);
  const int nl = (int)S.lv.size();
  t = TreeHost();
  t.levels = nl;
  const double eps = opt.eps;
  std::vector<std::vector<int>> direct(N);
  std::vector<std::vector<int>> pgroups(N);
  std::vector<std::pair<int, int>> shape_ids;  // (nr, nth) -> index
  auto shape_index = [&](GridShape s) {
    for (size_t i = 0; i < t.shapes.size(); ++i)
      if (t.shapes[i].nr == s.nr && t.shapes[i].nth == s.nth) return (int)i;
    t.shapes.push_back(s);
    return (int)t.shapes.size() - 1;
  };
  const int CH = std::max(1, opt.item_patches);  // source patches per P2L work item
  // Bounding circles (Section 7.3) of every group: smallest enclosing circle of the
  // members' centres in the gnomonic plane at their mean direction, radius + eps; then,
  // bottom-up, each radius grows until the disk contains the disks of its children that
  // may keep a grid, so that grid disks nest along the tree (needed by the downward pass).
  std::vector<std::vector<double>> gcirc(nl), grad(nl);
  for (int l = 0; l < nl; ++l) {
    const Level& L = S.lv[l];
    gcirc[l].resize(3 * L.keys.size());
    grad[l].resize(L.keys.size());
    const int64_t ng = (int64_t)L.keys.size();
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t g = 0; g < ng; ++g)
      grad[l][g] = bounding_circle(centres, L.members[g], &gcirc[l][3 * g]) + eps * (1.0 + 1e-9);
  }
  for (int l = nl - 1; l >= 1; --l) {
    const Level& L = S.lv[l];
    const Level& P = S.lv[l - 1];
    for (size_t g = 0; g < L.keys.size(); ++g) {
      // a single-patch group never keeps a grid, and its patch already lies in the
      // parent's disk (which includes eps around every member centre)
      if ((int)L.members[g].size() < opt.grid_min_members) continue;
      const int pg = P.group_of[L.members[g][0]];
      const double need = geodesic(&gcirc[l - 1][3 * pg], &gcirc[l][3 * g]) + grad[l][g];
      grad[l - 1][pg] = std::max(grad[l - 1][pg], need * (1.0 + 1e-12));
    }
  }
  // Per level, every group's plan (its interaction-list sources by distance, grid or
  // direct) is formed in parallel; the grid groups are then appended in group order, so
  // the lists do not depend on the thread count. A patch is a member of one group per
  // level, so the direct lists of a level's groups touch disjoint patches.
  struct GroupPlan {
    bool grid = false;
    GridShape gs;
    std::vector<int> srcs;     // sources sorted by distance from the circle centre
    std::vector<double> dist;  // their distances
  };
  for (int l = 0; l < nl; ++l) {
    const Level& L = S.lv[l];
    const int64_t ng = (int64_t)L.keys.size();
    std::vector<GroupPlan> plan(ng);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t g = 0; g < ng; ++g) {
      if (L.il[g].empty()) continue;
      const std::vector<int>& mem = L.members[g];
      std::vector<int> srcs;
      for (int h : L.il[g])
        for (int j : L.members[h]) srcs.push_back(j);
      const double* c = &gcirc[l][3 * g];
      const double R = grad[l][g];
      // sources sorted by distance, so that P2L work items hold similar distances
      std::vector<std::pair<double, int>> sd;
      sd.reserve(srcs.size());
      for (int j : srcs) sd.push_back({geodesic(c, &centres[3 * j]), j});
      std::sort(sd.begin(), sd.end());
      for (size_t q = 0; q < sd.size(); ++q) srcs[q] = sd[q].second;
      const double D = sd.front().first - eps;
      // grid or direct, by the pair-evaluation count of each (an L2P node-grid product
      // costs about a tenth of a kernel evaluation)
      bool use_grid = false;
      GridShape gs;
      if ((int)mem.size() >= opt.grid_min_members && D > 1.15 * R) {
        gs = grid_size(R, D, opt.grid_tol);
        double psum_grid = 0.0, psum_direct = 0.0;  // sums of integers: exact in any order
        for (size_t s = 0; s < sd.size(); s += CH)
          psum_grid += (double)(std::min(sd.size(), s + CH) - s) * rep_p(pc, select_rep(pc, sd[s].first - R));
        for (size_t q = 0; q < sd.size(); ++q) psum_direct += rep_p(pc, select_rep(pc, sd[q].first - R));
        const double cost_grid = gs.q() * psum_grid + opt.l2p_weight * (double)mem.size() * pc.Kstar * gs.q();
        const double cost_direct = (double)mem.size() * pc.Kstar * psum_direct;
        use_grid = cost_grid < cost_direct;
      }
      if (!use_grid) {
        for (int i : mem) direct[i].insert(direct[i].end(), srcs.begin(), srcs.end());
        continue;
      }
      GroupPlan& P = plan[g];
      P.grid = true;
      P.gs = gs;
      P.dist.resize(sd.size());
      for (size_t q = 0; q < sd.size(); ++q) P.dist[q] = sd[q].first;
      P.srcs = std::move(srcs);
    }
    for (int64_t g = 0; g < ng; ++g) {
      GroupPlan& P = plan[g];
      if (!P.grid) continue;
      const GridShape gs = P.gs;
      const double R = grad[l][g];
      const int gi = (int)t.gR.size();
      t.gcen.insert(t.gcen.end(), &gcirc[l][3 * g], &gcirc[l][3 * g] + 3);
      t.gR.push_back(R);
      t.glevel.push_back(l);
      t.gshape.push_back(shape_index(gs));
      t.goff.push_back(t.total_grid_points);
      t.total_grid_points += gs.q();
      for (size_t s = 0; s < P.srcs.size(); s += CH) {
        const size_t e = std::min(P.srcs.size(), s + CH);
        // grid points lie within R of the centre: every source of the item is at least
        // (its distance - R) away from them
        const int k = select_rep(pc, P.dist[s] - R);
        t.witem_group.push_back(gi);
        t.witem_rep.push_back(k);
        t.witem_lo.push_back((int64_t)t.isrc.size() + (int64_t)s);
        t.witem_hi.push_back((int64_t)t.isrc.size() + (int64_t)e);
        t.p2l_pairs += (int64_t)(e - s) * rep_p(pc, k) * gs.q();
      }
      t.isrc.insert(t.isrc.end(), P.srcs.begin(), P.srcs.end());
      for (int i : L.members[g]) {
        pgroups[i].push_back(gi);
        t.l2p_evals += (int64_t)pc.Kstar * gs.q();
      }
      std::vector<int>().swap(P.srcs);
      std::vector<double>().swap(P.dist);
    }
  }
  // leaf neighbours (Step 3), evaluated at the Zernike nodes
  {
    const Level& L = S.lv[nl - 1];
    for (size_t g = 0; g < L.keys.size(); ++g)
      for (int h : L.nbrs[g])
        for (int i : L.members[g])
          for (int j : L.members[h]) direct[i].push_back(j);
  }
  // Downward pass (a GB300-side reorganisation of Step 3.4): each grid group receives
  // the field of its nearest grid ancestor by interpolation at its own grid points when
  // its whole grid disk lies inside the ancestor's disk; a patch then interpolates only
  // its deepest grid, plus any ancestor whose link could not be made.
  const int G = (int)t.gR.size();
  {
    std::vector<int> parent(G, -1);
    std::vector<char> linked(G, 0);
    for (int i = 0; i < N; ++i)
      for (size_t a = 1; a < pgroups[i].size(); ++a) parent[pgroups[i][a]] = pgroups[i][a - 1];
    for (int g = 0; g < G; ++g) {
      const int a = parent[g];
      if (a < 0) continue;
      const double dist = geodesic(&t.gcen[3 * a], &t.gcen[3 * g]);
      linked[g] = (dist + t.gR[g] <= t.gR[a] * (1.0 - 1e-12)) ? 1 : 0;
    }
    t.gl_off.assign(nl + 1, 0);
    for (int g = 0; g < G; ++g) t.gl_off[t.glevel[g] + 1]++;
    for (int l = 0; l < nl; ++l) t.gl_off[l + 1] += t.gl_off[l];
    std::vector<std::vector<std::pair<int, int>>> bylevel(nl);
    for (int g = 0; g < G; ++g)
      if (linked[g]) {
        bylevel[t.glevel[parent[g]]].push_back({g, parent[g]});
        t.l2l_evals += (int64_t)t.shapes[t.gshape[g]].q() * t.shapes[t.gshape[parent[g]]].q();
      }
    t.l2l_off.assign(nl + 1, 0);
    for (int l = 0; l < nl; ++l) {
      for (auto& cp : bylevel[l]) {
        t.l2l_child.push_back(cp.first);
        t.l2l_parent.push_back(cp.second);
      }
      t.l2l_off[l + 1] = (int)t.l2l_child.size();
    }
    t.l2p_evals = 0;
    for (int i = 0; i < N; ++i) {
      if (pgroups[i].empty()) continue;
      std::vector<int> keep;
      int cur = pgroups[i].back();
      keep.push_back(cur);
      while (parent[cur] >= 0) {
        if (!linked[cur]) keep.push_back(parent[cur]);
        cur = parent[cur];
      }
      pgroups[i] = keep;
      for (int g : keep) t.l2p_evals += (int64_t)pc.Kstar * t.shapes[t.gshape[g]].q();
    }
  }
  t.pd_off.assign(N + 1, 0);
  t.pg_off.assign(N + 1, 0);
#pragma omp parallel for schedule(dynamic, 256)
  for (int i = 0; i < N; ++i) std::sort(direct[i].begin(), direct[i].end());
  for (int i = 0; i < N; ++i) {
    t.pd_off[i + 1] = t.pd_off[i] + (int64_t)direct[i].size();
    t.pg_off[i + 1] = t.pg_off[i] + (int64_t)pgroups[i].size();
  }
  t.pd.resize(t.pd_off[N]);
  t.pdk.resize(t.pd_off[N]);
  t.pg.reserve(t.pg_off[N]);
  int64_t dpairs = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : dpairs)
  for (int i = 0; i < N; ++i) {
    int64_t o = t.pd_off[i];
    for (int j : direct[i]) {
      // the Zernike nodes of patch i lie within eps of its centre
      const int k = select_rep(pc, geodesic(&centres[3 * i], &centres[3 * j]) - eps);
      t.pd[o] = j;
      t.pdk[o] = k;
      ++o;
      dpairs += (int64_t)rep_p(pc, k) * pc.Kstar;
    }
  }
  t.direct_pairs = dpairs;
  for (int i = 0; i < N; ++i) t.pg.insert(t.pg.end(), pgroups[i].begin(), pgroups[i].end());
  t.pairs_per_matvec = t.p2l_pairs + t.direct_pairs;
}

void tree_pairs(const std::vector<double>& centres, const Precomputed& pc, const TreeOptions& opt,
                std::vector<int>& tgt, std::vector<int>& src, std::vector<int>& level, std::vector<int>& kind) {
  (void)pc;
  Structure S;
  build_structure(centres, opt, S);
  const int nl = (int)S.lv.size();
  tgt.clear();
  src.clear();
  level.clear();
  kind.clear();
  for (int l = 0; l < nl; ++l) {
    const Level& L = S.lv[l];
    for (size_t g = 0; g < L.keys.size(); ++g)
      for (int h : L.il[g])
        for (int i : L.members[g])
          for (int j : L.members[h]) {
            tgt.push_back(i);
            src.push_back(j);
            level.push_back(l);
            kind.push_back(0);
          }
  }
  const Level& L = S.lv[nl - 1];
  for (size_t g = 0; g < L.keys.size(); ++g)
    for (int h : L.nbrs[g])
      for (int i : L.members[g])
        for (int j : L.members[h]) {
          tgt.push_back(i);
          src.push_back(j);
          level.push_back(nl - 1);
          kind.push_back(2);
        }
}

}  // namespace ncs
