// Cube-sphere quadtree, interaction lists and incoming grids (Kaye & Greengard,
// Sections 7.2-7.3, Step 2 of Section 7) and the device copy used by the tree product.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "precompute.hpp"

namespace ncs {

struct DeviceData;

struct TreeOptions {
  double eps = 0.0;
  double grid_tol = 1e-8;  // incoming-grid tolerance
  int max_level = 24;
  int grid_min_members = 2;  // groups with fewer patches evaluate directly at the Zernike nodes
  int item_patches = 16;     // interaction-list source patches per P2L work item
  double l2p_weight = 0.1;   // cost of one L2P node-grid product in kernel evaluations, used
                             // when a group chooses between a grid and direct evaluation
};

// Launch configuration of the FP32 pair kernels of the tree product (results differ only
// by the order of FP32 sums and by the logarithm's approximation, both within the FP32
// product's accuracy). Chosen per workload by ncs_tune.
struct KernelConfig {
  int p2l_tile = 16;    // source patches per shared-memory tile of a P2L work item: 8 or 16
  int p2l_poly = 4;     // of every 16 packed pair chains, how many take lg2 on the FMA pipe:
                        // 0, 2, 4 or 6 (the rest on the MUFU unit)
  int direct_poly = 4;  // the same for the direct lists
  int p2l_rsq = 0;      // of every 16 chains, how many take the reciprocal square root by
                        // Newton steps on the FMA pipe: 0, 4 or 8
  int direct_rsq = 0;   // the same for the direct lists
};
bool kernel_config_valid(const KernelConfig& k);

// One incoming-grid shape: n_r parity-restricted Chebyshev radii x n_theta angles.
struct GridShape {
  int nr = 0, nth = 0;
  int q() const { return nr * nth; }
};

struct TreeHost {
  int levels = 0;  // number of levels (0 .. levels-1); the last is the leaf level
  // ---- grid groups (patch groups whose incoming field is kept on a polar grid)
  std::vector<double> gcen;      // 3 per group: bounding-circle centre (unit)
  std::vector<double> gR;        // bounding-circle radius (geodesic)
  std::vector<int> glevel;       // level of the group
  std::vector<int> gshape;       // index into shapes
  std::vector<int64_t> goff;     // offset of the group's q grid values / coefficients
  std::vector<GridShape> shapes;
  // P2L work items: (grid group, range of source patches in isrc)
  std::vector<int> witem_group;
  std::vector<int> witem_rep;    // outgoing representation used by the item's sources
  std::vector<int64_t> witem_lo, witem_hi;
  std::vector<int> isrc;         // source patch indices (concatenated interaction lists)
  // L2P: for every patch, the grid groups it belongs to (CSR)
  std::vector<int64_t> pg_off;
  std::vector<int> pg;
  // direct part: for every patch, the source patches evaluated at its Zernike nodes (CSR)
  std::vector<int64_t> pd_off;
  std::vector<int> pd;
  std::vector<int> pdk;          // representation per direct entry
  // downward pass (grid-to-grid interpolation into the nearest grid descendants)
  std::vector<int> gl_off;       // levels+1: grid groups of level l are [gl_off[l], gl_off[l+1])
  std::vector<int> l2l_child, l2l_parent;  // links, grouped by the parent's level
  std::vector<int> l2l_off;      // levels+1
  int64_t l2l_evals = 0;         // child grid points x parent grid size
  // statistics
  int64_t total_grid_points = 0;
  int64_t pairs_per_matvec = 0;  // kernel evaluations (P2L + direct)
  int64_t p2l_pairs = 0, direct_pairs = 0, l2p_evals = 0;
  // for host-side checks: per level, for every patch, its box index and the
  // interaction-list / neighbour relation encoded as (target patch, source patch, level, kind)
  std::vector<int64_t> box_of;   // levels x N box ids
};

struct TreeDevice {
  int ngroups = 0, nitems = 0, nshapes = 0;
  int64_t ngrid = 0;
  int64_t N = 0;
  double* gcen = nullptr;        // 3*G
  double* gR = nullptr;
  int* gshape = nullptr;
  int64_t* goff = nullptr;
  int* shape_nr = nullptr;       // per shape
  int* shape_nth = nullptr;
  int* witem_group = nullptr;
  int* witem_rep = nullptr;
  int64_t* witem_lo = nullptr;
  int64_t* witem_hi = nullptr;
  int* isrc = nullptr;
  int64_t* pg_off = nullptr;
  int* pg = nullptr;
  int64_t* pd_off = nullptr;
  int* pd = nullptr;
  int* pdk = nullptr;
  double* gpos64 = nullptr;      // 3*ngrid grid-point offsets from the group centre
  float* gpos32 = nullptr;
  float* gframe = nullptr;       // 9*G: rows f1, f2, g of each group's frame (FP32)
  int* l2l_child = nullptr;
  int* l2l_parent = nullptr;
  std::vector<int> gl_off, l2l_off;  // host copies of the per-level ranges
  double* grid = nullptr;        // ngrid values (FP64 accumulation for both precisions)
  double* coef = nullptr;        // ngrid coefficients
  int max_q = 0, max_nr = 0, max_nth = 0;
  KernelConfig cfg;              // FP32 pair-kernel variants
};

void tree_build(const std::vector<double>& centres, const Precomputed& pc, const TreeOptions& opt, TreeHost& t);

// All (target, source) patch pairs the tree accounts for, with the level and
// kind (0 = interaction list on a grid, 1 = interaction list direct, 2 = leaf
// neighbour); used by the covering check.
void tree_pairs(const std::vector<double>& centres, const Precomputed& pc, const TreeOptions& opt,
                std::vector<int>& tgt, std::vector<int>& src, std::vector<int>& level, std::vector<int>& kind);

void tree_upload(const TreeHost& t, const Precomputed& pc, TreeDevice& d);
void tree_free(TreeDevice& d);
// ev (optional, 5 events): recorded before P2L, after P2L, after coef, after direct, after L2P.
cudaError_t launch_tree_field(const DeviceData& d, const TreeDevice& t, int mode, int prec, cudaStream_t s,
                              cudaEvent_t* ev = nullptr);

}  // namespace ncs
