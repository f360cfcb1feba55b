// Cube-sphere quadtree (Kaye & Greengard, Section 7.2) and its device copy.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "precompute.hpp"

namespace ncs {

struct DeviceData;

struct TreeOptions {
  double eps = 0.0;
  double grid_tol = 1e-8;
};

struct TreeHost {
  int levels = 0;
  int64_t total_grid_points = 0;
  int64_t pairs_per_matvec = 0;
};

struct TreeDevice {
  int levels = 0;
};

void tree_build(const std::vector<double>& centres, const Precomputed& pc, const TreeOptions& opt, TreeHost& t);
void tree_upload(const TreeHost& t, const Precomputed& pc, TreeDevice& d);
void tree_free(TreeDevice& d);
cudaError_t launch_tree_field(const DeviceData& d, const TreeDevice& t, int mode, int prec, cudaStream_t s);

}  // namespace ncs
