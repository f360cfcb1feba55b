#include "tree.hpp"

#include <stdexcept>

namespace ncs {

void tree_build(const std::vector<double>&, const Precomputed&, const TreeOptions&, TreeHost&) {
  throw std::runtime_error("tree method not available yet");
}
void tree_upload(const TreeHost&, const Precomputed&, TreeDevice&) {}
void tree_free(TreeDevice&) {}
cudaError_t launch_tree_field(const DeviceData&, const TreeDevice&, int, int, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace ncs
