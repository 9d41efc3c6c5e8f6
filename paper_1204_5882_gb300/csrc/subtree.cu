// Subtree decoder launchers, one translation unit per storage type (built in
// parallel); the kernel itself is in subtree_impl.cuh.
#include "node_impl.cuh"

namespace polar {

cudaError_t launch_subtree_f16(const SubtreeArgs &a, cudaStream_t s);
cudaError_t launch_subtree_i8(const SubtreeArgs &a, cudaStream_t s);
cudaError_t launch_node_f16(const NodeArgs &a, cudaStream_t s);
cudaError_t launch_node_i8(const NodeArgs &a, cudaStream_t s);

cudaError_t launch_subtree(const SubtreeArgs &a, cudaStream_t s) {
  if (a.prec == POLAR_FP16) return launch_subtree_f16(a, s);
  if (a.prec == POLAR_INT8) return launch_subtree_i8(a, s);
  return launch_s<float>(a, s);
}

cudaError_t launch_node(const NodeArgs &a, cudaStream_t s) {
  if (a.prec == POLAR_FP16) return launch_node_f16(a, s);
  if (a.prec == POLAR_INT8) return launch_node_i8(a, s);
  return launch_node_s<float>(a, s);
}

size_t node_smem_bytes_host(int t) { return node_smem_bytes(t); }

}  // namespace polar
