// INT8-storage instantiation of the subtree decoder (see subtree_impl.cuh).
#include "node_impl.cuh"

namespace polar {
cudaError_t launch_subtree_i8(const SubtreeArgs &a, cudaStream_t s) { return launch_s<int8_t>(a, s); }
cudaError_t launch_node_i8(const NodeArgs &a, cudaStream_t s) { return launch_node_s<int8_t>(a, s); }
}  // namespace polar
