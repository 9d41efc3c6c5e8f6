// FP16-storage instantiation of the subtree decoder (see subtree_impl.cuh).
#include "node_impl.cuh"

namespace polar {
cudaError_t launch_subtree_f16(const SubtreeArgs &a, cudaStream_t s) { return launch_s<__half>(a, s); }
cudaError_t launch_node_f16(const NodeArgs &a, cudaStream_t s) { return launch_node_s<__half>(a, s); }
}  // namespace polar
