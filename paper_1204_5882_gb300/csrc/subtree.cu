// Subtree decoder launchers, one translation unit per storage type (built in
// parallel); the kernel itself is in subtree_impl.cuh.
#include "subtree_impl.cuh"

namespace polar {

cudaError_t launch_subtree_f16(const SubtreeArgs &a, cudaStream_t s);
cudaError_t launch_subtree_i8(const SubtreeArgs &a, cudaStream_t s);

cudaError_t launch_subtree(const SubtreeArgs &a, cudaStream_t s) {
  if (a.prec == POLAR_FP16) return launch_subtree_f16(a, s);
  if (a.prec == POLAR_INT8) return launch_subtree_i8(a, s);
  return launch_s<float>(a, s);
}

}  // namespace polar
