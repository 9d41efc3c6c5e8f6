// INT8-storage instantiation of the persistent decoder (see persist_impl.cuh).
#include "persist_impl.cuh"

namespace polar {
cudaError_t launch_persistent_i8(int fkind, bool uhat, const PFrame *frames, uint32_t count,
                                  uint32_t *head, float *scratch, uint64_t cta_floats, int t,
                                  int grid, double int8_target, cudaStream_t s) {
  return launch_persistent_s<int8_t>(fkind, uhat, frames, count, head, scratch, cta_floats, t, grid,
                                  int8_target, s);
}
int persistent_ctas_per_sm_i8(int fkind, bool uhat, int t) {
  return persistent_ctas_per_sm_s<int8_t>(fkind, uhat, t);
}
cudaError_t launch_serve_i8(int fkind, ServeArgs a, int t, int grid, cudaStream_t s) {
  return launch_serve_s<int8_t>(fkind, a, t, grid, s);
}
int serve_ctas_per_sm_i8(int fkind, int t) { return serve_ctas_per_sm_s<int8_t>(fkind, t); }
}  // namespace polar
