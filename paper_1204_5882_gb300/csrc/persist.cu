// Persistent decoder launchers: float32 storage here, FP16 and INT8 storage
// in their own translation units (built in parallel); the kernels are in
// persist_impl.cuh.
#include "persist_impl.cuh"

namespace polar {

cudaError_t launch_persistent_f16(int fkind, bool uhat, const PFrame *frames, uint32_t count,
                                  uint32_t *head, float *scratch, uint64_t cta_floats, int t,
                                  int grid, double int8_target, cudaStream_t s);
cudaError_t launch_persistent_i8(int fkind, bool uhat, const PFrame *frames, uint32_t count,
                                 uint32_t *head, float *scratch, uint64_t cta_floats, int t,
                                 int grid, double int8_target, cudaStream_t s);
int persistent_ctas_per_sm_f16(int fkind, bool uhat, int t);
int persistent_ctas_per_sm_i8(int fkind, bool uhat, int t);
cudaError_t launch_serve_f16(int fkind, ServeArgs a, int t, int grid, cudaStream_t s);
cudaError_t launch_serve_i8(int fkind, ServeArgs a, int t, int grid, cudaStream_t s);
int serve_ctas_per_sm_f16(int fkind, int t);
int serve_ctas_per_sm_i8(int fkind, int t);

size_t persistent_smem_bytes(int t) { return persist_smem(t); }

int persistent_ctas_per_sm(int prec, int fkind, bool uhat, int t) {
  if (prec == POLAR_FP16) return persistent_ctas_per_sm_f16(fkind, uhat, t);
  if (prec == POLAR_INT8) return persistent_ctas_per_sm_i8(fkind, uhat, t);
  return persistent_ctas_per_sm_s<float>(fkind, uhat, t);
}

cudaError_t launch_persistent(int prec, int fkind, bool uhat, const PFrame *frames,
                              uint32_t count, uint32_t *head, float *scratch,
                              uint64_t cta_floats, int t, int grid, double int8_target,
                              cudaStream_t s) {
  if (prec == POLAR_FP16)
    return launch_persistent_f16(fkind, uhat, frames, count, head, scratch, cta_floats, t, grid,
                                 int8_target, s);
  if (prec == POLAR_INT8)
    return launch_persistent_i8(fkind, uhat, frames, count, head, scratch, cta_floats, t, grid,
                                int8_target, s);
  return launch_persistent_s<float>(fkind, uhat, frames, count, head, scratch, cta_floats, t,
                                    grid, int8_target, s);
}

int serve_ctas_per_sm(int prec, int fkind, int t) {
  if (prec == POLAR_FP16) return serve_ctas_per_sm_f16(fkind, t);
  if (prec == POLAR_INT8) return serve_ctas_per_sm_i8(fkind, t);
  return serve_ctas_per_sm_s<float>(fkind, t);
}

cudaError_t launch_serve(int prec, int fkind, ServeArgs a, int t, int grid, cudaStream_t s) {
  if (prec == POLAR_FP16) return launch_serve_f16(fkind, a, t, grid, s);
  if (prec == POLAR_INT8) return launch_serve_i8(fkind, a, t, grid, s);
  return launch_serve_s<float>(fkind, a, t, grid, s);
}

}  // namespace polar
