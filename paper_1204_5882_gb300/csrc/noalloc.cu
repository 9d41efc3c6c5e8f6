// Decoding without any device allocation, for callers that cannot allocate
// device memory themselves or through this library: processes whose device
// memory is all owned by another framework's fixed-size pool, latency-
// critical loops that cannot afford the implicit device synchronisation of
// cudaMalloc / cudaFree, and long-running services that must not meet an
// out-of-memory error in the middle of a session.
//
// The level scratch and the device copy of the frozen mask live in one
// file-scope device array of fixed size.  Every GPU that loads this library
// holds that array until the process exits.  With CUDA's lazy module loading
// (the default) the array is taken from device memory when the first call on
// a device looks up its address, so that first call should come before a
// caller's pool claims all of the device's memory; if no room is left then,
// the call returns POLAR_ENOMEM.
#include <cstdio>
#include <mutex>

#include "polar_internal.h"

#define POLAR_STATIC_SCRATCH_BYTES (16u << 20)

static __device__ __align__(256) unsigned char g_polar_static_scratch[POLAR_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_ptr[kMaxDevices];

// Device address of the array on the current device.  The host-side symbol
// is only a stand-in and must never reach a kernel; the real address is
// looked up once per device, with that device current.
int static_scratch(int dev, unsigned char **out) {
  if (dev < 0 || dev >= kMaxDevices) return POLAR_EINVAL;
  std::lock_guard<std::mutex> g(g_static_mu);
  if (!g_static_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_polar_static_scratch);
    if (e != cudaSuccess || !p) {
      polar::set_last_error(e != cudaSuccess ? cudaGetErrorString(e)
                                             : "no device address for the static array");
      cudaGetLastError();                 // reported here; leave no stale error behind
      return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : POLAR_ECUDA;
    }
    g_static_ptr[dev] = p;
  }
  *out = static_cast<unsigned char *>(g_static_ptr[dev]);
  return POLAR_OK;
}

}  // namespace

extern "C" size_t polar_static_scratch_bytes(void) { return POLAR_STATIC_SCRATCH_BYTES; }

extern "C" int polar_sc_decode_many_noalloc(const polar_frozen_set *fs, int nframes,
                                            const float *llr_dev,
                                            const uint32_t *frozen_vals_dev,
                                            uint32_t *xhat_dev, uint32_t *uhat_dev,
                                            polar_fkind fkind, polar_prec prec, void *stream) {
  if (!fs || nframes < 1 || !llr_dev || !frozen_vals_dev || !xhat_dev) return POLAR_EINVAL;
  if (prec != POLAR_FP32 && prec != POLAR_FP16 && prec != POLAR_INT8) return POLAR_EINVAL;
  polar_frozen_set *fsm = const_cast<polar_frozen_set *>(fs);
  // The options are read once: sizing, class table and launches all use
  // this snapshot, whatever other threads set meanwhile.
  const polar::ScratchOpts o = polar::scratch_opts(fs, nframes, (int)fkind, (int)prec);
  const size_t mask_bytes = ((fs->mask.size() * sizeof(uint32_t)) + 255) & ~size_t(255);
  const size_t level_bytes = polar::scratch_level_bytes(fs, nframes, (int)prec, o.t);
  // node-class table of the subtrees, when the shortcuts use one
  std::shared_ptr<std::vector<uint32_t>> ctab;
  if (o.shortcuts && o.t >= 5) ctab = polar::class_table_host(fsm, o.t);
  const size_t class_bytes =
      ctab ? ((ctab->size() * sizeof(uint32_t)) + 255) & ~size_t(255) : 0;
  const size_t need = mask_bytes + class_bytes + level_bytes;
  if (need > POLAR_STATIC_SCRATCH_BYTES) {
    static thread_local char msg[160];
    snprintf(msg, sizeof msg,
             "noalloc decode needs %zu bytes of scratch; the static array holds %u bytes",
             need, (unsigned)POLAR_STATIC_SCRATCH_BYTES);
    polar::set_last_error(msg);
    return POLAR_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    polar::set_last_error(cudaGetErrorString(e));
    return POLAR_ECUDA;
  }
  unsigned char *base = nullptr;
  int rc = static_scratch(dev, &base);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The mask and the class table are rewritten on every call: the array
  // keeps whatever the last call on this device left there.  The level
  // scratch needs no clearing: every level is written before it is read.
  e = cudaMemcpyAsync(base, fs->mask.data(), fs->mask.size() * sizeof(uint32_t),
                      cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && ctab)
    e = cudaMemcpyAsync(base + mask_bytes, ctab->data(), ctab->size() * sizeof(uint32_t),
                        cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    polar::set_last_error(cudaGetErrorString(e));
    return POLAR_ECUDA;
  }
  const size_t head = mask_bytes + class_bytes;
  return polar::decode_with_scratch(
      fs, nframes, llr_dev, frozen_vals_dev, xhat_dev, uhat_dev, (int)fkind, (int)prec, o,
      reinterpret_cast<uint32_t *>(base),
      ctab ? reinterpret_cast<uint32_t *>(base + mask_bytes) : nullptr, base + head,
      POLAR_STATIC_SCRATCH_BYTES - head, s);
}
