// Persistent SC decoder: one launch decodes a queue of frames of any lengths
// and codes.  Each CTA claims the next frame from a device counter and runs
// the whole SC recursion of that frame (Sec. 4) by itself:
//
//   * levels above the subtree size 2^t live in the CTA's own slice of a
//     global scratch buffer, stored as float, half or int8 like the launched
//     schedule's levels; their f and g steps stream through it (cta_step:
//     16-byte chunks staged by cp.async, the partial sums of g read from
//     x_hat, where the left child's beta sits in place);
//   * every subtree of 2^t leaves is decoded in shared memory and registers
//     by the same code as the per-subtree launches (subtree_body);
//   * nodes whose leaves are all frozen (rate 0) take beta = fv F^{(x)k}
//     directly, and f / g steps whose result only feeds a rate-0 child are
//     skipped, as in the launched schedule;
//   * with int8 storage the CTA first forms the frame's scale by the same
//     reduction, in the same order, as the launched schedule's scale kernel.
//
// Frames are independent, so CTAs never wait on one another; the queue keeps
// every SM busy while frames of different lengths finish at different times
// (the host orders the queue longest first).  Results are bit-identical to
// the launched schedule at the same subtree size: every f and g is the same
// operation on the same operands with the same storage rounding.
#pragma once

#include <algorithm>

#include "cta_step.cuh"
#include "subtree_impl.cuh"

namespace polar {

namespace {

constexpr uint32_t PT = kPersistThreads;

static_assert(PT == 128, "the subtree decoder runs with four warps");

__device__ __forceinline__ int upper_class(const PFrame &fr, int k, uint64_t o) {
  const int n = (int)fr.log2n;
  const uint64_t i = (uint64_t(1) << (n - k)) + (o >> k);
  if ((fr.ucls[i >> 5] >> (i & 31)) & 1u) return NODE_RATE0;
  const uint32_t uw = upper_class_words(n, (int)fr.t);
  if ((fr.ucls[uw + (i >> 5)] >> (i & 31)) & 1u) return NODE_RATE1;
  return NODE_MIXED;
}

// Rate-0 node of 2^k leaves (k >= 5) at leaf o: u_hat = fv, beta = fv F^{(x)k}.
__device__ void upper_rate0(const PFrame &fr, int k, uint64_t o) {
  const uint64_t w0 = o >> 5, nw = uint64_t(1) << (k - 5);
  for (uint64_t i = threadIdx.x; i < nw; i += PT) {
    const uint32_t v = fr.fv[w0 + i];
    if (fr.uhat) fr.uhat[w0 + i] = v;
    fr.xhat[w0 + i] = encode_word(v, 5);
  }
  for (uint64_t hw = 1; hw < nw; hw <<= 1) {
    __syncthreads();
    for (uint64_t j = threadIdx.x; j < nw / 2; j += PT) {
      const uint64_t a = (j / hw) * 2 * hw + (j % hw);
      fr.xhat[w0 + a] ^= fr.xhat[w0 + a + hw];
    }
  }
  __syncthreads();
}

// Per-frame scale of int8 storage: 2^rint(log2(target / mean |L|)) with the
// mean in double over the channel LLRs, clamped to 2^+-100, 1 if all L = 0 --
// 256 strided partial sums and a halving tree, the launched schedule's scale
// kernel's order (part: 256 doubles of shared memory).
__device__ float frame_int8_scale(const float *llr, uint64_t n, double target, double *part) {
  for (uint32_t v = threadIdx.x; v < 256; v += PT) {
    double acc = 0.0;
    for (uint64_t i = v; i < n; i += 256) acc += fabs((double)llr[i]);
    part[v] = acc;
  }
  __syncthreads();
  for (uint32_t w = 128; w > 0; w >>= 1) {
    for (uint32_t v = threadIdx.x; v < w; v += PT) part[v] += part[v + w];
    __syncthreads();
  }
  const double tot = part[0];
  __syncthreads();
  float sc = 1.0f;
  if (tot > 0.0) {
    double e = rint(log2(target / (tot / (double)n)));
    e = fmin(fmax(e, -100.0), 100.0);
    sc = (float)ldexp(1.0, (int)e);
  }
  return sc;
}

// s_scale: a float of shared memory that holds the frame's int8 scale for the
// subtree decoder.
template <typename S, int FK, bool UH>
__device__ void decode_frame(const PFrame &fr, S *lv, unsigned char *smraw, size_t smem,
                             double int8_target, float *s_scale) {
  float4 *stage = reinterpret_cast<float4 *>(smraw);
  const int n = (int)fr.log2n, t = (int)fr.t;
  const int stg_top = step_stages<float, S>(smem, PT), stg = step_stages<S, S>(smem, PT);
  constexpr bool I8 = sizeof(S) == 1;
  float sc = 1.0f;
  if (I8) {
    sc = frame_int8_scale(fr.llr, uint64_t(1) << n, int8_target,
                          reinterpret_cast<double *>(smraw));
    if (threadIdx.x == 0) *s_scale = sc;
    __syncthreads();
  }
  StParams p;
  p.in_stride = 0;
  p.in_o = 0;
  p.scale = I8 ? s_scale : nullptr;
  p.mask = fr.mask;
  p.fv = fr.fv;
  p.xhat = fr.xhat;
  p.uhat = fr.uhat;
  p.w_stride = 0;
  p.t = t;
  p.r = 0;
  p.pre = 0;
  // level k (t <= k < n) at lv + 2^k - 2^t; level n is the channel LLRs
  auto level = [&](int k) -> S * {
    return lv + ((uint64_t(1) << k) - (uint64_t(1) << t));
  };
  // one step from level k (the channel LLRs when k = n) to level k - 1
  auto step = [&](bool g, int k, const uint32_t *beta) {
    const uint32_t h = 1u << (k - 1);
    if (k == n) {
      if (g) cta_step_n<PT, float, S, FK, true>(stg_top, fr.llr, level(k - 1), h, beta, sc, stage);
      else cta_step_n<PT, float, S, FK, false>(stg_top, fr.llr, level(k - 1), h, beta, sc, stage);
    } else {
      if (g) cta_step_n<PT, S, S, FK, true>(stg, level(k), level(k - 1), h, beta, sc, stage);
      else cta_step_n<PT, S, S, FK, false>(stg, level(k), level(k - 1), h, beta, sc, stage);
    }
  };
  int k = n;
  uint64_t o = 0;
  for (;;) {
    for (;;) {                                    // descend to a unit
      if (n > t && upper_class(fr, k, o) == NODE_RATE0) {
        upper_rate0(fr, k, o);
        break;
      }
      if (k == t) {                               // n == t: the code is one subtree
        // float levels go through the float branch of subtree_body (cp.async
        // from the row); stored half / int8 levels through its stored-value
        // branch, the channel LLRs (n == t) through its scaled-LLR branch
        const bool as_llr = sizeof(S) == 4 || n == t;
        p.in = n == t ? static_cast<const void *>(fr.llr) : static_cast<const void *>(level(t));
        p.o = o;
        p.cls = fr.cls ? fr.cls + (o >> t) * 2 * class_words(t) : nullptr;
        subtree_body<4, S, FK, true, UH>(p, as_llr, 0, smraw);
        break;
      }
      if (upper_class(fr, k - 1, o) != NODE_RATE0) step(false, k, nullptr);
      --k;
    }
    int r = 0;                                    // ascend through right children
    while (k + r < n && ((o >> (k + r)) & 1u)) ++r;
    if (r > 0) {
      cascade_device(fr.xhat, k, o, r);
      k += r;
      o = (o >> k) << k;
    }
    if (k == n) break;
    if (upper_class(fr, k, o + (uint64_t(1) << k)) != NODE_RATE0)
      step(true, k + 1, fr.xhat + (o >> 5));
    o += uint64_t(1) << k;
  }
}

// Three CTAs per SM (168 registers, a few spills): the frame loop around the
// inlined subtree decoder would otherwise take ~240 registers and leave room
// for two CTAs per SM.
constexpr int kPersistMinBlocks = 3;

template <typename S, int FK, bool UH>
__global__ void __launch_bounds__(PT, kPersistMinBlocks)
    k_persist(const PFrame *frames, uint32_t count, uint32_t *head, float *scratch,
              uint64_t cta_floats, double int8_target, uint32_t smem) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ uint32_t s_idx;
  __shared__ float s_scale;
  S *lv = reinterpret_cast<S *>(scratch + (uint64_t)blockIdx.x * cta_floats);
  for (;;) {                                      // ends: *head only grows
    if (threadIdx.x == 0) s_idx = atomicAdd(head, 1u);
    __syncthreads();
    const uint32_t idx = s_idx;
    __syncthreads();
    if (idx >= count) break;
    const PFrame fr = frames[idx];
    decode_frame<S, FK, UH>(fr, lv, smraw, smem, int8_target, &s_scale);
  }
}

// ---------------------------------------------------------------- serving
// The same frame decoder fed by a ring that the host keeps filling while the
// launch runs (host-mapped memory): thread 0 of a CTA claims frame `head`
// once the host has published it (tail > head), decodes it with the CTA and
// then publishes done[i % R] = i + 1.  A CTA that finds no frame for idle_ns
// nanoseconds, or sees `stop`, leaves; the host relaunches when frames are
// published after the launch ended.
__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(uint32_t *p, uint32_t v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr uint32_t kNoFrame = 0xFFFFFFFFu;

// Thread 0: the next published frame, or kNoFrame (idle, stop, or the
// iteration cap, which bounds the wait independently of the timer).
__device__ uint32_t claim_frame(const ServeArgs &a) {
  const uint64_t t0 = global_ns();
  uint32_t nap = 128;
  for (uint32_t it = 0; it < (1u << 22); ++it) {
    const uint32_t tl = ld_acquire_sys(a.tail);
    uint32_t h = *reinterpret_cast<volatile uint32_t *>(a.head);
    while (h < tl) {                              // each failed CAS means h grew
      const uint32_t prev = atomicCAS(a.head, h, h + 1);
      if (prev == h) return h;
      h = prev;
    }
    if (ld_acquire_sys(a.stop)) return kNoFrame;
    if (global_ns() - t0 > a.idle_ns) return kNoFrame;
    __nanosleep(nap);
    nap = nap < 8192 ? 2 * nap : nap;
  }
  return kNoFrame;
}

template <typename S, int FK>
__global__ void __launch_bounds__(PT, kPersistMinBlocks) k_serve(ServeArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ uint32_t s_idx;
  __shared__ __align__(16) PFrame s_fr;
  __shared__ float s_scale;
  S *lv = reinterpret_cast<S *>(a.scratch + (uint64_t)blockIdx.x * a.cta_floats);
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t idx = claim_frame(a);
      if (idx != kNoFrame) {                      // the ring entry, read past any cache
        const volatile uint64_t *src =
            reinterpret_cast<const volatile uint64_t *>(a.ring + (idx & a.rmask));
        uint64_t *dst = reinterpret_cast<uint64_t *>(&s_fr);
        for (int w = 0; w < (int)(sizeof(PFrame) / 8); ++w) dst[w] = src[w];
      }
      s_idx = idx;
    }
    __syncthreads();
    const uint32_t idx = s_idx;
    const PFrame fr = s_fr;
    __syncthreads();
    if (idx == kNoFrame) break;
    decode_frame<S, FK, true>(fr, lv, smraw, a.smem, a.int8_target, &s_scale);
    __syncthreads();                              // every x_hat / u_hat word written
    if (threadIdx.x == 0) {
      __threadfence_system();
      st_release_sys(a.done + (idx & a.rmask), idx + 1);
    }
  }
}

// The subtree's levels and bit vectors, and at least one stage of step slots
// (the widest: float channel LLRs into int8 values).
inline size_t persist_smem(int t) {
  const size_t sub = bit_words(t) * sizeof(uint32_t) + 2 * (size_t(1) << t) * sizeof(float);
  const size_t slot = (size_t)StepShape<float, int8_t>::SL * 16 * PT;
  return std::max(sub, slot);
}

// The persistent CTAs leave only when the queue runs dry, so every CTA of
// the grid must be resident at once: ask for the largest shared-memory
// carveout (the occupancy query assumes it) and the dynamic size.
template <typename K>
cudaError_t prepare_persistent(K kern, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess && smem > 48 * 1024)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return e;
}

template <typename K>
int resident_per_sm(K kern, size_t smem) {
  if (prepare_persistent(kern, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, PT, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

template <typename S, int FK, bool UH>
cudaError_t launch_pk(const PFrame *frames, uint32_t count, uint32_t *head, float *scratch,
                      uint64_t cta_floats, int t, int grid, double int8_target,
                      cudaStream_t s) {
  const size_t smem = persist_smem(t);
  auto kern = k_persist<S, FK, UH>;
  cudaError_t e = prepare_persistent(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, PT, smem, s>>>(frames, count, head, scratch, cta_floats, int8_target,
                              (uint32_t)smem);
  return counted(cudaGetLastError(), 1);
}

// Per storage type: the persistent launch, its residency, the serving launch
// and its residency.
template <typename S>
cudaError_t launch_persistent_s(int fkind, bool uhat, const PFrame *frames, uint32_t count,
                                uint32_t *head, float *scratch, uint64_t cta_floats, int t,
                                int grid, double int8_target, cudaStream_t s) {
  if (fkind == 0)
    return uhat ? launch_pk<S, 0, true>(frames, count, head, scratch, cta_floats, t, grid,
                                        int8_target, s)
                : launch_pk<S, 0, false>(frames, count, head, scratch, cta_floats, t, grid,
                                         int8_target, s);
  return uhat ? launch_pk<S, 1, true>(frames, count, head, scratch, cta_floats, t, grid,
                                      int8_target, s)
              : launch_pk<S, 1, false>(frames, count, head, scratch, cta_floats, t, grid,
                                       int8_target, s);
}

template <typename S>
int persistent_ctas_per_sm_s(int fkind, bool uhat, int t) {
  const size_t smem = persist_smem(t);
  if (fkind == 0)
    return uhat ? resident_per_sm(k_persist<S, 0, true>, smem)
                : resident_per_sm(k_persist<S, 0, false>, smem);
  return uhat ? resident_per_sm(k_persist<S, 1, true>, smem)
              : resident_per_sm(k_persist<S, 1, false>, smem);
}

template <typename S>
cudaError_t launch_serve_s(int fkind, ServeArgs a, int t, int grid, cudaStream_t s) {
  const size_t smem = persist_smem(t);
  a.smem = (uint32_t)smem;
  auto kern = fkind == 0 ? k_serve<S, 0> : k_serve<S, 1>;
  cudaError_t e = prepare_persistent(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, PT, smem, s>>>(a);
  return counted(cudaGetLastError(), 1);
}

template <typename S>
int serve_ctas_per_sm_s(int fkind, int t) {
  const size_t smem = persist_smem(t);
  return fkind == 0 ? resident_per_sm(k_serve<S, 0>, smem) : resident_per_sm(k_serve<S, 1>, smem);
}

}  // namespace

}  // namespace polar
