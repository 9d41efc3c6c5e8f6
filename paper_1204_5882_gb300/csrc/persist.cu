// Persistent SC decoder: one launch decodes a queue of frames of any lengths
// and codes.  Each CTA claims the next frame from a device counter and runs
// the whole SC recursion of that frame (Sec. 4) by itself:
//
//   * levels above the subtree size 2^t live in the CTA's own slice of a
//     global scratch buffer; their f and g steps stream through it with
//     16-byte loads, the partial sums of g read from x_hat, where the left
//     child's beta sits in place;
//   * every subtree of 2^t leaves is decoded in shared memory and registers
//     by the same code as the per-subtree launches (subtree_body);
//   * nodes whose leaves are all frozen (rate 0) take beta = fv F^{(x)k}
//     directly, and f / g steps whose result only feeds a rate-0 child are
//     skipped, as in the launched schedule.
//
// Frames are independent, so CTAs never wait on one another; the queue keeps
// every SM busy while frames of different lengths finish at different times
// (the host orders the queue longest first).  Results are bit-identical to
// the launched schedule: every f and g is the same float32 operation on the
// same operands.
#include <algorithm>

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

// One upper step, level k -> k-1 over h = 2^(k-1) outputs (h >= 32):
//   f (G = false): c[i] = f(a[i], a[i + h]);
//   g (G = true):  c[i] = g(a[i], a[i + h], bit i of beta), beta = the left
//                  child's partial sums, word aligned.
// S stages of slots per thread stay in flight: a slot holds the float4 of a,
// the float4 of a + h and (g) the partial-sum word, 48 bytes apart (an odd
// multiple of 16 bytes, so a warp's 16-byte reads hit distinct banks).
template <int S, int FK, bool G>
__device__ void upper_step(const float *__restrict__ a, float *__restrict__ c, uint32_t h,
                           const uint32_t *__restrict__ beta, float4 *stage) {
  const float4 *x4 = reinterpret_cast<const float4 *>(a);
  const float4 *y4 = reinterpret_cast<const float4 *>(a + h);
  float4 *c4 = reinterpret_cast<float4 *>(c);
  const uint32_t h4 = h >> 2, tid = threadIdx.x;
  float4 *mine = stage + 3 * tid;
  const uint32_t iters = (h4 + PT - 1) / PT;
#pragma unroll
  for (uint32_t it = 0; it < (uint32_t)S; ++it) {
    const uint32_t i = it * PT + tid;
    float4 *sl = mine + it * 3 * PT;
    if (i < h4) {
      cp16(sl, x4 + i);
      cp16(sl + 1, y4 + i);
      if (G) cp4(sl + 2, beta + (i >> 3));
    }
    cp_commit();
  }
  for (uint32_t it = 0; it < iters; ++it) {
    cp_wait<S - 1>();                             // this thread's group `it` has landed
    const uint32_t i = it * PT + tid;
    float4 *sl = mine + (it % S) * 3 * PT;
    if (i < h4) {
      const float4 x = sl[0], y = sl[1];
      float4 r;
      if (G) {
        const uint32_t w = *reinterpret_cast<const uint32_t *>(sl + 2);
        const int j = (int)((i & 7) << 2);
        r = make_float4(g_bit(x.x, y.x, w, j), g_bit(x.y, y.y, w, j + 1),
                        g_bit(x.z, y.z, w, j + 2), g_bit(x.w, y.w, w, j + 3));
      } else {
        r = make_float4(f_op<FK>(x.x, y.x), f_op<FK>(x.y, y.y), f_op<FK>(x.z, y.z),
                        f_op<FK>(x.w, y.w));
      }
      __stcg(c4 + i, r);
    }
    const uint32_t in = (it + S) * PT + tid;      // refill the slot just read
    if (in < h4) {
      cp16(sl, x4 + in);
      cp16(sl + 1, y4 + in);
      if (G) cp4(sl + 2, beta + (in >> 3));
    }
    cp_commit();
  }
  cp_wait<0>();
  __syncthreads();
}

// Stages that fit in the CTA's dynamic shared memory (48-byte slots).
__host__ __device__ inline int upper_stages(size_t smem_bytes) {
  const size_t per = 48 * PT;
  int s = 1;
  while (s < 16 && (size_t)(2 * s) * per <= smem_bytes) s *= 2;
  return s;
}

template <int FK, bool G>
__device__ void upper(int S, const float *a, float *c, uint32_t h, const uint32_t *beta,
                      float4 *stage) {
  switch (S) {
    case 16: upper_step<16, FK, G>(a, c, h, beta, stage); break;
    case 8: upper_step<8, FK, G>(a, c, h, beta, stage); break;
    case 4: upper_step<4, FK, G>(a, c, h, beta, stage); break;
    case 2: upper_step<2, FK, G>(a, c, h, beta, stage); break;
    default: upper_step<1, FK, G>(a, c, h, beta, stage); break;
  }
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

template <int FK, bool UH>
__device__ void decode_frame(const PFrame &fr, float *lv, unsigned char *smraw, int S) {
  float4 *stage = reinterpret_cast<float4 *>(smraw);
  const int n = (int)fr.log2n, t = (int)fr.t;
  StParams p;
  p.in_stride = 0;
  p.in_o = 0;
  p.scale = nullptr;
  p.mask = fr.mask;
  p.fv = fr.fv;
  p.xhat = fr.xhat;
  p.uhat = fr.uhat;
  p.w_stride = 0;
  p.t = t;
  p.r = 0;
  p.pre = 0;
  // level k (t <= k < n) at lv + 2^k - 2^t; level n is the channel LLRs
  auto level = [&](int k) -> float * {
    return lv + ((uint64_t(1) << k) - (uint64_t(1) << t));
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
        p.in = n == t ? fr.llr : level(t);
        p.o = o;
        p.cls = fr.cls ? fr.cls + (o >> t) * 2 * class_words(t) : nullptr;
        subtree_body<4, float, FK, true, UH>(p, true, 0, smraw);
        break;
      }
      if (upper_class(fr, k - 1, o) != NODE_RATE0)
        upper<FK, false>(S, k == n ? fr.llr : level(k), level(k - 1), 1u << (k - 1), nullptr,
                         stage);
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
      upper<FK, true>(S, k + 1 == n ? fr.llr : level(k + 1), level(k), 1u << k,
                      fr.xhat + (o >> 5), stage);
    o += uint64_t(1) << k;
  }
}

// Three CTAs per SM (168 registers, a few spills): the frame loop around the
// inlined subtree decoder would otherwise take ~240 registers and leave room
// for two CTAs per SM.
constexpr int kPersistMinBlocks = 3;

template <int FK, bool UH>
__global__ void __launch_bounds__(PT, kPersistMinBlocks) k_persist(const PFrame *frames, uint32_t count,
                                                uint32_t *head, float *scratch,
                                                uint64_t cta_floats, int S) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ uint32_t s_idx;
  float *lv = scratch + (uint64_t)blockIdx.x * cta_floats;
  for (;;) {                                      // ends: *head only grows
    if (threadIdx.x == 0) s_idx = atomicAdd(head, 1u);
    __syncthreads();
    const uint32_t idx = s_idx;
    __syncthreads();
    if (idx >= count) break;
    const PFrame fr = frames[idx];
    decode_frame<FK, UH>(fr, lv, smraw, S);
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

template <int FK>
__global__ void __launch_bounds__(PT, kPersistMinBlocks) k_serve(ServeArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ uint32_t s_idx;
  __shared__ __align__(16) PFrame s_fr;
  float *lv = a.scratch + (uint64_t)blockIdx.x * a.cta_floats;
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
    decode_frame<FK, true>(fr, lv, smraw, a.S);
    __syncthreads();                              // every x_hat / u_hat word written
    if (threadIdx.x == 0) {
      __threadfence_system();
      st_release_sys(a.done + (idx & a.rmask), idx + 1);
    }
  }
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

template <int FK, bool UH>
cudaError_t launch_pk(const PFrame *frames, uint32_t count, uint32_t *head, float *scratch,
                      uint64_t cta_floats, int t, int grid, cudaStream_t s) {
  const size_t smem = persistent_smem_bytes(t);
  auto kern = k_persist<FK, UH>;
  cudaError_t e = prepare_persistent(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, PT, smem, s>>>(frames, count, head, scratch, cta_floats, upper_stages(smem));
  return counted(cudaGetLastError(), 1);
}

template <int FK, bool UH>
int occupancy(int t) {
  const size_t smem = persistent_smem_bytes(t);
  auto kern = k_persist<FK, UH>;
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

template <int FK>
int serve_occupancy(int t) {
  const size_t smem = persistent_smem_bytes(t);
  auto kern = k_serve<FK>;
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

}  // namespace

int serve_ctas_per_sm(int fkind, int t) {
  return fkind == 0 ? serve_occupancy<0>(t) : serve_occupancy<1>(t);
}

cudaError_t launch_serve(int fkind, ServeArgs a, int t, int grid, cudaStream_t s) {
  const size_t smem = persistent_smem_bytes(t);
  a.S = upper_stages(smem);
  auto kern = fkind == 0 ? k_serve<0> : k_serve<1>;
  cudaError_t e = prepare_persistent(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, PT, smem, s>>>(a);
  return counted(cudaGetLastError(), 1);
}

// The subtree's levels and bit vectors, and at least one stage of upper-step
// slots (48 bytes per thread).
size_t persistent_smem_bytes(int t) {
  const size_t sub = bit_words(t) * sizeof(uint32_t) + 2 * (size_t(1) << t) * sizeof(float);
  return std::max(sub, size_t(48) * PT);
}

int persistent_ctas_per_sm(int fkind, bool uhat, int t) {
  if (fkind == 0) return uhat ? occupancy<0, true>(t) : occupancy<0, false>(t);
  return uhat ? occupancy<1, true>(t) : occupancy<1, false>(t);
}

cudaError_t launch_persistent(int fkind, bool uhat, const PFrame *frames, uint32_t count,
                              uint32_t *head, float *scratch, uint64_t cta_floats, int t,
                              int grid, cudaStream_t s) {
  if (fkind == 0)
    return uhat ? launch_pk<0, true>(frames, count, head, scratch, cta_floats, t, grid, s)
                : launch_pk<0, false>(frames, count, head, scratch, cta_floats, t, grid, s);
  return uhat ? launch_pk<1, true>(frames, count, head, scratch, cta_floats, t, grid, s)
              : launch_pk<1, false>(frames, count, head, scratch, cta_floats, t, grid, s);
}

}  // namespace polar
