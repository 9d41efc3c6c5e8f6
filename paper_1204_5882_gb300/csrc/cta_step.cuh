// One CTA's f or g step of the SC recursion over one frame (Sec. 4), level
// k -> k - 1 with h = 2^(k-1) outputs, used by the node units of the launched
// schedule and by the persistent decoder:
//   f (G = false): c[j] = f(a[j], a[j + h]);
//   g (G = true):  c[j] = g(a[j], a[j + h], bit j of beta), beta = the left
//                  sibling's partial sums (word-aligned).
// Inputs are stored values of type S, or (Tin = float, top level) the float
// channel LLRs, which are scaled (int8) and rounded to S on load; outputs are
// rounded / saturated to S on store -- the streamed kernels' operations, so
// every value is bit-identical to theirs.  A thread handles units of one
// 16-byte output chunk (16 / sizeof(S) values); the unit's input chunks of a
// and a + h and (g) its partial-sum word are staged in a slot of shared
// memory by cp.async, STG slots in flight per thread, and the output goes to
// global memory with st.global.cg (L2; the next step reads it with cp.async).
#pragma once

#include "device_common.cuh"
#include "subtree_impl.cuh"   // g_bit

namespace polar {

namespace {

template <typename Tin, typename S>
struct StepShape {
  static constexpr uint32_t PER = 16 / sizeof(S);              // outputs per unit
  static constexpr uint32_t IC = PER * sizeof(Tin) / 16;       // input chunks per operand
  static constexpr uint32_t SL = 2 * IC + 1;                   // 16-byte words per slot
};

// Largest power-of-two stage count (<= 16) whose slots fit in smem_bytes.
template <typename Tin, typename S>
__host__ __device__ inline int step_stages(size_t smem_bytes, uint32_t nthreads) {
  const size_t per = (size_t)StepShape<Tin, S>::SL * 16 * nthreads;
  int s = 1;
  while (s < 16 && (size_t)(2 * s) * per <= smem_bytes) s *= 2;
  return s;
}

template <typename Tin, typename S>
__device__ __forceinline__ float step_load(const Tin *p, float sc) {
  if constexpr (sizeof(Tin) == 4 && sizeof(S) != 4) return rnd<S>(*p * sc);
  return Store<Tin>::ld(p);
}

template <int STG, uint32_t NTH, typename Tin, typename S, int FK, bool G>
__device__ void cta_step(const Tin *__restrict__ a, S *__restrict__ c, uint32_t h,
                         const uint32_t *__restrict__ beta, float sc, float4 *stage) {
  using SH = StepShape<Tin, S>;
  constexpr uint32_t PER = SH::PER, IC = SH::IC, SL = SH::SL;
  const float4 *x4 = reinterpret_cast<const float4 *>(a);
  const float4 *y4 = reinterpret_cast<const float4 *>(a + h);
  uint4 *c4 = reinterpret_cast<uint4 *>(c);
  const uint32_t hc = h / PER, tid = threadIdx.x;
  float4 *mine = stage + SL * tid;
  const uint32_t iters = (hc + NTH - 1) / NTH;
  auto issue = [&](uint32_t i, float4 *sl) {
#pragma unroll
    for (uint32_t q = 0; q < IC; ++q) {
      cp16(sl + q, x4 + i * IC + q);
      cp16(sl + IC + q, y4 + i * IC + q);
    }
    if (G) cp4(sl + 2 * IC, beta + ((PER * i) >> 5));
  };
#pragma unroll
  for (uint32_t it = 0; it < (uint32_t)STG; ++it) {
    const uint32_t i = it * NTH + tid;
    if (i < hc) issue(i, mine + it * SL * NTH);
    cp_commit();
  }
  for (uint32_t it = 0; it < iters; ++it) {
    cp_wait<STG - 1>();                           // this thread's group `it` has landed
    const uint32_t i = it * NTH + tid;
    float4 *sl = mine + (it % STG) * SL * NTH;
    if (i < hc) {
      const Tin *xs = reinterpret_cast<const Tin *>(sl);
      const Tin *ys = reinterpret_cast<const Tin *>(sl + IC);
      uint4 ov;
      S *os = reinterpret_cast<S *>(&ov);
      const uint32_t w = G ? *reinterpret_cast<const uint32_t *>(sl + 2 * IC) : 0u;
      const int j0 = (int)((PER * i) & 31u);
#pragma unroll
      for (uint32_t q = 0; q < PER; ++q) {
        const float xa = step_load<Tin, S>(xs + q, sc), yb = step_load<Tin, S>(ys + q, sc);
        const float v = G ? g_bit(xa, yb, w, j0 + (int)q) : f_st<S, FK>(xa, yb, sc);
        Store<S>::st(os + q, v);
      }
      __stcg(c4 + i, ov);
    }
    const uint32_t in = (it + STG) * NTH + tid;   // refill the slot just read
    if (in < hc) issue(in, sl);
    cp_commit();
  }
  cp_wait<0>();
  __syncthreads();
}

template <uint32_t NTH, typename Tin, typename S, int FK, bool G>
__device__ void cta_step_n(int stg, const Tin *a, S *c, uint32_t h, const uint32_t *beta,
                           float sc, float4 *stage) {
  switch (stg) {
    case 16: cta_step<16, NTH, Tin, S, FK, G>(a, c, h, beta, sc, stage); break;
    case 8: cta_step<8, NTH, Tin, S, FK, G>(a, c, h, beta, sc, stage); break;
    case 4: cta_step<4, NTH, Tin, S, FK, G>(a, c, h, beta, sc, stage); break;
    case 2: cta_step<2, NTH, Tin, S, FK, G>(a, c, h, beta, sc, stage); break;
    default: cta_step<1, NTH, Tin, S, FK, G>(a, c, h, beta, sc, stage); break;
  }
}

}  // namespace

}  // namespace polar
