// Node decoder of the launched schedule: one CTA per frame decodes a node of
// 2^s leaves (s > t) of the SC recursion (Sec. 4) by itself, instead of the
// 2^(s-t) subtree launches and the streamed f / g launches between them.
//
//   * the steps of the levels s .. t + 1 (f for a left child, g with the left
//     sibling's partial sums for a right child) run inside the CTA over its
//     frame's rows of the batch workspace (cta_step: 16-byte chunks of the
//     stored float, half or int8 values staged into shared memory by
//     cp.async, written back with st.global.cg);
//   * every subtree of 2^t leaves is decoded by subtree_body, from the
//     workspace's level t;
//   * rate-0 nodes above t take beta = fv F^{(x)k} directly, and steps whose
//     result only feeds a rate-0 child are skipped (the upper class table);
//   * partial sums combine in place in x_hat as the recursion ascends, and
//     the node's own combines above level s follow at the end.
//
// Each step is the streamed kernels' operation on the same operands with the
// same storage rounding (and int8 scale), so the decisions are bit-identical
// to the schedule that streams those levels with whole-GPU launches.  The
// node's levels are small (2^s stored values per frame and level), so they
// stay in L2 between the steps; what the node saves is the launch and
// dependency overhead of many short launches.
#pragma once

#include "cta_step.cuh"
#include "subtree_impl.cuh"

namespace polar {

namespace {

constexpr uint32_t NT = 32 * kScWarps;   // threads of a node CTA (the subtree decoder's warps)

struct NodeParams {
  const void *lv;           // level t of the workspace; level k at F (2^k - 2^t) values
  int F;                    // frames of the batch
  const uint32_t *mask;     // frozen mask (whole code)
  const uint32_t *cls;      // subtree class table (whole code) or null
  const uint32_t *ucls;     // upper class table (levels t..n)
  const float *scale;       // int8 per-frame scales or null
  const uint32_t *fv;
  uint32_t *xhat;
  uint32_t *uhat;
  size_t w_stride;
  uint64_t o;               // first leaf of the node
  int s, t, n, r;           // node level, subtree level, code level, combines after the node
  int stages;               // cp.async stages per thread in the steps
};

template <typename S>
__device__ __forceinline__ S *node_level(const NodeParams &p, int k, size_t fr) {
  return const_cast<S *>(reinterpret_cast<const S *>(p.lv)) +
         (size_t)p.F * ((size_t(1) << k) - (size_t(1) << p.t)) + fr * (size_t(1) << k);
}

__device__ __forceinline__ int node_class(const NodeParams &p, int k, uint64_t o) {
  const uint64_t i = (uint64_t(1) << (p.n - k)) + (o >> k);
  if ((p.ucls[i >> 5] >> (i & 31)) & 1u) return NODE_RATE0;
  const uint32_t uw = upper_class_words(p.n, p.t);
  if ((p.ucls[uw + (i >> 5)] >> (i & 31)) & 1u) return NODE_RATE1;
  return NODE_MIXED;
}

// Rate-0 node of 2^k leaves (k >= 5) at leaf o of one frame's rows.
__device__ void node_rate0(uint32_t *x, uint32_t *u, const uint32_t *fv, int k, uint64_t o) {
  const uint64_t w0 = o >> 5, nw = uint64_t(1) << (k - 5);
  for (uint64_t i = threadIdx.x; i < nw; i += NT) {
    const uint32_t v = fv[w0 + i];
    if (u) u[w0 + i] = v;
    x[w0 + i] = encode_word(v, 5);
  }
  for (uint64_t hw = 1; hw < nw; hw <<= 1) {
    __syncthreads();
    for (uint64_t j = threadIdx.x; j < nw / 2; j += NT) {
      const uint64_t a = (j / hw) * 2 * hw + (j % hw);
      x[w0 + a] ^= x[w0 + a + hw];
    }
  }
  __syncthreads();
}

template <typename S, int FK, bool UH>
__global__ void __launch_bounds__(NT, 1) k_node(NodeParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  pdl_enter();
  const size_t fr = blockIdx.x;
  float4 *stage = reinterpret_cast<float4 *>(smraw);
  const float sc = p.scale ? p.scale[fr] : 1.0f;
  uint32_t *xrow = p.xhat + fr * p.w_stride;
  uint32_t *urow = UH ? p.uhat + fr * p.w_stride : nullptr;
  const uint32_t *fvrow = p.fv + fr * p.w_stride;
  const int t = p.t;
  StParams sp;
  sp.in = node_level<S>(p, t, 0);                 // subtree_body adds fr * 2^t
  sp.in_stride = size_t(1) << t;
  sp.in_o = 0;
  sp.scale = p.scale;
  sp.mask = p.mask;
  sp.fv = p.fv;
  sp.xhat = p.xhat;
  sp.uhat = UH ? p.uhat : nullptr;
  sp.w_stride = p.w_stride;
  sp.t = t;
  sp.r = 0;
  sp.pre = 0;
  int k = p.s;
  uint64_t o = p.o;
  for (;;) {
    for (;;) {                                    // descend to a unit
      if (node_class(p, k, o) == NODE_RATE0) {      // k >= t >= 5
        node_rate0(xrow, urow, fvrow, k, o);
        break;
      }
      if (k == t) {
        sp.o = o;
        sp.cls = p.cls ? p.cls + (o >> t) * 2 * class_words(t) : nullptr;
        subtree_body<kScWarps, S, FK, true, UH>(sp, false, fr, smraw);
        break;
      }
      if (node_class(p, k - 1, o) != NODE_RATE0)
        cta_step_n<NT, S, S, FK, false>(p.stages, node_level<S>(p, k, fr),
                                        node_level<S>(p, k - 1, fr), 1u << (k - 1), nullptr, sc,
                                        stage);
      --k;
    }
    int r = 0;                                    // ascend through right children
    while (k + r < p.s && ((o >> (k + r)) & 1u)) ++r;
    if (r > 0) {
      cascade_device(xrow, k, o, r);
      k += r;
      o = (o >> k) << k;
    }
    if (k == p.s) break;
    if (node_class(p, k, o + (uint64_t(1) << k)) != NODE_RATE0)
      cta_step_n<NT, S, S, FK, true>(p.stages, node_level<S>(p, k + 1, fr),
                                     node_level<S>(p, k, fr), 1u << k, xrow + (o >> 5), sc,
                                     stage);
    o += uint64_t(1) << k;
  }
  if (p.r > 0) cascade_device(xrow, p.s, p.o, p.r);
}

// Shared memory of a node CTA: the subtree decoder's levels and bit vectors,
// and at least one stage of step slots (48 bytes per thread).
inline size_t node_smem_bytes(int t) {
  const size_t sub = bit_words(t) * sizeof(uint32_t) + 2 * (size_t(1) << t) * sizeof(float);
  return sub > size_t(48) * NT ? sub : size_t(48) * NT;
}

template <typename S, int FK, bool UH>
cudaError_t launch_node_t(const NodeArgs &a, cudaStream_t s) {
  const size_t smem = node_smem_bytes(a.t);
  auto kern = k_node<S, FK, UH>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  NodeParams p{a.lv,   a.nframes, a.mask,     a.cls, a.ucls, a.scale, a.fv,
               a.xhat, a.uhat,    a.w_stride, a.o,   a.s,    a.t,     a.n,
               a.r,    step_stages<S, S>(smem, NT)};
  return counted(launch_k(kern, a.nframes, NT, smem, s, p), 1);
}

template <typename S>
cudaError_t launch_node_s(const NodeArgs &a, cudaStream_t s) {
  const bool uh = a.uhat != nullptr;
  if (a.fkind == 0) return uh ? launch_node_t<S, 0, true>(a, s) : launch_node_t<S, 0, false>(a, s);
  return uh ? launch_node_t<S, 1, true>(a, s) : launch_node_t<S, 1, false>(a, s);
}

}  // namespace

}  // namespace polar
