// In-CTA subtree decoder: one warp runs the SC recursion (Sec. 4) over a
// node of 2^t leaves whose LLRs sit in shared memory, one CTA per frame.
//
// Shared memory: level k of the recursion (2^k LLRs) lives at L[2^k, 2^(k+1)),
// level t (the input) at L[2^t, 2^(t+1)); bit vectors beta (partial sums, in
// place), u_hat, the frozen mask and the frozen values take 2^t bits each.
//
// Node shortcuts (when enabled) return the exact SC result:
//   rate 0 (all frozen): beta = fv F^{(x)k} -- SC decides every leaf from fv
//                        and beta is the transform of the decisions;
//   rate 1 (all info):   beta = hard(L) when no input LLR is +-0 -- by
//                        induction f(a, b) is nonzero with the sign product
//                        (both f forms keep a nonzero magnitude for nonzero
//                        inputs) and g then reproduces sgn(b), so each leaf's
//                        decision is the hard decision of its input.  With
//                        zero inputs (frequent for the BSC, where g = c - c)
//                        nodes of up to 512 leaves take the bit recursion of
//                        rate1_word / Rate1Words, which gives SC's decisions
//                        exactly; larger nodes fall back to the recursion.
//
// With shortcuts on, node classes of the levels 5..t come from a table the
// host precomputes per subtree, and every mixed node of 32 leaves is decoded
// in registers by a fully unrolled recursion that all lanes run redundantly
// (min-sum: no shuffles, no shared-memory round trips below 32 leaves, and
// compile-time decoders for the few frozen patterns that dominate real codes;
// exact f: the node's top two levels are formed lane-parallel first, see
// dec32_lanes).  The plain variant (shortcuts off) runs every level
// lane-parallel through shared memory down to single leaves.
#pragma once

#include <type_traits>

#include "device_common.cuh"
#include "polar_internal.h"

namespace polar {

namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;

// Warps of a subtree / node CTA with shortcuts on: warp 0 runs the register
// tiles, all of them the shared-memory levels (8 measured 0.8-2 % faster
// than 4 on every float32 / FP16 workload: the level steps are latency-bound
// with one warp per scheduler).  Must be a power of two: the level loops
// step by four times the thread count and rely on it dividing the level.
constexpr int kScWarps = 8;
static_assert((kScWarps & (kScWarps - 1)) == 0, "kScWarps must be a power of two");

struct StParams {
  const void *in;
  size_t in_stride;
  uint64_t in_o;         // float input: element offset of the subtree in its row
  const uint32_t *cls;   // class table of this subtree (levels 5..t), or null
  const float *scale;    // per-frame int8 scale, or null
  const uint32_t *mask;
  const uint32_t *fv;
  uint32_t *xhat;
  uint32_t *uhat;
  size_t w_stride;
  uint64_t o;
  int t;
  int r;
  int pre;               // 0: in is level t; 1 / 2: in is the parent (level t + 1) and
                         // level t is its f / g, computed while loading
};

// g with the partial sum taken from bit j of a word: b + a or b - a (the
// latter as b + (-a), which IEEE addition makes identical).
__device__ __forceinline__ float g_bit(float a, float b, uint32_t word, int j) {
  return b + __uint_as_float(__float_as_uint(a) ^ ((word << (31 - j)) & 0x80000000u));
}

// Rate-1 test of a node held in registers: true (and the sign word in *b)
// when no input is +-0; min and OR trees keep the dependency depth at K.
template <int K>
__device__ __forceinline__ bool signs_if_nonzero(const float (&a)[1 << K], uint32_t *b) {
  constexpr int N = 1 << K;
  float m[N];
  uint32_t v[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    m[j] = fabsf(a[j]);
    v[j] = (__float_as_uint(a[j]) >> 31) << j;
  }
#pragma unroll
  for (int w = N / 2; w >= 1; w /= 2) {
#pragma unroll
    for (int j = 0; j < w; ++j) {
      m[j] = fminf(m[j], m[j + w]);
      v[j] |= v[j + w];
    }
  }
  *b = v[0];
  return m[0] > 0.0f;
}

// SC decisions (beta) of a rate-1 node of 2^K <= 32 leaves from two words of
// its inputs: H (bit j set iff input j < 0) and Z (bit j set iff input j is
// +-0).  Both f forms give +-0 exactly when an input is +-0 and otherwise a
// nonzero value with the sign product; g = b +- a is b when a = +-0, +-a when
// b = +-0, and a nonzero value with the sign of b when both are nonzero and
// the left decision is their hard-decision XOR.  By induction over the node:
//   - every nonzero input keeps its hard decision;
//   - with the halves (x, y) of the node, the left child sees
//     ZL = Zx | Zy and HL = Hx ^ Hy, the right child ZR = Zx & Zy and
//     HR = Hy where y != 0, Hx ^ betaL where y = 0;
//   - a zero leaf decides 0.
// So only the zero positions need the recursion, and a node without zero
// inputs returns H at once.  (Checked against recursive SC on rate-1 codes
// with dense +-0 inputs, both f forms, in the GPU parity tests.)
template <int K>
__device__ __forceinline__ uint32_t rate1_word(uint32_t H, uint32_t Z) {
  if (Z == 0u) return H;
  if constexpr (K == 0) {
    return 0u;
  } else {
    constexpr int Hh = 1 << (K - 1);
    constexpr uint32_t M = (1u << Hh) - 1u;
    const uint32_t Hx = H & M, Hy = (H >> Hh) & M, Zx = Z & M, Zy = (Z >> Hh) & M;
    const uint32_t ZL = Zx | Zy;
    const uint32_t bL = rate1_word<K - 1>((Hx ^ Hy) & ~ZL, ZL);
    const uint32_t ZR = Zx & Zy;
    const uint32_t bR = rate1_word<K - 1>(((Hy & ~Zy) | ((Hx ^ bL) & Zy)) & ~ZR, ZR);
    return (bL ^ bR) | (bR << Hh);
  }
}

// The same for a rate-1 node of 2^K leaves, 5 <= K <= 9, held as 2^(K-5)
// words (word r = leaves 32r .. 32r+31).
template <int K>
struct Rate1Words {
  static constexpr int R = 1 << (K - 5), Hf = R / 2;
  static __device__ __forceinline__ void run(const uint32_t (&H)[R], const uint32_t (&Z)[R],
                                             uint32_t (&b)[R]) {
    uint32_t any = 0u;
#pragma unroll
    for (int r = 0; r < R; ++r) any |= Z[r];
    if (any == 0u) {
#pragma unroll
      for (int r = 0; r < R; ++r) b[r] = H[r];
      return;
    }
    uint32_t h[Hf], z[Hf], bL[Hf], bR[Hf];
#pragma unroll
    for (int r = 0; r < Hf; ++r) {
      z[r] = Z[r] | Z[r + Hf];
      h[r] = (H[r] ^ H[r + Hf]) & ~z[r];
    }
    Rate1Words<K - 1>::run(h, z, bL);
#pragma unroll
    for (int r = 0; r < Hf; ++r) {
      z[r] = Z[r] & Z[r + Hf];
      h[r] = ((H[r + Hf] & ~Z[r + Hf]) | ((H[r] ^ bL[r]) & Z[r + Hf])) & ~z[r];
    }
    Rate1Words<K - 1>::run(h, z, bR);
#pragma unroll
    for (int r = 0; r < Hf; ++r) {
      b[r] = bL[r] ^ bR[r];
      b[r + Hf] = bR[r];
    }
  }
};

template <>
struct Rate1Words<5> {
  static __device__ __forceinline__ void run(const uint32_t (&H)[1], const uint32_t (&Z)[1],
                                             uint32_t (&b)[1]) {
    b[0] = rate1_word<5>(H[0], Z[0]);
  }
};

// SC over a node of 2^K leaves held in registers: returns beta (2^K bits)
// and u_hat in `u`.  frz / fv are the node's mask and frozen values in the
// low 2^K bits.  CHECK: test the node itself for rate 0 / rate 1 first.
// Nodes of up to 4 leaves take the generic path without class branches.
template <int K, int FK, bool CHECK, typename S>
struct Dec;

template <int K, int FK, bool CHECK, typename S>
struct DecGen {
  static constexpr int N = 1 << K, H = N / 2;
  static __device__ __forceinline__ uint32_t run(const float (&a)[N], uint32_t frz, uint32_t fv,
                                                 uint32_t &u, float sc) {
    constexpr uint32_t M = (N == 32) ? 0xFFFFFFFFu : ((1u << N) - 1u);
    constexpr uint32_t MH = (1u << H) - 1u;
    if (CHECK && K >= 5) {
      if (frz == M) {
        u = fv;
        return encode_word(fv, K);
      }
      if (frz == 0u) {
        uint32_t b;
        if (signs_if_nonzero<K>(a, &b)) {   // no zero input: signs are the decisions
          u = encode_word(b, K);
          return b;
        }
      }
    }
    float l[H], gp[H], gm[H];
    // Both outcomes of the right child's g, formed before the left child's
    // partial sums are known (b - a is b + (-a) in IEEE arithmetic, as in
    // g_bit); only a select waits for them.
#pragma unroll
    for (int j = 0; j < H; ++j) {
      gp[j] = rnd<S>(a[j + H] + a[j]);
      gm[j] = rnd<S>(a[j + H] - a[j]);
    }
    uint32_t uL, bL;
    const uint32_t fzL = frz & MH, fvL = fv & MH;
    if (K >= 3 && fzL == MH) {     // rate-0 left child: its f is never needed
      uL = fvL;
      bL = encode_word(fvL, K - 1);
    } else {
#pragma unroll
      for (int j = 0; j < H; ++j) l[j] = rnd<S>(f_scaled<FK>(a[j], a[j + H], sc));
      bL = Dec<K - 1, FK, true, S>::run(l, fzL, fvL, uL, sc);
    }
#pragma unroll
    for (int j = 0; j < H; ++j) l[j] = ((bL >> j) & 1u) ? gm[j] : gp[j];
    uint32_t uR;
    const uint32_t bR = Dec<K - 1, FK, true, S>::run(l, frz >> H, fv >> H, uR, sc);
    u = uL | (uR << H);
    return (bL ^ bR) | (bR << H);
  }
};

template <int K, int FK, bool CHECK, typename S>
struct Dec : DecGen<K, FK, CHECK, S> {};

// Two leaves.  The left leaf decides 1 iff f(a, b) < 0, and only that sign
// is ever used: f's magnitude feeds nothing else.  Both f forms return a
// nonzero magnitude with the sign product when a and b are nonzero and +-0
// when either is zero, so the decision is read off the sign bits -- for exact
// f that skips a whole special-function evaluation per node.  With an int8
// scale below 1 the scaled floor of exact f can underflow to zero, so scaled
// frames keep the full evaluation.  Same decisions, same bits.
template <int FK, bool CHECK, typename S>
struct Dec<1, FK, CHECK, S> {
  static __device__ __forceinline__ uint32_t run(const float (&a)[2], uint32_t frz, uint32_t fv,
                                                 uint32_t &u, float sc) {
    const float gp = rnd<S>(a[1] + a[0]), gm = rnd<S>(a[1] - a[0]);
    uint32_t u0;
    if (frz & 1u) {
      u0 = fv & 1u;
    } else if (FK == 0 || sc == 1.0f) {
      const uint32_t x0 = __float_as_uint(a[0]), x1 = __float_as_uint(a[1]);
      u0 = ((x0 ^ x1) >> 31) & (uint32_t)((x0 << 1) != 0u) & (uint32_t)((x1 << 1) != 0u);
    } else {
      u0 = rnd<S>(f_scaled<FK>(a[0], a[1], sc)) < 0.0f ? 1u : 0u;
    }
    const float r = u0 ? gm : gp;
    const uint32_t u1 = (frz & 2u) ? ((fv >> 1) & 1u) : (r < 0.0f ? 1u : 0u);
    u = u0 | (u1 << 1);
    return (u0 ^ u1) | (u1 << 1);
  }
};

template <int FK, bool CHECK, typename S>
struct Dec<0, FK, CHECK, S> {
  static __device__ __forceinline__ uint32_t run(const float (&a)[1], uint32_t frz, uint32_t fv,
                                                 uint32_t &u, float) {
    u = (frz & 1u) ? (fv & 1u) : (a[0] < 0.0f ? 1u : 0u);
    return u;
  }
};

// Hard-decision word (bit j = sign bit of a[j]) and zero word (bit j set iff
// a[j] is +-0) of N <= 32 values.  The sign bit of -0 is set, but
// rate1_word masks every zero position out of H, so it needs no test.
template <int N>
__device__ __forceinline__ void sign_zero_words(const float (&a)[N], uint32_t &h, uint32_t &z) {
  h = 0u;
  z = 0u;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const uint32_t x = __float_as_uint(a[j]);
    h |= (x >> 31) << j;
    z |= (uint32_t)((x << 1) == 0u) << j;
  }
}

// SC over a node of 2^K leaves whose frozen pattern PAT is known at compile
// time (bit j = leaf j frozen): the recursion of Dec with every class test
// resolved.  A rate-0 child is its encoded frozen values (and needs no f:
// the sibling's g then reads known partial sums); a rate-1 node takes the
// zero-aware closed form.  Same decisions, same bits.
template <int K, uint32_t PAT, int FK, typename S>
struct DecP {
  static constexpr int N = 1 << K, H = N / 2;
  static constexpr uint32_t M = (N == 32) ? 0xFFFFFFFFu : ((1u << N) - 1u);
  static constexpr uint32_t MH = (1u << H) - 1u;
  static constexpr uint32_t PL = PAT & MH, PR = (PAT >> H) & MH;
  static __device__ __forceinline__ uint32_t run(const float (&a)[N], uint32_t fv, uint32_t &u,
                                                 float sc) {
    if constexpr (PAT == M) {
      u = fv;
      return encode_word(fv, K);
    } else if constexpr (PAT == 0u && K >= 2) {
      uint32_t hb, zb;
      sign_zero_words<N>(a, hb, zb);
      const uint32_t b = rate1_word<K>(hb, zb);
      u = encode_word(b, K);
      return b;
    } else if constexpr (K == 1) {
      return Dec<1, FK, true, S>::run(a, PAT, fv, u, sc);
    } else {
      float l[H];
      uint32_t uL, bL;
      const uint32_t fvL = fv & MH;
      if constexpr (PL == MH) {
        uL = fvL;
        bL = encode_word(fvL, K - 1);
#pragma unroll
        for (int j = 0; j < H; ++j) l[j] = rnd<S>(g_bit(a[j], a[j + H], bL, j));
      } else {
        float gp[H], gm[H];
#pragma unroll
        for (int j = 0; j < H; ++j) {
          gp[j] = rnd<S>(a[j + H] + a[j]);
          gm[j] = rnd<S>(a[j + H] - a[j]);
        }
#pragma unroll
        for (int j = 0; j < H; ++j) l[j] = rnd<S>(f_scaled<FK>(a[j], a[j + H], sc));
        bL = DecP<K - 1, PL, FK, S>::run(l, fvL, uL, sc);
#pragma unroll
        for (int j = 0; j < H; ++j) l[j] = ((bL >> j) & 1u) ? gm[j] : gp[j];
      }
      uint32_t uR;
      const uint32_t bR = DecP<K - 1, PR, FK, S>::run(l, (fv >> H) & MH, uR, sc);
      u = uL | (uR << H);
      return (bL ^ bR) | (bR << H);
    }
  }
};

// 8-leaf nodes: the frozen patterns a polar construction can produce at 3
// index bits (the partial order of bit-channel reliability is a total order
// there, so a frozen set is one of its 9 down-sets) take specialised code;
// any other pattern the generic recursion.
template <int FK, typename S>
__device__ __noinline__ uint32_t dec8(const float (&a)[8], uint32_t frz, uint32_t fv, uint32_t &u,
                                      float sc) {
  switch (frz) {
    case 0xFFu: return DecP<3, 0xFFu, FK, S>::run(a, fv, u, sc);
    case 0x00u: return DecP<3, 0x00u, FK, S>::run(a, fv, u, sc);
    case 0x7Fu: return DecP<3, 0x7Fu, FK, S>::run(a, fv, u, sc);
    case 0x3Fu: return DecP<3, 0x3Fu, FK, S>::run(a, fv, u, sc);
    case 0x1Fu: return DecP<3, 0x1Fu, FK, S>::run(a, fv, u, sc);
    case 0x17u: return DecP<3, 0x17u, FK, S>::run(a, fv, u, sc);
    case 0x07u: return DecP<3, 0x07u, FK, S>::run(a, fv, u, sc);
    case 0x03u: return DecP<3, 0x03u, FK, S>::run(a, fv, u, sc);
    case 0x01u: return DecP<3, 0x01u, FK, S>::run(a, fv, u, sc);
    default: return DecGen<3, FK, true, S>::run(a, frz, fv, u, sc);
  }
}

// Exact f only: there each skipped node saves special-function chains, and
// one out-of-line copy keeps the code small (measured on the register tiles
// of the 2^20 BSC workload: 28 % fewer cycles).  Min-sum keeps the generic
// recursion, which measured faster there (its f is two instructions).
template <bool CHECK, typename S>
struct Dec<3, 1, CHECK, S> {
  static __device__ __forceinline__ uint32_t run(const float (&a)[8], uint32_t frz, uint32_t fv,
                                                 uint32_t &u, float sc) {
    return dec8<1, S>(a, frz, fv, u, sc);
  }
};

// ---------------------------------------------------------------- register tiles
// A node of 2^K leaves, 5 <= K <= 9, decoded in registers: element j of the
// node sits in lane j % 32, register j / 32, so every f and g of the levels
// 6..K pairs values of the same lane.  Masks, frozen values and partial sums
// are uniform words (identical in every lane).  A mixed node of 32 leaves is
// gathered through shared memory into every lane and decoded by Dec<5>.

// A 16-leaf node whose left child's f values q are already known (the rest
// of Dec<4>: same operations in the same order).
template <int FK, typename S>
__device__ __forceinline__ uint32_t dec16_given_left(const float (&l)[16], const float (&q)[8],
                                                     uint32_t frz, uint32_t fv, uint32_t &u,
                                                     float sc) {
  uint32_t uL, bL;
  const uint32_t fzL = frz & 0xFFu, fvL = fv & 0xFFu;
  if (fzL == 0xFFu) {              // rate-0 left child
    uL = fvL;
    bL = encode_word(fvL, 3);
  } else {
    bL = Dec<3, FK, true, S>::run(q, fzL, fvL, uL, sc);
  }
  float r[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) r[j] = rnd<S>(g_bit(l[j], l[j + 8], bL, j));
  uint32_t uR;
  const uint32_t bR = Dec<3, FK, true, S>::run(r, (frz >> 8) & 0xFFu, (fv >> 8) & 0xFFu, uR, sc);
  u = uL | (uR << 8);
  return (bL ^ bR) | (bR << 8);
}

// Mixed 32-leaf node with exact f (whose special-function cost dominates):
// the f and g values of the two top levels are computed once, lane-parallel
// (lane j forms value j), and gathered through shared memory; the 8-leaf
// nodes below run redundantly in every lane like Dec<5>.  Every value is the
// one Dec<5> forms, by the same operations, so the result is bit-identical.
// (A variant that runs both halves through one copy of the code, to relieve
// the instruction cache, measured 16 % slower.)
template <int FK, typename S>
__device__ __forceinline__ uint32_t dec32_lanes(float v, uint32_t m, uint32_t fv, uint32_t &u,
                                                float sc, float *gbuf, int lane) {
  const float hi = __shfl_down_sync(FULL, v, 16);   // leaf LLR lane + 16 (lanes < 16)
  float l[16], q[8];
  uint32_t uL, bL;
  if ((m & 0xFFFFu) == 0xFFFFu) {                    // rate-0 left child: no f values
    uL = fv & 0xFFFFu;
    bL = encode_word(uL, 4);
  } else {
    // Left 16-leaf child: its 16 f values, then its own left child's 8 f values.
    const float c = rnd<S>(f_scaled<FK>(v, hi, sc));
    const float d = rnd<S>(f_scaled<FK>(c, __shfl_down_sync(FULL, c, 8), sc));
    if (lane < 16) gbuf[lane] = c;
    if (lane < 8) gbuf[16 + lane] = d;
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 16; j += 4) {
      const float4 x = *reinterpret_cast<const float4 *>(gbuf + j);
      l[j] = x.x, l[j + 1] = x.y, l[j + 2] = x.z, l[j + 3] = x.w;
    }
#pragma unroll
    for (int j = 0; j < 8; j += 4) {
      const float4 x = *reinterpret_cast<const float4 *>(gbuf + 16 + j);
      q[j] = x.x, q[j + 1] = x.y, q[j + 2] = x.z, q[j + 3] = x.w;
    }
    bL = dec16_given_left<FK, S>(l, q, m & 0xFFFFu, fv & 0xFFFFu, uL, sc);
  }
  // Right child: its 16 g values with the left child's partial sums, then
  // its left child's 8 f values.
  const float c = rnd<S>(g_bit(v, hi, bL, lane));
  const float d = rnd<S>(f_scaled<FK>(c, __shfl_down_sync(FULL, c, 8), sc));
  if (lane < 16) gbuf[32 + lane] = c;
  if (lane < 8) gbuf[48 + lane] = d;
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 16; j += 4) {
    const float4 x = *reinterpret_cast<const float4 *>(gbuf + 32 + j);
    l[j] = x.x, l[j + 1] = x.y, l[j + 2] = x.z, l[j + 3] = x.w;
  }
#pragma unroll
  for (int j = 0; j < 8; j += 4) {
    const float4 x = *reinterpret_cast<const float4 *>(gbuf + 48 + j);
    q[j] = x.x, q[j + 1] = x.y, q[j + 2] = x.z, q[j + 3] = x.w;
  }
  __syncwarp();
  uint32_t uR;
  const uint32_t bR = dec16_given_left<FK, S>(l, q, m >> 16, fv >> 16, uR, sc);
  u = uL | (uR << 16);
  return (bL ^ bR) | (bR << 16);
}

// Mixed or shortcut 32-leaf node; v = this lane's LLR.  Returns beta in the low
// word and u_hat in the high word.
template <int FK, typename S, bool UH>
__device__ __forceinline__ uint64_t tile32_body(float v, uint32_t m, uint32_t fv, float sc,
                                                float *gbuf, int lane) {
  if (m == FULL) return (uint64_t)encode_word(fv, 5) | ((uint64_t)fv << 32);
  if (m == 0u) {                                    // rate 1, zero inputs included
    const uint32_t b =
        rate1_word<5>(__ballot_sync(FULL, v < 0.0f), __ballot_sync(FULL, v == 0.0f));
    return (uint64_t)b | ((uint64_t)(UH ? encode_word(b, 5) : 0u) << 32);
  }
  if (FK != 0 && m != 0x7FFFFFFFu) {    // exact f; a repetition node needs no f at all
    uint32_t u;
    const uint32_t b = dec32_lanes<FK, S>(v, m, fv, u, sc, gbuf, lane);
    return (uint64_t)b | ((uint64_t)(UH ? u : 0u) << 32);
  }
  gbuf[lane] = v;
  __syncwarp();
  float a[32];
#pragma unroll
  for (int j = 0; j < 32; j += 4) {
    const float4 q = *reinterpret_cast<const float4 *>(gbuf + j);
    a[j] = q.x;
    a[j + 1] = q.y;
    a[j + 2] = q.z;
    a[j + 3] = q.w;
  }
  __syncwarp();
  uint32_t u, b;
  if constexpr (FK != 0) {
    b = DecP<5, 0x7FFFFFFFu, FK, S>::run(a, fv, u, sc);   // the repetition node
  } else {
    // Min-sum: compile-time decoders for the five mixed patterns that make up
    // 60-90 % of the mixed 32-leaf nodes of every tested code (BSC and BI-AWGN,
    // 2^16..2^22, rates 0.44..0.82): the repetition node, the single-parity
    // node and three down-sets between them.  Other patterns take the generic
    // recursion.
    switch (m) {
      case 0x7FFFFFFFu: b = DecP<5, 0x7FFFFFFFu, FK, S>::run(a, fv, u, sc); break;
      case 0x177F7FFFu: b = DecP<5, 0x177F7FFFu, FK, S>::run(a, fv, u, sc); break;
      case 0x0117177Fu: b = DecP<5, 0x0117177Fu, FK, S>::run(a, fv, u, sc); break;
      case 0x00010117u: b = DecP<5, 0x00010117u, FK, S>::run(a, fv, u, sc); break;
      case 0x00000001u: b = DecP<5, 0x00000001u, FK, S>::run(a, fv, u, sc); break;
      default: b = Dec<5, FK, false, S>::run(a, m, fv, u, sc); break;
    }
  }
  return (uint64_t)b | ((uint64_t)(UH ? u : 0u) << 32);
}

// The one out-of-line copy of the 32-leaf decoder that every 32-leaf node of a
// min-sum register tile calls (inlining it at the tile's 16 call sites
// doubled the tile's time: instruction cache).
template <int FK, typename S, bool UH>
__device__ __noinline__ uint64_t tile32(float v, uint32_t m, uint32_t fv, float sc, float *gbuf,
                                        int lane) {
  return tile32_body<FK, S, UH>(v, m, fv, sc, gbuf, lane);
}

template <int K, int FK, typename S, bool UH>
struct Tile;

template <int FK, typename S, bool UH>
__device__ __noinline__ uint4 tile64(float c0, float c1, uint32_t m0, uint32_t m1, uint32_t f0,
                                     uint32_t f1, float sc, float *gbuf, int lane);

// Child node of 2^K leaves of a register tile.  Exact f decodes each 64-leaf
// node in one out-of-line call (tile64, with the 32-leaf decoder inlined into
// it) and so makes half the calls (1-3 % faster there); min-sum keeps one
// call per 32-leaf node (the same change measured 6.6 % slower with it).
template <int K, int FK, typename S, bool UH>
__device__ __forceinline__ void tile_child(const float (&c)[1 << (K - 5)], const uint32_t *m,
                                           const uint32_t *fv, uint32_t (&b)[1 << (K - 5)],
                                           uint32_t (&u)[1 << (K - 5)], float sc, float *gbuf,
                                           int lane) {
  if constexpr (K == 6 && FK != 0) {
    const uint4 r = tile64<FK, S, UH>(c[0], c[1], m[0], m[1], fv[0], fv[1], sc, gbuf, lane);
    b[0] = r.x;
    b[1] = r.y;
    u[0] = r.z;
    u[1] = r.w;
  } else {
    Tile<K, FK, S, UH>::run(c, m, fv, b, u, sc, gbuf, lane);
  }
}

template <int K, int FK, typename S, bool UH>
struct Tile {
  static constexpr int R = 1 << (K - 5), H = R / 2;
  static __device__ __forceinline__ void run(const float (&v)[R], const uint32_t *m,
                                             const uint32_t *fv, uint32_t (&bo)[R],
                                             uint32_t (&uo)[R], float sc, float *gbuf, int lane) {
    bool all1 = true, all0 = true;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      all1 &= (m[r] == FULL);
      all0 &= (m[r] == 0u);
    }
    if (all1) {                                   // rate 0
#pragma unroll
      for (int r = 0; r < R; ++r) {
        bo[r] = encode_word(fv[r], 5);
        uo[r] = fv[r];
      }
#pragma unroll
      for (int hw = 1; hw < R; hw *= 2)
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (!(r & hw)) bo[r] ^= bo[r + hw];
      return;
    }
    if (all0) {                                   // rate 1, zero inputs included
      uint32_t H[R], Z[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        H[r] = __ballot_sync(FULL, v[r] < 0.0f);
        Z[r] = __ballot_sync(FULL, v[r] == 0.0f);
      }
      Rate1Words<K>::run(H, Z, bo);
      if (UH) {
#pragma unroll
        for (int r = 0; r < R; ++r) uo[r] = encode_word(bo[r], 5);
#pragma unroll
        for (int hw = 1; hw < R; hw *= 2)
#pragma unroll
          for (int r = 0; r < R; ++r)
            if (!(r & hw)) uo[r] ^= uo[r + hw];
      }
      return;
    }
    float c[H];
    uint32_t bL[H], uL[H], bR[H], uR[H];
    bool left0 = true;
#pragma unroll
    for (int r = 0; r < H; ++r) left0 &= (m[r] == FULL);
    if (left0) {                                  // rate-0 left child: no f needed
#pragma unroll
      for (int r = 0; r < H; ++r) {
        bL[r] = encode_word(fv[r], 5);
        uL[r] = fv[r];
      }
#pragma unroll
      for (int hw = 1; hw < H; hw *= 2)
#pragma unroll
        for (int r = 0; r < H; ++r)
          if (!(r & hw)) bL[r] ^= bL[r + hw];
    } else {
#pragma unroll
      for (int r = 0; r < H; ++r) c[r] = rnd<S>(f_scaled<FK>(v[r], v[r + H], sc));
      tile_child<K - 1, FK, S, UH>(c, m, fv, bL, uL, sc, gbuf, lane);
    }
    const int sh = 31 - lane;
#pragma unroll
    for (int r = 0; r < H; ++r)
      c[r] = rnd<S>(v[r + H] + __uint_as_float(__float_as_uint(v[r]) ^
                                              ((bL[r] << sh) & 0x80000000u)));
    tile_child<K - 1, FK, S, UH>(c, m + H, fv + H, bR, uR, sc, gbuf, lane);
#pragma unroll
    for (int r = 0; r < H; ++r) {
      bo[r] = bL[r] ^ bR[r];
      bo[r + H] = bR[r];
      uo[r] = uL[r];
      uo[r + H] = uR[r];
    }
  }
};

template <int FK, typename S, bool UH>
struct Tile<5, FK, S, UH> {
  static __device__ __forceinline__ void run(const float (&v)[1], const uint32_t *m,
                                             const uint32_t *fv, uint32_t (&bo)[1],
                                             uint32_t (&uo)[1], float sc, float *gbuf, int lane) {
    uint64_t r;
    if constexpr (FK != 0) r = tile32_body<FK, S, UH>(v[0], m[0], fv[0], sc, gbuf, lane);
    else r = tile32<FK, S, UH>(v[0], m[0], fv[0], sc, gbuf, lane);
    bo[0] = (uint32_t)r;
    uo[0] = (uint32_t)(r >> 32);
  }
};

template <int FK, typename S, bool UH>
__device__ __noinline__ uint4 tile64(float c0, float c1, uint32_t m0, uint32_t m1, uint32_t f0,
                                     uint32_t f1, float sc, float *gbuf, int lane) {
  const float v[2] = {c0, c1};
  const uint32_t m[2] = {m0, m1}, fv[2] = {f0, f1};
  uint32_t b[2], u[2];
  Tile<6, FK, S, UH>::run(v, m, fv, b, u, sc, gbuf, lane);
  return make_uint4(b[0], b[1], u[0], u[1]);
}

// The CTA of NW warps decoding one subtree.  Shared-memory levels use every
// thread; register tiles and the 32-leaf decoder run in warp 0 only.
template <typename S, int NW>
struct Warp {
  static constexpr uint32_t nth = 32 * NW;
  S *L;
  uint32_t *beta, *uh, *msk, *fvw;
  const uint32_t *cr0, *cr1;   // class table: bit 2^(t-k) + (o >> k) for level k >= 5
  int lane, t;
  uint32_t tid;

  __device__ __forceinline__ void sync() const {
    if (NW == 1) __syncwarp();
    else __syncthreads();
  }
  __device__ __forceinline__ bool any(bool b) const {
    if (NW == 1) return __any_sync(FULL, b);
    return __syncthreads_or(b) != 0;
  }
  float sc;                    // int8 per-frame scale (1 otherwise)
  float *gbuf;                 // 64 floats: gather buffer of the register tiles

  // Node of 2^K leaves (5 <= K <= 9) at leaf o, decoded by a register tile.
  template <int K, int FK, bool UH>
  __device__ void tile(uint32_t o) const {
    constexpr int R = 1 << (K - 5);
    const S *src = lvl(K);
    float v[R];
    uint32_t m[R], fv[R], bo[R], uo[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      v[r] = Store<S>::ld(src + 32 * r + lane);
      m[r] = msk[(o >> 5) + r];
      fv[r] = fvw[(o >> 5) + r];
    }
    Tile<K, FK, S, UH>::run(v, m, fv, bo, uo, sc, gbuf, lane);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (lane == r) {
        beta[(o >> 5) + r] = bo[r];
        if (UH) uh[(o >> 5) + r] = uo[r];
      }
    }
    __syncwarp();
  }

  template <int FK, bool UH>
  __device__ void tile_k(int k, uint32_t o) const {
    switch (k) {
      case 5: tile<5, FK, UH>(o); break;
      case 6: tile<6, FK, UH>(o); break;
      case 7: tile<7, FK, UH>(o); break;
      case 8: tile<8, FK, UH>(o); break;
      default: tile<9, FK, UH>(o); break;
    }
  }

  __device__ __forceinline__ S *lvl(int k) const { return L + (1u << k); }

  // Class of a node of level k >= 5 from the table.
  __device__ __forceinline__ int cls_tab(int k, uint32_t o) const {
    uint32_t i = (1u << (t - k)) + (o >> k);
    uint32_t b0 = (cr0[i >> 5] >> (i & 31)) & 1u, b1 = (cr1[i >> 5] >> (i & 31)) & 1u;
    return b0 ? NODE_RATE0 : (b1 ? NODE_RATE1 : NODE_MIXED);
  }

  // Mixed node of 2^K leaves (K <= 5) at leaf o, decoded in registers.
  template <int K, int FK, bool CHECK, bool UH>
  __device__ void leafblock(uint32_t o) const {
    constexpr int N = 1 << K;
    const S *src = lvl(K);
    float a[N];
    if constexpr (sizeof(S) == 4 && N >= 4) {     // level K starts 16-byte aligned
#pragma unroll
      for (int j = 0; j < N; j += 4) {
        float4 q = *reinterpret_cast<const float4 *>(src + j);
        a[j] = q.x;
        a[j + 1] = q.y;
        a[j + 2] = q.z;
        a[j + 3] = q.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < N; ++j) a[j] = Store<S>::ld(src + j);
    }
    const uint32_t m = N == 32 ? 0xFFFFFFFFu : ((1u << N) - 1u);
    const uint32_t sh = o & 31;
    uint32_t u;
    uint32_t b =
        Dec<K, FK, CHECK, S>::run(a, (msk[o >> 5] >> sh) & m, (fvw[o >> 5] >> sh) & m, u, sc);
    if (lane == 0) {
      insert(beta, o, N, b);
      if (UH) insert(uh, o, N, u);
    }
    __syncwarp();
  }

  // Cross-word transform levels of the words [w0, w0 + nw) of `v`.
  __device__ void xword_encode(uint32_t *v, uint32_t w0, uint32_t nw) const {
    for (uint32_t hw = 1; hw < nw; hw <<= 1) {
      sync();
      for (uint32_t j = tid; j < nw / 2; j += nth) {
        uint32_t a = (j / hw) * 2 * hw + (j % hw);
        v[w0 + a] ^= v[w0 + a + hw];
      }
    }
    sync();
  }

  __device__ void insert(uint32_t *v, uint32_t o, int nbits, uint32_t bits) const {
    uint32_t m = low_mask(nbits) << (o & 31);
    v[o >> 5] = (v[o >> 5] & ~m) | ((bits << (o & 31)) & m);
  }

  template <bool UH = true>
  __device__ void rate0(int k, uint32_t o) const {
    if (k >= 5) {
      uint32_t w0 = o >> 5, nw = 1u << (k - 5);
      for (uint32_t i = tid; i < nw; i += nth) {
        uint32_t v = fvw[w0 + i];
        if (UH) uh[w0 + i] = v;
        beta[w0 + i] = encode_word(v, 5);
      }
      xword_encode(beta, w0, nw);
    } else {
      if (tid == 0) {
        uint32_t v = (fvw[o >> 5] >> (o & 31)) & low_mask(1 << k);
        insert(uh, o, 1 << k, v);
        insert(beta, o, 1 << k, encode_word(v, k));
      }
      sync();
    }
  }

  // Rate-1 shortcut (k >= 5); false (nothing written) when some input is +-0.
  // Each lane builds whole words of hard decisions (32 LLRs per word), so a
  // node costs one pass over its LLRs and one vote.
  template <bool UH>
  __device__ bool rate1(int k, uint32_t o) const {
    const S *Lk = lvl(k);
    const uint32_t w0 = o >> 5, nw = 1u << (k - 5);
    if (NW == 1 && nw == 1) {
      const float v = Store<S>::ld(Lk + lane);
      if (__any_sync(FULL, v == 0.0f)) return false;
      const uint32_t b = __ballot_sync(FULL, v < 0.0f);
      if (lane == 0) {
        beta[w0] = b;
        if (UH) uh[w0] = encode_word(b, 5);
      }
      __syncwarp();
      return true;
    }
    bool z = false;
    uint32_t words[8];                   // nw <= 2^(t-5) <= 512: 16 words per lane at most
#pragma unroll
    for (int r = 0; r < 8; ++r) words[r] = 0u;
    for (uint32_t i = tid, r = 0; i < nw; i += nth, ++r) {
      uint32_t b = 0u;
      const S *q = Lk + 32 * i;
      if constexpr (sizeof(S) == 4) {   // level k >= 6 starts 16-byte aligned
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          const float4 v = *reinterpret_cast<const float4 *>(q + j);
          z |= (v.x == 0.0f) | (v.y == 0.0f) | (v.z == 0.0f) | (v.w == 0.0f);
          b |= ((v.x < 0.0f ? 1u : 0u) | (v.y < 0.0f ? 2u : 0u) | (v.z < 0.0f ? 4u : 0u) |
                (v.w < 0.0f ? 8u : 0u)) << j;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float v = Store<S>::ld(q + j);
          z |= (v == 0.0f);
          b |= (v < 0.0f ? 1u : 0u) << j;
        }
      }
      if (r < 8) words[r] = b;
      else beta[w0 + i] = b;             // beyond the register window: park directly
    }
    if (any(z)) return false;
    for (uint32_t i = tid, r = 0; i < nw && r < 8; i += nth, ++r) beta[w0 + i] = words[r];
    if (UH) {
      sync();
      for (uint32_t i = tid; i < nw; i += nth) uh[w0 + i] = encode_word(beta[w0 + i], 5);
      xword_encode(uh, w0, nw);
    } else {
      sync();
    }
    return true;
  }

  __device__ void leaf(uint32_t o) const {
    if (tid == 0) {
      uint32_t w = o >> 5, s = o & 31;
      uint32_t u = ((msk[w] >> s) & 1u) ? ((fvw[w] >> s) & 1u)
                                        : (uint32_t)(Store<S>::ld(lvl(0)) < 0.0f);
      insert(beta, o, 1, u);
      insert(uh, o, 1, u);
    }
    sync();
  }

  template <int FK>
  __device__ void f(int k) const {
    const S *__restrict__ a = lvl(k);
    S *__restrict__ c = lvl(k - 1);
    const uint32_t h = 1u << (k - 1);
    if (h >= 4 * nth) {
      for (uint32_t i = tid; i < h; i += 4 * nth) {
        float x[4], y[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          x[q] = Store<S>::ld(a + i + nth * q);
          y[q] = Store<S>::ld(a + h + i + nth * q);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) Store<S>::st(c + i + nth * q, f_scaled<FK>(x[q], y[q], sc));
      }
    } else {
      for (uint32_t i = tid; i < h; i += nth)
        Store<S>::st(c + i, f_scaled<FK>(Store<S>::ld(a + i), Store<S>::ld(a + h + i), sc));
    }
    sync();
  }

  // Right child of the node of level k whose left child starts at leaf o.
  __device__ void g(int k, uint32_t o) const {
    const S *__restrict__ a = lvl(k);
    S *__restrict__ c = lvl(k - 1);
    const uint32_t h = 1u << (k - 1);
    if (h >= 4 * nth) {
      for (uint32_t i = tid; i < h; i += 4 * nth) {
        float x[4], y[4];
        uint32_t wd[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          x[q] = Store<S>::ld(a + i + nth * q);
          y[q] = Store<S>::ld(a + h + i + nth * q);
          wd[q] = beta[(o + i + nth * q) >> 5];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
          Store<S>::st(c + i + nth * q, g_bit(x[q], y[q], wd[q], (o + i) & 31));
      }
    } else {
      for (uint32_t i = tid; i < h; i += nth) {
        uint32_t p = o + i;
        Store<S>::st(c + i, g_bit(Store<S>::ld(a + i), Store<S>::ld(a + h + i), beta[p >> 5],
                                  p & 31));
      }
    }
    sync();
  }

  // Parent of level K at leaf base: left half ^= right half.
  __device__ void combine(int K, uint32_t base) const {
    const uint32_t h = 1u << (K - 1);
    if (h >= 32) {
      uint32_t w0 = base >> 5, hw = h >> 5;
      for (uint32_t i = tid; i < hw; i += nth) beta[w0 + i] ^= beta[w0 + hw + i];
    } else if (tid == 0) {
      uint32_t w = beta[base >> 5], s = base & 31;
      uint32_t r = (w >> (s + h)) & low_mask(h);
      beta[base >> 5] = w ^ (r << s);
    }
    sync();
  }
};

// Words of shared memory before the LLR levels: beta, u_hat, mask, frozen
// values (W each), the two class-table halves (CW each), rounded up to 16 B,
// then the 32-float gather buffer of the register tiles.
__host__ __device__ inline uint32_t bit_words(int t) {
  const uint32_t W = t >= 5 ? (1u << (t - 5)) : 1u;
  const uint32_t CW = t >= 9 ? (1u << (t - 9)) : 1u;
  return ((4 * W + 2 * CW + 3u) & ~3u) + 64u;
}

// Tin: storage of the level-t input (the streamed levels); inside the CTA
// every level is float.
// NW warps: kScWarps with shortcuts (shared-memory levels spread over the CTA), 1
// for the plain decoder.
// Decodes the subtree of frame `fr` (row fr of every strided argument) with
// the CTA's threads; smraw is the dynamic shared memory (bit_words(t) words
// then 2^(t+1) floats).  The whole CTA must call it.
template <int NW, typename Tin, int FK, bool SC, bool UH>
__device__ __forceinline__ void subtree_body(const StParams &p, bool in_is_llr, size_t fr,
                                             unsigned char *smraw) {
  using S = float;
  constexpr uint32_t nth = 32 * NW;
  const int t = p.t;
  const uint32_t T = 1u << t;
  const uint32_t W = T >= 32 ? T / 32 : 1;
  const uint32_t CW = t >= 9 ? (1u << (t - 9)) : 1u;
  const uint32_t tid = threadIdx.x;
  const int lane = tid & 31;
  const bool warp0 = tid < 32;

  Warp<S, NW> w;
  w.lane = lane;
  w.tid = tid;
  w.t = t;
  w.sc = p.scale ? p.scale[fr] : 1.0f;
  w.beta = reinterpret_cast<uint32_t *>(smraw);
  w.uh = w.beta + W;
  w.msk = w.beta + 2 * W;
  w.fvw = w.beta + 3 * W;
  uint32_t *ctab = w.beta + 4 * W;
  w.cr0 = ctab;
  w.cr1 = ctab + CW;
  w.L = reinterpret_cast<S *>(w.beta + bit_words(t));
  w.gbuf = reinterpret_cast<float *>(w.beta + bit_words(t) - 64);

  const uint64_t ow = p.o >> 5;
  const uint32_t *fvf = p.fv + fr * p.w_stride + ow;
  for (uint32_t i = tid; i < W; i += nth) {
    w.msk[i] = p.mask[ow + i];
    w.fvw[i] = fvf[i];
    w.beta[i] = 0u;
    w.uh[i] = 0u;
  }
  if (SC && p.cls)
    for (uint32_t i = tid; i < 2 * CW; i += nth) ctab[i] = p.cls[i];
  S *Lt = w.lvl(t);
  if (std::is_same<Tin, float>::value && !p.scale && T >= 32) {
    // float32 storage (the only one the schedule fuses the parent's step
    // into): the input rows go to shared memory with cp.async, every copy in
    // flight at once.  pre = 0: level t itself, straight into Lt.
    // pre = 1 / 2: the parent's 2T values into L[0, 2T) (the lower half is
    // free -- it holds the levels below t), then level t is formed in place:
    // its f (left child) or its g with the left child's partial sums from
    // x_hat (right child) -- the float operations of the streamed step this
    // replaces.
    const float *src = reinterpret_cast<const float *>(p.in) + fr * p.in_stride + p.in_o;
    float *dst = p.pre ? w.L : Lt;
    const uint32_t n4 = (p.pre ? 2 * T : T) / 4;
    for (uint32_t i = tid; i < n4; i += nth) cp16(dst + 4 * i, src + 4 * i);
    cp_commit();
    cp_wait<0>();
    w.sync();
    if (p.pre) {
      const uint32_t *bw = p.pre == 2 ? p.xhat + fr * p.w_stride + ((p.o - T) >> 5) : nullptr;
      const float4 *a4 = reinterpret_cast<const float4 *>(w.L);
      float4 *b4 = reinterpret_cast<float4 *>(Lt);
      for (uint32_t i = tid; i < T / 4; i += nth) {
        const float4 a = a4[i], b = b4[i];
        float4 v;
        if (p.pre == 1) {
          v = make_float4(f_st<Tin, FK>(a.x, b.x, 1.0f), f_st<Tin, FK>(a.y, b.y, 1.0f),
                          f_st<Tin, FK>(a.z, b.z, 1.0f), f_st<Tin, FK>(a.w, b.w, 1.0f));
        } else {
          const uint32_t wd = bw[i >> 3];
          const int j = (int)((i & 7) << 2);
          v = make_float4(g_bit(a.x, b.x, wd, j), g_bit(a.y, b.y, wd, j + 1),
                          g_bit(a.z, b.z, wd, j + 2), g_bit(a.w, b.w, wd, j + 3));
        }
        b4[i] = v;                                 // element i of level t, in place
      }
    }
  } else if (in_is_llr) {
    // Level-t LLRs into shared memory with 16-byte loads, eight in flight per
    // lane (one warp would otherwise wait a memory latency per element).
    const float *src = reinterpret_cast<const float *>(p.in) + fr * p.in_stride + p.in_o;
    if (T >= 4) {
      const float4 *s4 = reinterpret_cast<const float4 *>(src);
      for (uint32_t b = 0; b < T / 4; b += nth * 8) {
        float4 q[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const uint32_t i = b + nth * r + tid;
          if (i < T / 4) q[r] = s4[i];
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const uint32_t i = b + nth * r + tid;
          if (i < T / 4) {
            Lt[4 * i] = rnd<Tin>(q[r].x * w.sc);
            Lt[4 * i + 1] = rnd<Tin>(q[r].y * w.sc);
            Lt[4 * i + 2] = rnd<Tin>(q[r].z * w.sc);
            Lt[4 * i + 3] = rnd<Tin>(q[r].w * w.sc);
          }
        }
      }
    } else {
      for (uint32_t i = tid; i < T; i += nth) Lt[i] = rnd<Tin>(src[i] * w.sc);
    }
  } else {
    // Tin-typed level t widened to float: a thread loads four values at a time
    // (8 bytes of half, 4 of int8; eight loads in flight, past L1 since a node
    // CTA writes level t with st.cg) and stores them as one float4, so a warp's
    // shared-memory stores are consecutive 16-byte words (no bank conflicts).
    const Tin *src = reinterpret_cast<const Tin *>(p.in) + fr * p.in_stride;
    using Q = typename std::conditional<
        sizeof(Tin) == 2, uint2,
        typename std::conditional<sizeof(Tin) == 1, uint32_t, uint4>::type>::type;
    constexpr uint32_t PER = sizeof(Q) / sizeof(Tin);        // 4
    const uint32_t nq = T / PER;                             // T >= 32 here
    const Q *sq = reinterpret_cast<const Q *>(src);
    for (uint32_t b = 0; b < nq; b += nth * 8) {
      Q q[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const uint32_t i = b + nth * r + tid;
        if (i < nq) q[r] = __ldcg(sq + i);
      }
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const uint32_t i = b + nth * r + tid;
        if (i < nq) {
          const Tin *e = reinterpret_cast<const Tin *>(&q[r]);
          *reinterpret_cast<float4 *>(Lt + PER * i) =
              make_float4(Store<Tin>::ld(e), Store<Tin>::ld(e + 1), Store<Tin>::ld(e + 2),
                          Store<Tin>::ld(e + 3));
        }
      }
    }
  }
  w.sync();

  if (SC && t < 5) {
    // whole code shorter than a word: one register block with class checks
    if (warp0) {
      switch (t) {
        case 1: w.template leafblock<1, FK, true, UH>(0); break;
        case 2: w.template leafblock<2, FK, true, UH>(0); break;
        case 3: w.template leafblock<3, FK, true, UH>(0); break;
        default: w.template leafblock<4, FK, true, UH>(0); break;
      }
    }
    w.sync();
  } else {
    int k = t;
    uint32_t o = 0;
    for (;;) {
      for (;;) {                                 // descend
        if (SC) {
          if (k <= 9) {                          // register tile (k = min(t, 9))
            if (warp0) w.template tile_k<FK, UH>(k, o);
            w.sync();
            break;
          }
          const int cls = w.cls_tab(k, o);
          if (cls == NODE_RATE0) {
            w.template rate0<UH>(k, o);
            break;
          }
          if (cls == NODE_RATE1 && w.template rate1<UH>(k, o)) break;
          if (w.cls_tab(k - 1, o) != NODE_RATE0) w.template f<FK>(k);
        } else {
          if (k == 0) {
            w.leaf(o);
            break;
          }
          w.template f<FK>(k);
        }
        --k;
      }
      while (k < t && ((o >> k) & 1u)) {         // ascend through right children
        w.combine(k + 1, o - (1u << k));
        o -= 1u << k;
        ++k;
      }
      if (k == t) break;
      w.g(k + 1, o);                             // right sibling's LLRs
      o += 1u << k;
    }
  }

  uint32_t *xf = p.xhat + fr * p.w_stride + ow;
  uint32_t *uf = p.uhat ? p.uhat + fr * p.w_stride + ow : nullptr;
  const uint32_t keep = T >= 32 ? FULL : low_mask(T);
  for (uint32_t i = tid; i < W; i += nth) {
    xf[i] = w.beta[i] & keep;
    if (uf) uf[i] = w.uh[i] & keep;
  }
  __syncthreads();
  if (p.r > 0) cascade_device(p.xhat + fr * p.w_stride, t, p.o, p.r);
}

template <int NW, typename Tin, int FK, bool SC, bool UH>
__global__ void __launch_bounds__(32 * NW) k_subtree(StParams p, bool in_is_llr) {
  extern __shared__ __align__(16) unsigned char smraw[];
  pdl_enter();
  subtree_body<NW, Tin, FK, SC, UH>(p, in_is_llr, blockIdx.x, smraw);
}

template <typename Tin, int FK, bool SC, bool UH>
cudaError_t launch_t(const SubtreeArgs &a, cudaStream_t s) {
  using S = float;
  constexpr int NW = SC ? kScWarps : 1;
  const uint32_t T = 1u << a.t;
  const uint32_t W = T >= 32 ? T / 32 : 1;
  (void)W;
  size_t smem = bit_words(a.t) * sizeof(uint32_t) + 2 * (size_t)T * sizeof(S);
  auto kern = k_subtree<NW, Tin, FK, SC, UH>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  // float input rows are whole frames: the subtree's (or its parent's) offset
  const uint64_t in_o = !a.in_is_llr ? 0 : a.pre ? (a.o >> (a.t + 1)) << (a.t + 1) : a.o;
  StParams p{a.in,   a.in_stride, in_o,       a.cls, a.scale, a.mask, a.fv,
             a.xhat, a.uhat,      a.w_stride, a.o,   a.t,     a.r,    a.pre};
  return counted(launch_k(kern, a.nframes, 32 * NW, smem, s, p, a.in_is_llr), 1);
}

template <typename S>
cudaError_t launch_s(const SubtreeArgs &a, cudaStream_t s) {
  const bool uh = a.uhat != nullptr;
  if (a.fkind == 0) {
    if (!a.shortcuts) return launch_t<S, 0, false, true>(a, s);
    return uh ? launch_t<S, 0, true, true>(a, s) : launch_t<S, 0, true, false>(a, s);
  }
  if (!a.shortcuts) return launch_t<S, 1, false, true>(a, s);
  return uh ? launch_t<S, 1, true, true>(a, s) : launch_t<S, 1, true, false>(a, s);
}

}  // namespace

}  // namespace polar
