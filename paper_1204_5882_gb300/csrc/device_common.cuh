// Device-side building blocks shared by the streamed and the subtree kernels.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <utility>

namespace polar {

// ---------------------------------------------------------------- launches
// Programmatic dependent launch (PDL): a kernel of the decode sequence first
// waits until the grids it depends on have completed and their writes are
// visible, then lets the next grid of the stream start launching, so that
// the next kernel's launch and block scheduling overlap this one's tail.
// Both instructions are no-ops in a grid launched without the attribute.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

extern std::atomic<int> g_pdl;   // 1 = launch the decode sequence with PDL

// <<<grid, block, smem, s>>> with the programmatic-serialization attribute
// when g_pdl is set.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t s, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = g_pdl.load(std::memory_order_relaxed);
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Asynchronous global -> shared copies (cp.async): a thread's copies land
// in shared memory without holding registers while in flight; the thread
// waits for its own groups (cp_wait) and a barrier publishes them to the CTA.
__device__ __forceinline__ void cp16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------- f and g
// Min-sum check-node update: sign = - iff exactly one input has its sign bit
// set, magnitude = min(|a|, |b|).  Bit-exact with a float32 recursive SC.
__device__ __forceinline__ float f_minsum(float a, float b) {
  float m = fminf(fabsf(a), fabsf(b));
  uint32_t s = (__float_as_uint(a) ^ __float_as_uint(b)) & 0x80000000u;
  return __uint_as_float(__float_as_uint(m) | s);
}

// Exact check-node update f = 2 atanh(tanh(a/2) tanh(b/2)) (Sec. 4's update
// through phi), evaluated as
//   sgn(a) sgn(b) [min(A,B) + c(A+B) - c(|A-B|)],  c(d) = ln(1 + e^-d),
// which never forms atanh(+-1).  With e^x = 2^(x log2 e) and
// ln y = ln 2 * log2 y, the two corrections are taken in base 2 on the
// special-function unit (ex2 / lg2, approximate: absolute error ~1e-7, far
// below any LLR that decides a bit), their difference first, then one fused
// multiply-add with ln 2 onto min(A,B).  Every step is an explicit
// instruction or rounded operation, so the result is the same in every
// calling context, and an input of +-0 (where the two corrections are the
// same number) gives exactly +-0.  For small inputs the terms cancel and
// rounding can leave zero or a negative value where the exact update is tiny
// but nonzero; the magnitude is then raised to the smallest positive float.
// The result thus always carries the exact update's sign: the product of the
// input signs when both are nonzero, +-0 otherwise -- what the rate-1 shortcut
// and the 2-leaf decision rule rely on.  Exact f is compared with the float64
// oracle statistically (frame and bit error rates).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// log2(1 + e^-d), i.e. c(d) / ln 2
__device__ __forceinline__ float corr_log2(float d) {
  return lg2_approx(1.0f + ex2_approx(d * -1.4426950408889634f));
}

__device__ __forceinline__ float f_exact(float a, float b) {
  float A = fabsf(a), B = fabsf(b);
  const float dl = __fsub_rn(corr_log2(A + B), corr_log2(fabsf(A - B)));
  float m = __fmaf_rn(dl, 0.69314718055994531f, fminf(A, B));
  m = fmaxf(m, fminf(A, B) > 0.0f ? __uint_as_float(1u) : 0.0f);
  uint32_t s = (__float_as_uint(a) ^ __float_as_uint(b)) & 0x80000000u;
  return __uint_as_float(__float_as_uint(m) | s);
}

template <int FK>
__device__ __forceinline__ float f_op(float a, float b) {
  if (FK == 0) return f_minsum(a, b);
  return f_exact(a, b);
}

// Variable-node update with the left child's partial sum u: b + a or b - a.
__device__ __forceinline__ float g_op(float a, float b, uint32_t u) {
  return u ? (b - a) : (b + a);
}

// ---------------------------------------------------------------- storage
// Intermediate LLRs are stored as float, half (round to nearest even,
// saturated at +-65504) or int8 (round to nearest even, saturated at +-127,
// values are L * per-frame scale); every f and g runs in float.
template <typename S>
struct Store;

template <>
struct Store<float> {
  static __device__ __forceinline__ float ld(const float *p) { return *p; }
  static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};

template <>
struct Store<__half> {
  static __device__ __forceinline__ float ld(const __half *p) { return __half2float(*p); }
  static __device__ __forceinline__ void st(__half *p, float v) {
    *p = __float2half_rn(fminf(fmaxf(v, -65504.0f), 65504.0f));
  }
};

template <>
struct Store<int8_t> {
  static __device__ __forceinline__ float ld(const int8_t *p) { return (float)*p; }
  static __device__ __forceinline__ void st(int8_t *p, float v) {
    *p = (int8_t)fminf(fmaxf(rintf(v), -127.0f), 127.0f);
  }
};

// Value as it would be after a store to S (storage rounding / saturation);
// used for levels that stay in registers and for channel LLRs on entry.
template <typename S>
__device__ __forceinline__ float rnd(float v);
template <>
__device__ __forceinline__ float rnd<float>(float v) { return v; }
template <>
__device__ __forceinline__ float rnd<__half>(float v) {
  return __half2float(__float2half_rn(fminf(fmaxf(v, -65504.0f), 65504.0f)));
}
template <>
__device__ __forceinline__ float rnd<int8_t>(float v) {
  return fminf(fmaxf(rintf(v), -127.0f), 127.0f);
}

// f on stored values.  int8 values are L * s (s a per-frame power of two):
// min-sum commutes with that scale exactly; exact f is evaluated on L.
template <typename S, int FK>
__device__ __forceinline__ float f_st(float a, float b, float s) {
  if (FK == 0) return f_minsum(a, b);
  if (sizeof(S) == 1) return s * f_exact(a / s, b / s);
  return f_exact(a, b);
}

// f on values that may carry a per-frame scale s (int8 storage: values are
// L * s; s = 1 otherwise): min-sum commutes with the scale, exact f is taken
// on L.  With s = 1 both are bit-identical to f_op (a / 1 and 1 * x are exact,
// so that case skips the divisions: s is uniform across the frame).
template <int FK>
__device__ __forceinline__ float f_scaled(float a, float b, float s) {
  if (FK == 0) return f_minsum(a, b);
  if (s == 1.0f) return f_exact(a, b);
  return s * f_exact(a / s, b / s);
}

// ---------------------------------------------------------------- bits
// x = u F^{(x)k} on the low 2^k bits of a word (k <= 5): for h = 1, 2, ...,
// the low half of every block of 2h bits is XORed with its high half.
__device__ __forceinline__ uint32_t encode_word(uint32_t w, int k) {
  if (k > 0) w ^= (w >> 1) & 0x55555555u;
  if (k > 1) w ^= (w >> 2) & 0x33333333u;
  if (k > 2) w ^= (w >> 4) & 0x0F0F0F0Fu;
  if (k > 3) w ^= (w >> 8) & 0x00FF00FFu;
  if (k > 4) w ^= (w >> 16) & 0x0000FFFFu;
  return w;
}

__device__ __forceinline__ uint32_t low_mask(int nbits) {
  return nbits >= 32 ? 0xFFFFFFFFu : ((1u << nbits) - 1u);
}

// Partial sums live in place in x_hat: a node of 2^k leaves at leaf o keeps
// its beta in bits [o, o + 2^k).  When a unit of 2^ku leaves at ou finishes as
// a right child for r levels, each parent (left half ^= right half) is formed
// in turn by the calling CTA, levels in order (ku >= 5: whole words).
__device__ __forceinline__ void cascade_device(uint32_t *x, int ku, uint64_t ou, int r) {
  for (int m = 0; m < r; ++m) {
    int L = ku + m;
    uint64_t base = (ou >> (L + 1)) << (L + 1);
    uint64_t hw = (uint64_t(1) << L) >> 5;
    uint32_t *left = x + (base >> 5);
    for (uint64_t b = threadIdx.x; b < hw; b += (uint64_t)blockDim.x * 8) {
      uint32_t a[8], c[8];                       // eight loads in flight per thread
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint64_t i = b + (uint64_t)q * blockDim.x;
        if (i < hw) {
          a[q] = left[i];
          c[q] = left[hw + i];
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint64_t i = b + (uint64_t)q * blockDim.x;
        if (i < hw) left[i] = a[q] ^ c[q];
      }
    }
    __syncthreads();
  }
}

}  // namespace polar
