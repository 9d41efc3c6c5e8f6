// Streamed kernels: channel LLR map, the f and g of levels above the subtree
// size (long vectors through HBM), the transform on packed bits, and the
// partial-sum combines.  All are grid-stride, 128-bit where the data allows.
#include "device_common.cuh"
#include "polar_internal.h"

namespace polar {

static inline int grid_for(size_t work, int block, int max_blocks = 152 * 16) {
  size_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > (size_t)max_blocks) g = max_blocks;
  return (int)g;
}

// ---------------------------------------------------------------- LLR maps
// BSC (Sec. 1): L = y ? -c : c; one float4 per thread (4 bits of y).
__global__ void k_llr_bsc(const uint32_t *__restrict__ y, float4 *__restrict__ llr,
                          size_t n4, float c) {
  pdl_enter();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4;
       i += (size_t)gridDim.x * blockDim.x) {
    uint32_t b = (y[i >> 3] >> ((i & 7) * 4)) & 0xFu;
    float4 v;
    v.x = (b & 1u) ? -c : c;
    v.y = (b & 2u) ? -c : c;
    v.z = (b & 4u) ? -c : c;
    v.w = (b & 8u) ? -c : c;
    llr[i] = v;
  }
}

// BI-AWGN (Sec. 2.2): L = float(y * (2 / sigma^2)), product in double.
__global__ void k_llr_biawgn(const double2 *__restrict__ y, float2 *__restrict__ llr,
                             size_t n2, double s) {
  pdl_enter();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2;
       i += (size_t)gridDim.x * blockDim.x) {
    double2 v = y[i];
    llr[i] = make_float2((float)(v.x * s), (float)(v.y * s));
  }
}

__global__ void k_llr_biawgn_tail(const double *__restrict__ y, float *__restrict__ llr,
                                  size_t first, size_t n, double s) {
  pdl_enter();
  size_t i = first + blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) llr[i] = (float)(y[i] * s);
}

cudaError_t launch_llr_bsc(const uint32_t *y, float *llr, size_t n_total, float c,
                           cudaStream_t s) {
  size_t n4 = n_total / 4;
  return counted(launch_k(k_llr_bsc, grid_for(n4, 256), 256, 0, s, y,
                          reinterpret_cast<float4 *>(llr), n4, c), 1);
}

cudaError_t launch_llr_biawgn(const double *y, float *llr, size_t n_total, double scale,
                              cudaStream_t s) {
  size_t n2 = n_total / 2;
  cudaError_t e = cudaSuccess;
  if (n2) {
    e = launch_k(k_llr_biawgn, grid_for(n2, 256), 256, 0, s, reinterpret_cast<const double2 *>(y),
                 reinterpret_cast<float2 *>(llr), n2, scale);
  }
  if (e == cudaSuccess && (n_total & 1))
    e = launch_k(k_llr_biawgn_tail, 1, 32, 0, s, y, llr, n2 * 2, n_total, scale);
  return counted(e, (n2 ? 1 : 0) + (n_total & 1));
}

// ---------------------------------------------------------------- transform
// Region r of nregions covers words [base + r*stride, +nw) (nw = 2^(k-5)).
__global__ void k_encode_inword(uint32_t *__restrict__ w, size_t stride, size_t off,
                                size_t nw, int nregions, int k) {
  pdl_enter();
  size_t total = nw * (size_t)nregions;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    size_t r = i / nw, j = i - r * nw;
    uint32_t *p = w + r * stride + off + j;
    if (k >= 5) {
      *p = encode_word(*p, 5);
    } else {
      uint32_t m = low_mask(1 << k);
      uint32_t v = *p;
      *p = (v & ~m) | (encode_word(v & m, k) & m);
    }
  }
}

// Cross-word levels 0 .. lv-1 of blocks of 2^lv consecutive words, in shared
// memory (one block per CTA).  Block b of the region grid covers
// words [r*stride + off + b*2^lv, +2^lv).
__global__ void k_encode_xword_smem(uint32_t *__restrict__ w, size_t stride, size_t off,
                                    size_t nw, int nregions, int lv) {
  pdl_enter();
  extern __shared__ uint32_t sm[];
  const size_t bw = size_t(1) << lv;
  const size_t blocks_per_region = nw / bw;
  const size_t total = blocks_per_region * (size_t)nregions;
  for (size_t b = blockIdx.x; b < total; b += gridDim.x) {
    size_t r = b / blocks_per_region, bb = b - r * blocks_per_region;
    uint32_t *p = w + r * stride + off + bb * bw;
    for (size_t i = threadIdx.x; i < bw; i += blockDim.x) sm[i] = p[i];
    __syncthreads();
    for (size_t hw = 1; hw < bw; hw <<= 1) {
      for (size_t i = threadIdx.x; i < bw / 2; i += blockDim.x) {
        size_t a = ((i / hw) * 2 * hw) + (i % hw);
        sm[a] ^= sm[a + hw];
      }
      __syncthreads();
    }
    for (size_t i = threadIdx.x; i < bw; i += blockDim.x) p[i] = sm[i];
    __syncthreads();
  }
}

// One cross-word level: word a ^= word a + hw for a with bit hw clear.
__global__ void k_encode_xword_level(uint32_t *__restrict__ w, size_t stride, size_t off,
                                     size_t nw, int nregions, size_t hw) {
  pdl_enter();
  size_t half = nw / 2;
  size_t total = half * (size_t)nregions;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    size_t r = i / half, j = i - r * half;
    size_t a = ((j / hw) * 2 * hw) + (j % hw);
    uint32_t *p = w + r * stride + off;
    p[a] ^= p[a + hw];
  }
}

cudaError_t launch_encode_regions(uint32_t *words, size_t stride_w, size_t off_w, int log2len,
                                  int nframes, cudaStream_t s) {
  size_t nw = log2len >= 5 ? (size_t(1) << (log2len - 5)) : 1;
  uint64_t launched = 1;
  cudaError_t e = launch_k(k_encode_inword, grid_for(nw * nframes, 256), 256, 0, s, words,
                           stride_w, off_w, nw, nframes, log2len);
  if (e == cudaSuccess && nw > 1) {
    int lvw = log2len - 5;
    int lv = lvw < 12 ? lvw : 12;
    size_t bw = size_t(1) << lv;
    size_t nblocks = (nw / bw) * nframes;
    int grid = (int)(nblocks < 4096 ? nblocks : 4096);
    e = launch_k(k_encode_xword_smem, grid, 256, bw * sizeof(uint32_t), s, words, stride_w,
                 off_w, nw, nframes, lv);
    launched++;
    for (int l = lv; l < lvw && e == cudaSuccess; ++l) {
      size_t hw = size_t(1) << l;
      e = launch_k(k_encode_xword_level, grid_for(nw / 2 * nframes, 256), 256, 0, s, words,
                   stride_w, off_w, nw, nframes, hw);
      launched++;
    }
  }
  return counted(e, launched);
}

// dst[f][off + j] = src[f][off + j] (& and_mask[off + j] if given).
__global__ void k_copy_regions(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                               size_t stride, size_t off, size_t nw, int nregions,
                               const uint32_t *__restrict__ and_mask) {
  pdl_enter();
  size_t total = nw * (size_t)nregions;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    size_t r = i / nw, j = i - r * nw;
    uint32_t v = src[r * stride + off + j];
    if (and_mask) v &= and_mask[off + j];
    dst[r * stride + off + j] = v;
  }
}

cudaError_t launch_copy_regions(const uint32_t *src, uint32_t *dst, size_t stride_w,
                                size_t off_w, size_t nwords, int nframes,
                                const uint32_t *and_mask, cudaStream_t s) {
  return counted(launch_k(k_copy_regions, grid_for(nwords * nframes, 256), 256, 0, s, src, dst,
                          stride_w, off_w, nwords, nframes, and_mask), 1);
}

// ---------------------------------------------------------------- combine
// One CTA per frame; see cascade_device.
__global__ void k_cascade(uint32_t *__restrict__ xhat, size_t stride, int ku, uint64_t ou,
                          int r) {
  pdl_enter();
  cascade_device(xhat + blockIdx.x * stride, ku, ou, r);
}

cudaError_t launch_cascade(uint32_t *xhat, size_t stride_w, int k_unit, uint64_t o_unit, int r,
                           int nframes, cudaStream_t s) {
  if (r <= 0) return cudaSuccess;
  return counted(launch_k(k_cascade, nframes, 512, 0, s, xhat, stride_w, k_unit, o_unit, r), 1);
}

// ---------------------------------------------------------------- stream f / g
// Level k -> k-1 for every frame: out[j] = f(in[j], in[j+h]) or
// g(in[j], in[j+h], beta[o+j]), j < h.  grid.y = frame; each thread handles
// 4 consecutive j per step.  When the input is the float channel LLR array
// and the storage is not float, inputs are scaled (int8) and rounded on load.
template <typename Tin, typename Tout>
__device__ __forceinline__ float load_in(const Tin *p, float sc) {
  if constexpr (sizeof(Tin) == 4 && sizeof(Tout) != 4) return rnd<Tout>(*p * sc);
  return Store<Tin>::ld(p);
}

// Reduced storage: a thread moves 16 bytes of output per step (8 FP16 or 16
// INT8 values) and the matching 16 or 32..64 bytes of each input operand,
// with the per-value conversions, rounding and saturation of load_in / Store.
template <typename Tin, typename Tout>
struct Vec16 {
  static constexpr int N = 16 / sizeof(Tout);                    // values per step
  static constexpr int NIN = N * (int)sizeof(Tin) / 16;          // 16-byte loads per operand
  static __device__ __forceinline__ void load(const Tin *p, float (&v)[N], float sc) {
    uint4 q[NIN];
#pragma unroll
    for (int k = 0; k < NIN; ++k) q[k] = reinterpret_cast<const uint4 *>(p)[k];
    const Tin *e = reinterpret_cast<const Tin *>(q);
#pragma unroll
    for (int c = 0; c < N; ++c) v[c] = load_in<Tin, Tout>(e + c, sc);
  }
  static __device__ __forceinline__ void store(Tout *p, const float (&v)[N]) {
    uint4 q;
    Tout *e = reinterpret_cast<Tout *>(&q);
#pragma unroll
    for (int c = 0; c < N; ++c) Store<Tout>::st(e + c, v[c]);
    *reinterpret_cast<uint4 *>(p) = q;
  }
};

template <typename Tin, typename Tout, int FK>
__global__ void k_stream_f(const Tin *__restrict__ in, size_t in_stride, Tout *__restrict__ out,
                           size_t out_stride, uint64_t h, const float *__restrict__ scale) {
  pdl_enter();
  const Tin *a = in + blockIdx.y * in_stride;
  const Tin *b = a + h;
  Tout *o = out + blockIdx.y * out_stride;
  const float sc = scale ? scale[blockIdx.y] : 1.0f;
  using V = Vec16<Tin, Tout>;
  const uint64_t hv = h / V::N;                   // h is a power of two >= 32
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < hv;
       i += (uint64_t)gridDim.x * blockDim.x) {
    if constexpr (sizeof(Tin) == 4 && sizeof(Tout) == 4) {
      float4 x = reinterpret_cast<const float4 *>(a)[i];
      float4 y = reinterpret_cast<const float4 *>(b)[i];
      float4 z;
      z.x = f_op<FK>(x.x, y.x);
      z.y = f_op<FK>(x.y, y.y);
      z.z = f_op<FK>(x.z, y.z);
      z.w = f_op<FK>(x.w, y.w);
      reinterpret_cast<float4 *>(o)[i] = z;
    } else {
      float x[V::N], y[V::N];
      V::load(a + i * V::N, x, sc);
      V::load(b + i * V::N, y, sc);
#pragma unroll
      for (int c = 0; c < V::N; ++c) x[c] = f_st<Tout, FK>(x[c], y[c], sc);
      V::store(o + i * V::N, x);
    }
  }
}

template <typename Tin, typename Tout>
__global__ void k_stream_g(const Tin *__restrict__ in, size_t in_stride, Tout *__restrict__ out,
                           size_t out_stride, uint64_t h, const uint32_t *__restrict__ xhat,
                           size_t x_stride, uint64_t o_bits, const float *__restrict__ scale) {
  pdl_enter();
  const Tin *a = in + blockIdx.y * in_stride;
  const Tin *b = a + h;
  Tout *o = out + blockIdx.y * out_stride;
  const uint32_t *beta = xhat + blockIdx.y * x_stride + (o_bits >> 5);
  const float sc = scale ? scale[blockIdx.y] : 1.0f;
  using V = Vec16<Tin, Tout>;
  const uint64_t hv = h / V::N;                   // h is a power of two >= 32
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < hv;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t e0 = i * V::N;                 // first value of this step
    const uint32_t bits = (beta[e0 >> 5] >> (e0 & 31)) & ((1u << V::N) - 1u);
    if constexpr (sizeof(Tin) == 4 && sizeof(Tout) == 4) {
      float4 x = reinterpret_cast<const float4 *>(a)[i];
      float4 y = reinterpret_cast<const float4 *>(b)[i];
      float4 z;
      z.x = g_op(x.x, y.x, bits & 1u);
      z.y = g_op(x.y, y.y, bits & 2u);
      z.z = g_op(x.z, y.z, bits & 4u);
      z.w = g_op(x.w, y.w, bits & 8u);
      reinterpret_cast<float4 *>(o)[i] = z;
    } else {
      float x[V::N], y[V::N];
      V::load(a + e0, x, sc);
      V::load(b + e0, y, sc);
#pragma unroll
      for (int c = 0; c < V::N; ++c) x[c] = g_op(x[c], y[c], (bits >> c) & 1u);
      V::store(o + e0, x);
    }
  }
}

// units = thread steps per frame (h / Vec16<., T>::N values each).
static dim3 stream_grid(uint64_t units, int nframes) {
  uint64_t want = (units + 255) / 256;
  uint64_t cap = (uint64_t)(152 * 8 + nframes - 1) / nframes;   // ~8 CTAs/SM overall
  if (cap < 1) cap = 1;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return dim3((unsigned)want, (unsigned)nframes);
}

template <typename T>
static cudaError_t stream_f_t(int fkind, const void *in, size_t in_stride, bool in_is_llr,
                              void *out, size_t out_stride, uint64_t h, int nframes,
                              const float *scale, cudaStream_t s) {
  dim3 g = stream_grid(h / (16 / sizeof(T)), nframes);
  cudaError_t e;
  if (in_is_llr) {
    e = fkind == 0 ? launch_k(k_stream_f<float, T, 0>, g, 256, 0, s, (const float *)in,
                              in_stride, (T *)out, out_stride, h, scale)
                   : launch_k(k_stream_f<float, T, 1>, g, 256, 0, s, (const float *)in,
                              in_stride, (T *)out, out_stride, h, scale);
  } else {
    e = fkind == 0 ? launch_k(k_stream_f<T, T, 0>, g, 256, 0, s, (const T *)in, in_stride,
                              (T *)out, out_stride, h, scale)
                   : launch_k(k_stream_f<T, T, 1>, g, 256, 0, s, (const T *)in, in_stride,
                              (T *)out, out_stride, h, scale);
  }
  return counted(e, 1);
}

template <typename T>
static cudaError_t stream_g_t(const void *in, size_t in_stride, bool in_is_llr, void *out,
                              size_t out_stride, uint64_t h, const uint32_t *xhat,
                              size_t xs, uint64_t o, int nframes, const float *scale,
                              cudaStream_t s) {
  dim3 g = stream_grid(h / (16 / sizeof(T)), nframes);
  cudaError_t e =
      in_is_llr ? launch_k(k_stream_g<float, T>, g, 256, 0, s, (const float *)in, in_stride,
                           (T *)out, out_stride, h, xhat, xs, o, scale)
                : launch_k(k_stream_g<T, T>, g, 256, 0, s, (const T *)in, in_stride, (T *)out,
                           out_stride, h, xhat, xs, o, scale);
  return counted(e, 1);
}

// ---------------------------------------------------------------- fused chains
// One launch for a run of the recursion's streamed steps: level kt -> kt-1 by
// f (left child) or g (right child, partial sums of the left sibling read
// from x_hat), then f down to level kb.  The work is split in columns: column
// c of a frame holds, at every level k in kb..kt, the elements whose index
// modulo 2^kb lies in [c*B, c*B + B); f and g pair index j with j + 2^(k-1),
// which stays inside the column, so a CTA runs all levels of its column in
// shared memory and writes each level once (no re-reads, one launch).
// Stored values are rounded to Tout before the next level uses them.
// Four consecutive values of a storage type, widened to / narrowed from float.
template <typename T>
struct Quad;
template <>
struct Quad<float> {
  static __device__ __forceinline__ float4 ld(const float *p) {
    return *reinterpret_cast<const float4 *>(p);
  }
  static __device__ __forceinline__ void st(float *p, float4 v) {
    *reinterpret_cast<float4 *>(p) = v;
  }
};
template <>
struct Quad<__half> {
  static __device__ __forceinline__ float4 ld(const __half *p) {
    const uint2 u = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
  }
  static __device__ __forceinline__ void st(__half *p, float4 v) {   // v already rounded
    __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t *>(&a);
    u.y = *reinterpret_cast<uint32_t *>(&b);
    *reinterpret_cast<uint2 *>(p) = u;
  }
};
template <>
struct Quad<int8_t> {
  static __device__ __forceinline__ float4 ld(const int8_t *p) {
    const char4 c = *reinterpret_cast<const char4 *>(p);
    return make_float4((float)c.x, (float)c.y, (float)c.z, (float)c.w);
  }
  static __device__ __forceinline__ void st(int8_t *p, float4 v) {   // v already rounded
    *reinterpret_cast<char4 *>(p) =
        make_char4((signed char)v.x, (signed char)v.y, (signed char)v.z, (signed char)v.w);
  }
};

template <typename Tin, typename Tout>
__device__ __forceinline__ float4 load4_in(const Tin *p, float sc) {
  float4 v = Quad<Tin>::ld(p);
  if constexpr (sizeof(Tin) == 4 && sizeof(Tout) != 4) {
    v.x = rnd<Tout>(v.x * sc);
    v.y = rnd<Tout>(v.y * sc);
    v.z = rnd<Tout>(v.z * sc);
    v.w = rnd<Tout>(v.w * sc);
  }
  return v;
}

// One launch for a run of the recursion's streamed steps: level kt -> kt-1 by
// f (left child) or g (right child, partial sums of the left sibling read
// from x_hat), then f down to level kb.  The work is split in columns: column
// c of a frame holds, at every level k in kb..kt, the elements whose index
// modulo 2^kb lies in [c*B, c*B + B); f and g pair index j with j + 2^(k-1),
// which stays inside the column, so a CTA runs all levels of its column in
// shared memory and writes each level once (no re-reads, one launch).
// Threads work on four consecutive elements; stored values are rounded to
// Tout before the next level uses them.
template <typename Tin, typename Tout, int FK, bool FIRST_G>
__global__ void __launch_bounds__(256) k_chain(const Tin *__restrict__ in, size_t in_stride,
                                               Tout *__restrict__ lv_base, int t, int nframes,
                                               int kt, int kb, int logB,
                                               const uint32_t *__restrict__ xhat,
                                               size_t x_stride, uint64_t o_left,
                                               const float *__restrict__ scale) {
  pdl_enter();
  extern __shared__ float4 cs4[];
  const int cols = 1 << (kb - logB);
  const int f = blockIdx.x >> (kb - logB), c = blockIdx.x & (cols - 1);
  const float sc = scale ? scale[f] : 1.0f;
  const Tin *src = in + (size_t)f * in_stride;
  const uint32_t qB = (1u << logB) >> 2;                  // quads per row
  const int lq = logB - 2;
  const uint32_t nin = qB << (kt - kb);
  const uint64_t col0 = (uint64_t)c << logB;
  for (uint32_t b = threadIdx.x; b < nin; b += blockDim.x * 4) {
    float4 q[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const uint32_t e = b + r * blockDim.x;
      if (e < nin) {
        const uint64_t j = ((uint64_t)(e >> lq) << kb) + col0 + ((e & (qB - 1)) << 2);
        q[r] = load4_in<Tin, Tout>(src + j, sc);
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const uint32_t e = b + r * blockDim.x;
      if (e < nin) cs4[e] = q[r];
    }
  }
  __syncthreads();
  const uint32_t *beta = FIRST_G ? xhat + (size_t)f * x_stride : nullptr;
  for (int k = kt; k > kb; --k) {
    const uint32_t half = qB << (k - 1 - kb);             // quads of level k-1
    Tout *dst = lv_base + (size_t)nframes * ((size_t(1) << (k - 1)) - (size_t(1) << t)) +
                (size_t)f * (size_t(1) << (k - 1));
    for (uint32_t e = threadIdx.x; e < half; e += blockDim.x) {
      const float4 a = cs4[e], bq = cs4[e + half];
      const uint64_t j = ((uint64_t)(e >> lq) << kb) + col0 + ((e & (qB - 1)) << 2);
      float4 v;
      if (FIRST_G && k == kt) {
        const uint64_t pos = o_left + j;
        const uint32_t bits = (beta[pos >> 5] >> (pos & 31)) & 0xFu;
        v.x = g_op(a.x, bq.x, bits & 1u);
        v.y = g_op(a.y, bq.y, bits & 2u);
        v.z = g_op(a.z, bq.z, bits & 4u);
        v.w = g_op(a.w, bq.w, bits & 8u);
      } else {
        v.x = f_st<Tout, FK>(a.x, bq.x, sc);
        v.y = f_st<Tout, FK>(a.y, bq.y, sc);
        v.z = f_st<Tout, FK>(a.z, bq.z, sc);
        v.w = f_st<Tout, FK>(a.w, bq.w, sc);
      }
      v.x = rnd<Tout>(v.x);
      v.y = rnd<Tout>(v.y);
      v.z = rnd<Tout>(v.z);
      v.w = rnd<Tout>(v.w);
      Quad<Tout>::st(dst + j, v);
      cs4[e] = v;                      // in place: quad e is read by this thread only
    }
    __syncthreads();
  }
}

template <typename T, int FK, bool G>
static cudaError_t chain_t(const void *in, size_t in_stride, bool in_is_llr, void *lv_base, int t,
                           int nframes, int kt, int kb, const uint32_t *xhat, size_t xs,
                           uint64_t o, const float *scale, cudaStream_t s) {
  // Row width 2^logB: about a thousand CTAs over the batch, at most 64 KB of
  // float column per CTA, at least 32 elements per row.
  int want = 0;
  while ((nframes << want) < 1024) ++want;                  // columns per frame, log2
  int logB = kb - want;
  if (logB > 14 - (kt - kb)) logB = 14 - (kt - kb);
  if (logB < 5) logB = 5;
  if (logB > kb) logB = kb;
  const size_t smem = (size_t(1) << (logB + kt - kb)) * sizeof(float);
  const unsigned grid = (unsigned)nframes << (kb - logB);
  cudaError_t e;
  if (in_is_llr) {
    auto kern = k_chain<float, T, FK, G>;
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    e = launch_k(kern, grid, 256, smem, s, (const float *)in, in_stride, (T *)lv_base, t,
                 nframes, kt, kb, logB, xhat, xs, o, scale);
  } else {
    auto kern = k_chain<T, T, FK, G>;
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    e = launch_k(kern, grid, 256, smem, s, (const T *)in, in_stride, (T *)lv_base, t, nframes,
                 kt, kb, logB, xhat, xs, o, scale);
  }
  return counted(e, 1);
}

template <typename T>
static cudaError_t chain_p(int fkind, bool first_g, const void *in, size_t in_stride,
                           bool in_is_llr, void *lv_base, int t, int nframes, int kt, int kb,
                           const uint32_t *xhat, size_t xs, uint64_t o, const float *scale,
                           cudaStream_t s) {
  if (fkind == 0)
    return first_g ? chain_t<T, 0, true>(in, in_stride, in_is_llr, lv_base, t, nframes, kt, kb,
                                         xhat, xs, o, scale, s)
                   : chain_t<T, 0, false>(in, in_stride, in_is_llr, lv_base, t, nframes, kt, kb,
                                          xhat, xs, o, scale, s);
  return first_g ? chain_t<T, 1, true>(in, in_stride, in_is_llr, lv_base, t, nframes, kt, kb,
                                       xhat, xs, o, scale, s)
                 : chain_t<T, 1, false>(in, in_stride, in_is_llr, lv_base, t, nframes, kt, kb,
                                        xhat, xs, o, scale, s);
}

cudaError_t launch_chain(int prec, int fkind, bool first_g, const void *in, size_t in_stride,
                         bool in_is_llr, void *lv_base, int t, int nframes, int kt, int kb,
                         const uint32_t *xhat, size_t xhat_stride_w, uint64_t o_left,
                         const float *scale, cudaStream_t s) {
  if (prec == POLAR_FP16)
    return chain_p<__half>(fkind, first_g, in, in_stride, in_is_llr, lv_base, t, nframes, kt, kb,
                           xhat, xhat_stride_w, o_left, scale, s);
  if (prec == POLAR_INT8)
    return chain_p<int8_t>(fkind, first_g, in, in_stride, in_is_llr, lv_base, t, nframes, kt,
                           kb, xhat, xhat_stride_w, o_left, scale, s);
  return chain_p<float>(fkind, first_g, in, in_stride, in_is_llr, lv_base, t, nframes, kt, kb,
                        xhat, xhat_stride_w, o_left, scale, s);
}

// ---------------------------------------------------------------- int8 scale
// One CTA per frame: mean |L| in double (fixed reduction tree), then
// s = 2^rint(log2(target / mean)), clamped to 2^+-100; s = 1 if every L = 0.
__global__ void k_int8_scale(const float *__restrict__ llr, size_t n, double target,
                             float *__restrict__ scale) {
  pdl_enter();
  __shared__ double part[256];
  const float *p = llr + blockIdx.x * n;
  double acc = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) acc += fabs((double)p[i]);
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double tot = part[0];
    float sc = 1.0f;
    if (tot > 0.0) {
      double e = rint(log2(target / (tot / (double)n)));
      e = fmin(fmax(e, -100.0), 100.0);
      sc = (float)ldexp(1.0, (int)e);
    }
    scale[blockIdx.x] = sc;
  }
}

cudaError_t launch_int8_scale(const float *llr, size_t n, int nframes, double target,
                              float *scale, cudaStream_t s) {
  return counted(launch_k(k_int8_scale, nframes, 256, 0, s, llr, n, target, scale), 1);
}

// ---------------------------------------------------------------- verification
// Keyed linear hash of a frame's packed bits, for the verification step that
// discards wrongly decoded blocks (Sec. 2.1): h = sum_i w_i c_i mod p,
// p = 2^61 - 1, w_i the frame's 32-bit words, c_i the SplitMix64 output for
// (key, i) reduced mod p.  Two different frames collide with probability
// 1/p when the coefficients are uniform.  One CTA per frame.
constexpr uint64_t kHashP = (uint64_t(1) << 61) - 1;

__device__ __forceinline__ uint64_t hash_coef(uint64_t key, uint64_t i) {
  uint64_t z = key + (i + 1) * 0x9E3779B97F4A7C15ull;      // SplitMix64 step i
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  z = (z & kHashP) + (z >> 61);
  return z >= kHashP ? z - kHashP : z;
}

__device__ __forceinline__ uint64_t hash_mulmod(uint64_t w, uint64_t c) {   // w < 2^32, c < p
  const uint64_t lo = w * c, hi = __umul64hi(w, c);
  uint64_t r = (lo & kHashP) + ((hi << 3) | (lo >> 61));
  return r >= kHashP ? r - kHashP : r;
}

__device__ __forceinline__ uint64_t hash_addmod(uint64_t a, uint64_t b) {
  const uint64_t r = a + b;
  return r >= kHashP ? r - kHashP : r;
}

__global__ void k_frame_hash(const uint32_t *__restrict__ words, size_t stride, size_t nw,
                             uint64_t key, uint64_t *__restrict__ out) {
  __shared__ uint64_t part[256];
  const uint32_t *w = words + blockIdx.x * stride;
  uint64_t acc = 0;
  for (size_t i = threadIdx.x; i < nw; i += blockDim.x)
    acc = hash_addmod(acc, hash_mulmod(w[i], hash_coef(key, i)));
  part[threadIdx.x] = acc;
  __syncthreads();
  for (unsigned h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) part[threadIdx.x] = hash_addmod(part[threadIdx.x], part[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = part[0];
}

cudaError_t launch_frame_hash(const uint32_t *words, size_t stride_w, size_t nwords,
                              int nframes, uint64_t key, uint64_t *out, cudaStream_t s) {
  k_frame_hash<<<nframes, 256, 0, s>>>(words, stride_w, nwords, key, out);
  return counted(cudaGetLastError(), 1);
}

std::atomic<uint64_t> g_kernel_launches{0};
std::atomic<int> g_pdl{0};

size_t storage_bytes(int prec) { return prec == POLAR_FP32 ? 4 : (prec == POLAR_FP16 ? 2 : 1); }

cudaError_t launch_stream_f(int prec, int fkind, const void *in, size_t in_stride,
                            bool in_is_llr, void *out, size_t out_stride, uint64_t h,
                            int nframes, const float *scale, cudaStream_t s) {
  if (prec == POLAR_FP16)
    return stream_f_t<__half>(fkind, in, in_stride, in_is_llr, out, out_stride, h, nframes,
                              scale, s);
  if (prec == POLAR_INT8)
    return stream_f_t<int8_t>(fkind, in, in_stride, in_is_llr, out, out_stride, h, nframes,
                              scale, s);
  return stream_f_t<float>(fkind, in, in_stride, in_is_llr, out, out_stride, h, nframes, scale,
                           s);
}

cudaError_t launch_stream_g(int prec, const void *in, size_t in_stride, bool in_is_llr,
                            void *out, size_t out_stride, uint64_t h, const uint32_t *xhat,
                            size_t xhat_stride_w, uint64_t o, int nframes, const float *scale,
                            cudaStream_t s) {
  if (prec == POLAR_FP16)
    return stream_g_t<__half>(in, in_stride, in_is_llr, out, out_stride, h, xhat, xhat_stride_w,
                              o, nframes, scale, s);
  if (prec == POLAR_INT8)
    return stream_g_t<int8_t>(in, in_stride, in_is_llr, out, out_stride, h, xhat, xhat_stride_w,
                              o, nframes, scale, s);
  return stream_g_t<float>(in, in_stride, in_is_llr, out, out_stride, h, xhat, xhat_stride_w, o,
                           nframes, scale, s);
}

}  // namespace polar
