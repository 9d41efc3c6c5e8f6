// Frozen-set construction on the GPU in double precision (Sec. 3: the frozen
// bits are the least reliable bit-channels; K from a rate, or the largest K
// whose most reliable bit-channels have a summed error probability within a
// budget).  The same reliability measures as the host construction:
//   BSC     Bhattacharyya recursion  ln Z- = ln Z + ln(2 - Z),  ln Z+ = 2 ln Z;
//   BIAWGN  Gaussian approximation of density evolution (Chung, Richardson,
//           Urbanke 2001, with the small-x piece of Ha, Kim and McLaughlin
//           2004): m+ = 2m, m- = phi^-1(1 - (1 - phi(m))^2), P_e = Q(sqrt(m/2)).
// Each level of the polarisation doubles the array in one launch (children
// 2j <- minus, 2j+1 <- plus, so the first step sets the most significant
// index bit).  The channels are then ranked by a stable least-significant-
// digit radix sort of (reliability, index) -- fed in descending index order,
// so that equal reliabilities leave the higher index more reliable and the
// lower index is frozen first, the host's tie rule -- and the first K of the
// ranking are the information set.  Sec. 3's sum rule takes a fixed-order
// prefix sum of P_e along the ranking.
//
// The device's exp / log / pow round differently from the host's in the last
// bit, so a reliability within rounding of the K-th one may fall on the other
// side of the cut than on the host; everything else is identical.
#include <cmath>
#include <cstdio>
#include <vector>

#include "polar_internal.h"

namespace polar {

namespace {

// ------------------------------------------------------------ reliabilities
__device__ __forceinline__ double bh_minus(double l) { return l + log1p(-expm1(l)); }

__device__ double ga_lnphi_d(double x) {
  if (x < 0.867) return 0.0564 * x * x - 0.48560 * x;
  if (x < 10.0) return -0.4527 * pow(x, 0.86) + 0.0218;
  return 0.5 * log(3.141592653589793 / x) - 0.25 * x + log1p(-10.0 / (7.0 * x));
}

// Inverse of ln phi on the piece whose range holds t (the lowest such piece:
// the pieces are decreasing and do not meet at x = 10); on the x >= 10 piece
// Newton steps inside a shrinking bracket.
__device__ double ga_lnphi_inv_d(double t) {
  const double q867 = 0.0564 * 0.867 * 0.867 - 0.48560 * 0.867;
  if (t > q867) {
    if (t >= 0.0) return 0.0;
    return -2.0 * t / (0.48560 + sqrt(0.48560 * 0.48560 + 4.0 * 0.0564 * t));
  }
  const double left10 = -0.4527 * pow(10.0, 0.86) + 0.0218;
  if (t > left10) {
    const double v = (0.0218 - t) / 0.4527;
    return v > 0.0 ? pow(v, 1.0 / 0.86) : 0.0;
  }
  double lo = 10.0, hi = fmax(20.0, -8.0 * t);
  for (int i = 0; i < 64 && ga_lnphi_d(hi) > t; ++i) hi *= 2.0;
  double x = fmin(fmax(-4.0 * t, lo), hi);
  for (int it = 0; it < 100; ++it) {
    const double fx = ga_lnphi_d(x) - t;
    if (fx > 0.0) lo = x;
    else hi = x;
    const double a = 10.0 / (7.0 * x);
    const double d = -0.5 / x - 0.25 + (a / x) / (1.0 - a);
    double nx = x - fx / d;
    if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
    if (nx == x || hi - lo <= 1e-15 * hi) break;
    x = nx;
  }
  // the first double from x upwards with ln phi <= t (x is within a few ulp)
  for (int i = 0; i < 256 && ga_lnphi_d(x) > t; ++i) x = nextafter(x, hi + 1.0);
  return x;
}

__device__ __forceinline__ double ga_minus(double m) {
  const double lp = ga_lnphi_d(m);
  return ga_lnphi_inv_d(lp + log1p(-expm1(lp)));   // ln(phi (2 - phi))
}

// ln Q(x), x >= 0: Q(x) = erfcx(x / sqrt 2) e^{-x^2/2} / 2, no underflow.
__device__ __forceinline__ double ln_q_d(double x) {
  return log(0.5 * erfcx(x * 0.70710678118654752)) - 0.5 * x * x;
}

// One polarisation level: out[2j] = minus(in[j]), out[2j+1] = plus(in[j]).
__global__ void k_polarise(const double *__restrict__ in, double *__restrict__ out, uint64_t len,
                           int ga) {
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < len;
       j += (uint64_t)gridDim.x * blockDim.x) {
    const double v = in[j];
    out[2 * j] = ga ? ga_minus(v) : bh_minus(v);
    out[2 * j + 1] = 2.0 * v;
  }
}

// Ranking keys: ascending 64-bit key = ascending unreliability ln P_e (GA:
// ln Q(sqrt(m/2)); BSC: ln Z), element e holding index N-1-e.
__global__ void k_keys(const double *__restrict__ v, uint64_t n, int ga,
                       unsigned long long *__restrict__ key, uint32_t *__restrict__ val) {
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = n - 1 - e;
    double b = ga ? ln_q_d(sqrt(v[i] * 0.5)) : v[i];
    if (b == 0.0) b = 0.0;                         // one zero
    const unsigned long long u = (unsigned long long)__double_as_longlong(b);
    key[e] = (u >> 63) ? ~u : (u | 0x8000000000000000ull);
    val[e] = (uint32_t)i;
  }
}

__device__ __forceinline__ double key_value(unsigned long long k) {
  const unsigned long long u = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double((long long)u);
}

// ------------------------------------------------------------ radix sort
// Stable LSD radix sort of (64-bit key, 32-bit value) pairs, 8 bits a pass.
// A block owns a tile of TILE consecutive elements; its 8 warps own
// consecutive sub-tiles of SUB elements, walked in chunks of 32, so ranks
// follow element order: (digit count of earlier blocks) + (earlier warps)
// + (earlier chunks of this warp) + (earlier lanes with the same digit).
constexpr int RW = 8;                 // warps per block
constexpr int RT = 32 * RW;
constexpr int SUB = 512;              // elements per warp
constexpr int TILE = RW * SUB;

__device__ __forceinline__ uint32_t digit_of(unsigned long long k, int shift) {
  return (uint32_t)(k >> shift) & 0xFFu;
}

__global__ void k_rhist(const unsigned long long *__restrict__ key, uint64_t n, int shift,
                        uint32_t *__restrict__ counts, uint32_t nblocks) {
  __shared__ uint32_t h[256];
  for (int d = threadIdx.x; d < 256; d += RT) h[d] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * TILE;
  for (uint32_t j = threadIdx.x; j < (uint32_t)TILE; j += RT) {
    const uint64_t e = base + j;
    if (e < n) atomicAdd(&h[digit_of(key[e], shift)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += RT) counts[(uint64_t)d * nblocks + blockIdx.x] = h[d];
}

// Exclusive scan of m counts in place, one block of 1024 threads: each
// thread a consecutive segment, then the segment sums.
__global__ void k_rscan(uint32_t *__restrict__ c, uint64_t m) {
  __shared__ uint32_t part[1024];
  const uint64_t per = (m + 1023) / 1024;
  const uint64_t a = threadIdx.x * per, b = a + per < m ? a + per : m;
  uint32_t s = 0;
  for (uint64_t i = a; i < b; ++i) s += c[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int i = 0; i < 1024; ++i) {
      const uint32_t v = part[i];
      part[i] = run;
      run += v;
    }
  }
  __syncthreads();
  uint32_t run = part[threadIdx.x];
  for (uint64_t i = a; i < b; ++i) {
    const uint32_t v = c[i];
    c[i] = run;
    run += v;
  }
}

__global__ void k_rscatter(const unsigned long long *__restrict__ key,
                           const uint32_t *__restrict__ val, uint64_t n, int shift,
                           const uint32_t *__restrict__ offs, uint32_t nblocks,
                           unsigned long long *__restrict__ okey, uint32_t *__restrict__ oval) {
  __shared__ uint32_t cnt[RW][256];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int d = lane; d < 256; d += 32) cnt[w][d] = 0;
  __syncwarp();
  const uint64_t base = (uint64_t)blockIdx.x * TILE + (uint64_t)w * SUB;
  const uint32_t lt = (1u << lane) - 1u;
  // digit counts of this warp's sub-tile
  for (int c = 0; c < SUB / 32; ++c) {
    const uint64_t e = base + 32 * c + lane;
    const bool ok = e < n;
    const uint32_t d = ok ? digit_of(key[e], shift) : 256u + lane;
    const uint32_t same = __match_any_sync(0xFFFFFFFFu, d);
    if (ok && (same & lt) == 0) cnt[w][d] += __popc(same);
    __syncwarp();
  }
  __syncthreads();
  // first position of each (warp, digit)
  for (int d = threadIdx.x; d < 256; d += RT) {
    uint32_t run = offs[(uint64_t)d * nblocks + blockIdx.x];
    for (int v = 0; v < RW; ++v) {
      const uint32_t x = cnt[v][d];
      cnt[v][d] = run;
      run += x;
    }
  }
  __syncthreads();
  for (int c = 0; c < SUB / 32; ++c) {
    const uint64_t e = base + 32 * c + lane;
    const bool ok = e < n;
    unsigned long long k = 0;
    uint32_t d = 256u + lane;
    if (ok) {
      k = key[e];
      d = digit_of(k, shift);
    }
    const uint32_t same = __match_any_sync(0xFFFFFFFFu, d);
    if (ok) {
      const uint32_t pos = cnt[w][d] + __popc(same & lt);
      okey[pos] = k;
      oval[pos] = val[e];
    }
    __syncwarp();
    if (ok && (same & lt) == 0) cnt[w][d] += __popc(same);
    __syncwarp();
  }
}

// ------------------------------------------------------------ selection
// Block sums (fixed order) of P_e along the ranking.
constexpr int ST = 256;
constexpr int SPER = 16;              // elements per thread

__device__ __forceinline__ double block_sum(double s, double *sh) {
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int h = ST / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void k_psum(const unsigned long long *__restrict__ key, uint64_t n,
                       double *__restrict__ bsum) {
  __shared__ double sh[ST];
  const uint64_t a = ((uint64_t)blockIdx.x * ST + threadIdx.x) * SPER;
  double s = 0.0;
  for (int q = 0; q < SPER; ++q)
    if (a + q < n) s += exp(key_value(key[a + q]));
  const double b = block_sum(s, sh);
  if (threadIdx.x == 0) bsum[blockIdx.x] = b;
}

// Count of ranks r whose prefix sum of P_e (ranks 0..r) stays within the
// budget; the prefix is monotone, so that count is Sec. 3's K.  Also the
// prefix at each block's end for sum_pe.
__global__ void k_pcount(const unsigned long long *__restrict__ key, uint64_t n,
                         const double *__restrict__ bsum, uint32_t nb, double budget,
                         unsigned long long *__restrict__ count) {
  __shared__ double sh[ST];
  __shared__ double s_off;
  if (threadIdx.x == 0) {
    double off = 0.0;
    for (uint32_t b = 0; b < blockIdx.x; ++b) off += bsum[b];
    s_off = off;
  }
  const uint64_t a = ((uint64_t)blockIdx.x * ST + threadIdx.x) * SPER;
  double pe[SPER];
  double s = 0.0;
  for (int q = 0; q < SPER; ++q) {
    pe[q] = a + q < n ? exp(key_value(key[a + q])) : 0.0;
    s += pe[q];
  }
  // exclusive prefix of the thread sums within the block (fixed order)
  sh[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double run = s_off;
    for (int i = 0; i < ST; ++i) {
      const double v = sh[i];
      sh[i] = run;
      run += v;
    }
  }
  __syncthreads();
  double run = sh[threadIdx.x];
  unsigned long long c = 0;
  for (int q = 0; q < SPER; ++q) {
    if (a + q >= n) break;
    run += pe[q];
    if (run <= budget) ++c;
  }
  if (c) atomicAdd(count, c);
  (void)nb;
}

// sum of P_e over ranks [0, K) in the same order (sum_pe of the set)
__global__ void k_psum_k(const unsigned long long *__restrict__ key, uint64_t k,
                         double *__restrict__ bsum) {
  __shared__ double sh[ST];
  const uint64_t a = ((uint64_t)blockIdx.x * ST + threadIdx.x) * SPER;
  double s = 0.0;
  for (int q = 0; q < SPER; ++q)
    if (a + q < k) s += exp(key_value(key[a + q]));
  const double b = block_sum(s, sh);
  if (threadIdx.x == 0) bsum[blockIdx.x] = b;
}

__global__ void k_mask_all(uint32_t *m, uint64_t words) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < words;
       i += (uint64_t)gridDim.x * blockDim.x)
    m[i] = 0xFFFFFFFFu;
}

// Information bits: the first K of the ranking.
__global__ void k_mask_info(const uint32_t *__restrict__ val, uint64_t k, uint32_t *m) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < k;
       r += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = val[r];
    atomicAnd(&m[i >> 5], ~(1u << (i & 31)));
  }
}

unsigned grid_for(uint64_t n, unsigned threads) {
  const uint64_t g = (n + threads - 1) / threads;
  return (unsigned)(g < 152 * 16 ? (g ? g : 1) : 152 * 16);
}

struct DevBuf {
  void *p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace

int build_frozen_set_device(uint32_t log2n, polar_channel ch, double param, double rate,
                            double sum_max, cudaStream_t s, polar_frozen_set **out) {
  NvtxRange nv("polar construct on the device");
  if (!out || log2n < 1 || log2n > 27) return POLAR_EINVAL;
  if (!(rate >= 0.0 && rate <= 1.0) || !(sum_max >= 0.0)) return POLAR_EINVAL;
  if (ch == POLAR_BSC) {
    if (!(param > 0.0 && param < 0.5)) return POLAR_EINVAL;
  } else if (ch == POLAR_BIAWGN) {
    if (!(param > 0.0 && std::isfinite(param))) return POLAR_EINVAL;
  } else {
    return POLAR_EINVAL;
  }
  const bool sum_rule = rate == 0.0;
  const int ga = ch == POLAR_BIAWGN;
  const uint64_t N = uint64_t(1) << log2n;
  const uint64_t W = N >= 32 ? N / 32 : 1;
  const uint32_t nblocks = (uint32_t)((N + TILE - 1) / TILE);
  const uint32_t nsb = (uint32_t)((N + (uint64_t)ST * SPER - 1) / ((uint64_t)ST * SPER));
  DevBuf lv[2], key[2], val[2], counts, bsum, cnt, mask;
  auto fail = [](cudaError_t e) {
    set_last_error(cudaGetErrorString(e));
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : POLAR_ECUDA;
  };
#define DCK(x)                                   \
  do {                                           \
    cudaError_t e_ = (x);                        \
    if (e_ != cudaSuccess) return fail(e_);      \
  } while (0)
  for (int b = 0; b < 2; ++b) {
    DCK(cudaMalloc(&lv[b].p, N * sizeof(double)));
    DCK(cudaMalloc(&key[b].p, N * sizeof(unsigned long long)));
    DCK(cudaMalloc(&val[b].p, N * sizeof(uint32_t)));
  }
  DCK(cudaMalloc(&counts.p, (size_t)256 * nblocks * sizeof(uint32_t)));
  DCK(cudaMalloc(&bsum.p, (size_t)nsb * sizeof(double)));
  DCK(cudaMalloc(&cnt.p, sizeof(unsigned long long)));
  DCK(cudaMalloc(&mask.p, W * sizeof(uint32_t)));
  // one-channel parameter, then n polarisation levels (ping-pong)
  const double v0 = ga ? 2.0 / param : std::log(2.0) + 0.5 * (std::log(param) + std::log1p(-param));
  DCK(cudaMemcpyAsync(lv[0].p, &v0, sizeof(double), cudaMemcpyHostToDevice, s));
  int cur = 0;
  for (uint32_t l = 0; l < log2n; ++l) {
    const uint64_t len = uint64_t(1) << l;
    k_polarise<<<grid_for(len, 256), 256, 0, s>>>(static_cast<double *>(lv[cur].p),
                                                 static_cast<double *>(lv[cur ^ 1].p), len, ga);
    DCK(cudaGetLastError());
    cur ^= 1;
  }
  k_keys<<<grid_for(N, 256), 256, 0, s>>>(static_cast<double *>(lv[cur].p), N, ga,
                                          static_cast<unsigned long long *>(key[0].p),
                                          static_cast<uint32_t *>(val[0].p));
  DCK(cudaGetLastError());
  // ranking: 8 passes of 8 bits
  int kb = 0;
  for (int shift = 0; shift < 64; shift += 8) {
    k_rhist<<<nblocks, RT, 0, s>>>(static_cast<unsigned long long *>(key[kb].p), N, shift,
                                   static_cast<uint32_t *>(counts.p), nblocks);
    DCK(cudaGetLastError());
    k_rscan<<<1, 1024, 0, s>>>(static_cast<uint32_t *>(counts.p), (uint64_t)256 * nblocks);
    DCK(cudaGetLastError());
    k_rscatter<<<nblocks, RT, 0, s>>>(
        static_cast<unsigned long long *>(key[kb].p), static_cast<uint32_t *>(val[kb].p), N,
        shift, static_cast<uint32_t *>(counts.p), nblocks,
        static_cast<unsigned long long *>(key[kb ^ 1].p), static_cast<uint32_t *>(val[kb ^ 1].p));
    DCK(cudaGetLastError());
    kb ^= 1;
  }
  const auto *rk = static_cast<unsigned long long *>(key[kb].p);
  const auto *rv = static_cast<uint32_t *>(val[kb].p);
  uint64_t K;
  if (sum_rule) {
    k_psum<<<nsb, ST, 0, s>>>(rk, N, static_cast<double *>(bsum.p));
    DCK(cudaGetLastError());
    DCK(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), s));
    k_pcount<<<nsb, ST, 0, s>>>(rk, N, static_cast<double *>(bsum.p), nsb, sum_max,
                                static_cast<unsigned long long *>(cnt.p));
    DCK(cudaGetLastError());
    unsigned long long kk = 0;
    DCK(cudaMemcpyAsync(&kk, cnt.p, sizeof kk, cudaMemcpyDeviceToHost, s));
    DCK(cudaStreamSynchronize(s));
    K = kk;
  } else {
    K = std::min<uint64_t>(N, (uint64_t)std::floor(rate * (double)N));
  }
  k_mask_all<<<grid_for(W, 256), 256, 0, s>>>(static_cast<uint32_t *>(mask.p), W);
  DCK(cudaGetLastError());
  if (K > 0) {
    k_mask_info<<<grid_for(K, 256), 256, 0, s>>>(rv, K, static_cast<uint32_t *>(mask.p));
    DCK(cudaGetLastError());
  }
  double sum_pe = 0.0;
  if (K > 0) {
    k_psum_k<<<nsb, ST, 0, s>>>(rk, K, static_cast<double *>(bsum.p));
    DCK(cudaGetLastError());
    std::vector<double> hs(nsb);
    DCK(cudaMemcpyAsync(hs.data(), bsum.p, nsb * sizeof(double), cudaMemcpyDeviceToHost, s));
    DCK(cudaStreamSynchronize(s));
    for (double v : hs) sum_pe += v;
  }
  std::vector<uint32_t> hm(W);
  DCK(cudaMemcpyAsync(hm.data(), mask.p, W * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  DCK(cudaStreamSynchronize(s));
#undef DCK
  if (N < 32) hm[0] &= (1u << N) - 1u;
  polar_frozen_set *fs = nullptr;
  int rc = frozen_set_from_mask(log2n, hm.data(), &fs);
  if (rc) return rc;
  fs->K = K;
  fs->sum_pe = sum_pe;
  // the device mask is already resident: keep it for the decodes
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    std::lock_guard<std::mutex> g(fs->mu);
    if (N >= 32 && !fs->dmask.count(dev)) {   // (below a word the host copy is masked)
      fs->dmask[dev] = static_cast<uint32_t *>(mask.p);
      mask.p = nullptr;
    }
  }
  cudaGetLastError();
  *out = fs;
  return POLAR_OK;
}

}  // namespace polar
