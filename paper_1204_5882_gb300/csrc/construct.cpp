// Frozen-set construction on the host (Sec. 3: the frozen bits are the
// bit-channels of lowest capacity found by density evolution; equal
// reliabilities freeze the lower index first).
//
// Reliability measures, in double precision and in the log domain so that
// nothing underflows up to N = 2^27:
//   BSC     Bhattacharyya recursion  ln Z- = ln Z + ln(2 - Z),  ln Z+ = 2 ln Z,
//           ln Z0 = ln 2 + (ln p + ln(1 - p)) / 2;
//   BIAWGN  Gaussian approximation of density evolution (Chung, Richardson,
//           Urbanke 2001): m0 = 2 / sigma^2, m+ = 2 m,
//           m- = phi^-1(1 - (1 - phi(m))^2),  P_e = Q(sqrt(m / 2)).
// The first polarisation step sets the most significant index bit, which is
// the top split of the natural-order decoder.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>

#include "polar_internal.h"

namespace polar {

static std::atomic<uint64_t> g_fs_ids{1};

// ---------------------------------------------------------------- BSC
static inline double bh_step(double lz, bool plus) {
  if (plus) return 2.0 * lz;
  return lz + std::log1p(-std::expm1(lz));   // ln(2Z - Z^2)
}

// ---------------------------------------------------------------- GA
// ln phi_GA(x): Chung-Richardson-Urbanke phi completed by a small-x piece
// so that phi(0) = 1 (without it the minus step has a fixed point at
// m = 0.029 and long codes get "minus^k plus^j" channels rated reliable):
//   exp(0.0564 x^2 - 0.48560 x) below 0.867, exp(-0.4527 x^0.86 + 0.0218)
//   below 10, sqrt(pi/x) e^{-x/4} (1 - 10/(7x)) from 10 on.
static inline double ga_lnphi(double x) {
  if (x < 0.867) return 0.0564 * x * x - 0.48560 * x;
  if (x < 10.0) return -0.4527 * std::pow(x, 0.86) + 0.0218;
  return 0.5 * std::log(M_PI / x) - 0.25 * x + std::log1p(-10.0 / (7.0 * x));
}

// d/dx ln phi_GA on the x >= 10 piece.
static inline double ga_dlnphi_hi(double x) {
  double a = 10.0 / (7.0 * x);
  return -0.5 / x - 0.25 + (a / x) / (1.0 - a);
}

// Inverse of ln phi_GA.  The pieces are decreasing; at x = 10 they do not
// meet (ln phi jumps up from -3.2576 to -3.2331), so targets in that gap have
// two preimages.  The lowest piece whose range holds the target is used: the
// quadratic piece (its smaller root, -2t / (b + sqrt(b^2 + 4at))) above its
// value at 0.867, then the middle piece in closed form above its limit at
// 10; on the x >= 10 piece the result is the smallest double x with
// ln phi(x) <= t, found by Newton steps from x ~ -4t and finished by ulp steps.
static double ga_lnphi_inv(double t) {
  const double q867 = 0.0564 * 0.867 * 0.867 - 0.48560 * 0.867;
  if (t > q867) {
    if (t >= 0.0) return 0.0;
    return -2.0 * t / (0.48560 + std::sqrt(0.48560 * 0.48560 + 4.0 * 0.0564 * t));
  }
  const double left10 = -0.4527 * std::pow(10.0, 0.86) + 0.0218;
  if (t > left10) {
    double v = (0.0218 - t) / 0.4527;
    return v > 0.0 ? std::pow(v, 1.0 / 0.86) : 0.0;
  }
  double lo = 10.0, hi = std::max(20.0, -8.0 * t);
  while (ga_lnphi(hi) > t) hi *= 2.0;
  double x = std::min(std::max(-4.0 * t, lo), hi);
  for (int it = 0; it < 100; ++it) {
    double fx = ga_lnphi(x) - t;
    if (fx > 0) lo = x; else hi = x;
    double nx = x - fx / ga_dlnphi_hi(x);
    if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
    if (nx == x) break;
    x = nx;
    if (hi - lo <= 4.0 * std::nextafter(hi, INFINITY) - 4.0 * hi) break;
  }
  // smallest double with ln phi(x) <= t
  while (ga_lnphi(x) > t) x = std::nextafter(x, INFINITY);
  for (;;) {
    double p = std::nextafter(x, 0.0);
    if (p < 10.0 || ga_lnphi(p) > t) break;
    x = p;
  }
  return x;
}

static inline double ga_step(double m, bool plus) {
  if (plus) return 2.0 * m;
  double lp = ga_lnphi(m);
  return ga_lnphi_inv(lp + std::log1p(-std::expm1(lp)));   // ln(phi (2 - phi))
}

// ln Q(x), x >= 0.
static inline double ln_q(double x) {
  if (x < 30.0) return std::log(0.5 * std::erfc(x / M_SQRT2));
  double x2 = x * x;
  double s = 1.0 - 1.0 / x2 + 3.0 / (x2 * x2) - 15.0 / (x2 * x2 * x2);
  return -0.5 * x2 - std::log(x) - 0.5 * std::log(2.0 * M_PI) + std::log(s);
}

// Expand the one-channel parameter into 2^n bit-channel parameters, level by
// level, in place from the top down (children 2j <- minus, 2j+1 <- plus).
template <class Step>
static void polarise(std::vector<double> &v, uint32_t n, Step step) {
  for (uint32_t s = 0; s < n; ++s) {
    size_t len = size_t(1) << s;
    if (len >= 4096) {
      // parallel over disjoint chunks, each written from its end backwards
      unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
      std::vector<double> tmp(2 * len);
      std::vector<std::thread> th;
      for (unsigned w = 0; w < nt; ++w)
        th.emplace_back([&, w] {
          size_t a = len * w / nt, b = len * (w + 1) / nt;
          for (size_t j = a; j < b; ++j) {
            tmp[2 * j] = step(v[j], false);
            tmp[2 * j + 1] = step(v[j], true);
          }
        });
      for (auto &x : th) x.join();
      std::copy(tmp.begin(), tmp.end(), v.begin());
    } else {
      for (size_t j = len; j-- > 0;) {
        double p = v[j];
        v[2 * j + 1] = step(p, true);
        v[2 * j] = step(p, false);
      }
    }
  }
}

static polar_frozen_set *new_set(uint32_t log2n) {
  auto *fs = new (std::nothrow) polar_frozen_set();
  if (!fs) return nullptr;
  fs->id = g_fs_ids.fetch_add(1);
  fs->log2n = log2n;
  fs->N = uint64_t(1) << log2n;
  fs->mask.assign(std::max<uint64_t>(1, fs->N / 32), 0u);
  return fs;
}

// Bhattacharyya (BSC) / GA (BI-AWGN) set; K = floor(rate N), or (sum_rule)
// the largest K whose most reliable channels have sum exp(bad) <= sum_max.
static int bound_set(uint32_t log2n, polar_channel ch, double param, bool sum_rule,
                     double rate, double sum_max, polar_frozen_set **out) {
  NvtxRange nv("polar construct (bound / GA)");
  if (!out || log2n < 1 || log2n > 27) return POLAR_EINVAL;
  if (!(rate >= 0.0 && rate <= 1.0) || !(sum_max >= 0.0)) return POLAR_EINVAL;
  if (ch == POLAR_BSC) {
    if (!(param > 0.0 && param < 0.5)) return POLAR_EINVAL;
  } else if (ch == POLAR_BIAWGN) {
    if (!(param > 0.0 && std::isfinite(param))) return POLAR_EINVAL;
  } else {
    return POLAR_EINVAL;
  }
  const uint64_t N = uint64_t(1) << log2n;
  std::vector<double> bad;
  try {
    bad.assign(N, 0.0);
  } catch (...) {
    return POLAR_ENOMEM;
  }
  if (ch == POLAR_BSC) {
    bad[0] = std::log(2.0) + 0.5 * (std::log(param) + std::log1p(-param));
    polarise(bad, log2n, bh_step);
  } else {
    bad[0] = 2.0 / param;
    polarise(bad, log2n, ga_step);
    for (auto &m : bad) m = ln_q(std::sqrt(m / 2.0));
  }
  polar_frozen_set *fs = new_set(log2n);
  if (!fs) return POLAR_ENOMEM;
  // Rank by unreliability (descending), lower index first on ties; the
  // first N-K are frozen.
  std::vector<uint32_t> idx(N);
  for (uint64_t i = 0; i < N; ++i) idx[i] = (uint32_t)i;
  auto worse = [&](uint32_t a, uint32_t b) {
    if (bad[a] != bad[b]) return bad[a] > bad[b];
    return a < b;
  };
  if (sum_rule) {
    std::sort(idx.begin(), idx.end(), worse);
    double acc = 0.0;
    fs->K = 0;
    for (uint64_t r = N; r-- > 0;) {
      acc += std::exp(bad[idx[r]]);
      if (acc > sum_max) break;
      ++fs->K;
    }
  } else {
    fs->K = std::min<uint64_t>(N, (uint64_t)std::floor(rate * (double)N));
  }
  const uint64_t nf = N - fs->K;
  if (!sum_rule && nf > 0 && nf < N)
    std::nth_element(idx.begin(), idx.begin() + nf, idx.end(), worse);
  for (uint64_t r = 0; r < nf; ++r) fs->mask[idx[r] >> 5] |= 1u << (idx[r] & 31);
  double s = 0.0;
  for (uint64_t r = nf; r < N; ++r) s += std::exp(bad[idx[r]]);
  fs->sum_pe = s;
  *out = fs;
  return POLAR_OK;
}

int build_frozen_set(uint32_t log2n, polar_channel ch, double param, double rate,
                     polar_frozen_set **out) {
  return bound_set(log2n, ch, param, false, rate, 0.0, out);
}

int build_frozen_set_sum(uint32_t log2n, polar_channel ch, double param, double sum_pe_max,
                         polar_frozen_set **out) {
  return bound_set(log2n, ch, param, true, 0.0, sum_pe_max, out);
}

// ---------------------------------------------------------------- degraded construction
// Sec. 3's density evolution made finite after Tal & Vardy ("How to construct
// polar codes", 2013).  A binary-input symmetric channel is a mixture of
// BSCs: each conjugate output pair is one class with probability mass w and
// crossover z <= 1/2 (the error probability of the ML decision on that pair),
// and the channel's error probability is sum w z.  For two independent looks
// at classes (w1, z1), (w2, z2):
//   check node (minus):  one class, mass w1 w2, crossover z1 (1-z2) + z2 (1-z1);
//   variable node (plus): the looks agree -- mass w1 w2 ((1-z1)(1-z2) + z1 z2),
//                         crossover z1 z2 / that sum -- or disagree -- mass
//                         w1 w2 (z1 (1-z2) + z2 (1-z1)), crossover the smaller
//                         of the two products / that sum.
// Merging two classes into (w1 + w2, (w1 z1 + w2 z2) / (w1 + w2)) gives a
// channel degraded with respect to the original, so every error probability
// computed here bounds the true one from above.  A channel is kept at M = mu/2
// classes: they are ordered by crossover and the neighbours whose merger
// loses the least capacity, w1 C(z1) + w2 C(z2) - (w1 + w2) C(z12) with
// C(z) = 1 - h2(z), are merged first (on equal loss the pair of larger
// crossover), which is Tal and Vardy's greedy merging.  A BI-AWGN start is cut into 4M classes
// by |LLR| thresholds at which the BSC capacity 1 - h2(1 / (1 + e^|l|)) steps
// by 1 / (4M).  Every leaf of the tree is computed by the same operations in
// the same order whichever thread walks it.
namespace {

struct Cls {
  double w, z;
};

inline double h2(double z) {
  double h = 0.0;
  if (z > 0.0) h -= z * std::log2(z);
  if (z < 1.0) h -= (1.0 - z) * std::log2(1.0 - z);
  return h;
}
inline double cap_of(const Cls &c) { return c.w * (1.0 - h2(c.z)); }

inline Cls merged(const Cls &x, const Cls &y) {
  const double w = x.w + y.w;
  return Cls{w, w > 0.0 ? (x.w * x.z + y.w * y.z) / w : 0.0};
}

// Classes of the check-node / variable-node channel of two looks at c[0..L).
// Unordered pairs i <= j; i != j counts both orders.
size_t combine(const Cls *c, size_t L, bool plus, Cls *out) {
  size_t m = 0;
  for (size_t i = 0; i < L; ++i) {
    for (size_t j = i; j < L; ++j) {
      const double mass = (i == j ? 1.0 : 2.0) * c[i].w * c[j].w;
      const double zi = c[i].z, zj = c[j].z;
      if (!plus) {
        out[m++] = Cls{mass, zi * (1.0 - zj) + zj * (1.0 - zi)};
        continue;
      }
      const double agree = (1.0 - zi) * (1.0 - zj) + zi * zj;
      const double p1 = zi * (1.0 - zj), p2 = zj * (1.0 - zi), differ = p1 + p2;
      if (agree > 0.0) out[m++] = Cls{mass * agree, zi * zj / agree};
      if (differ > 0.0) out[m++] = Cls{mass * differ, std::min(p1, p2) / differ};
    }
  }
  return m;
}

// Greedy merging down to at most M classes.  A min-heap holds each adjacent
// pair's loss keyed by (loss, position of its left class); merged-away or
// stale entries are skipped when they surface.
struct Merger {
  std::vector<Cls> cls;
  std::vector<int> prev, next;
  std::vector<uint32_t> stamp;
  struct Item {
    double loss;
    int left;
    uint32_t s1, s2;
    bool operator>(const Item &o) const {
      return loss != o.loss ? loss > o.loss : left > o.left;
    }
  };
  std::vector<Item> heap;

  size_t run(Cls *c, size_t L, size_t M) {
    size_t n = 0;
    for (size_t k = 0; k < L; ++k)
      if (c[k].w > 0.0) c[n++] = c[k];
    // likelihood ratio (1 - z) / z ascending: crossover descending, then mass
    std::sort(c, c + n, [](const Cls &x, const Cls &y) {
      return x.z != y.z ? x.z > y.z : x.w < y.w;
    });
    if (n <= M) return n;
    cls.assign(c, c + n);
    prev.resize(n);
    next.resize(n);
    stamp.assign(n, 0u);
    for (size_t k = 0; k < n; ++k) {
      prev[k] = (int)k - 1;
      next[k] = k + 1 < n ? (int)k + 1 : -1;
    }
    auto loss_at = [&](int l) {
      const int r = next[l];
      return cap_of(cls[l]) + cap_of(cls[r]) - cap_of(merged(cls[l], cls[r]));
    };
    heap.clear();
    for (int k = 0; k + 1 < (int)n; ++k) heap.push_back(Item{loss_at(k), k, 0u, 0u});
    std::make_heap(heap.begin(), heap.end(), std::greater<Item>());
    size_t live = n;
    while (live > M && !heap.empty()) {
      std::pop_heap(heap.begin(), heap.end(), std::greater<Item>());
      const Item it = heap.back();
      heap.pop_back();
      const int l = it.left, r = next[l];
      if (r < 0 || stamp[l] != it.s1 || stamp[r] != it.s2) continue;   // stale
      cls[l] = merged(cls[l], cls[r]);
      ++stamp[l];
      stamp[r] = 0xFFFFFFFFu;                       // gone
      next[l] = next[r];
      if (next[r] >= 0) prev[next[r]] = l;
      --live;
      if (prev[l] >= 0) {
        const int q = prev[l];
        heap.push_back(Item{loss_at(q), q, stamp[q], stamp[l]});
        std::push_heap(heap.begin(), heap.end(), std::greater<Item>());
      }
      if (next[l] >= 0) {
        heap.push_back(Item{loss_at(l), l, stamp[l], stamp[next[l]]});
        std::push_heap(heap.begin(), heap.end(), std::greater<Item>());
      }
    }
    size_t m = 0;
    for (int k = 0; k >= 0; k = next[k]) c[m++] = cls[k];
    return m;
  }
};

inline double gauss_tail(double x) { return 0.5 * std::erfc(x / M_SQRT2); }

// |LLR| at which the BSC of crossover 1 / (1 + e^l) has capacity c (0 < c < 1).
double llr_at_capacity(double c) {
  // 1 - h2(z) = c for z in (0, 1/2): h2 is increasing there, bisect on z
  double lo = 0.0, hi = 0.5;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (1.0 - h2(mid) > c) lo = mid;
    else hi = mid;
  }
  const double z = 0.5 * (lo + hi);
  return std::log((1.0 - z) / z);
}

// The channel's starting classes.
std::vector<Cls> start_classes(polar_channel ch, double param, size_t M0) {
  if (ch == POLAR_BSC) return {Cls{1.0, param}};
  const double sg = std::sqrt(param);
  std::vector<Cls> out;
  double y0 = 0.0;                                  // class k: |y| in [y0, y1)
  for (size_t k = 0; k < M0; ++k) {
    const double y1 =
        k + 1 < M0 ? llr_at_capacity((double)(k + 1) / (double)M0) * param / 2.0 : INFINITY;
    // mass given x = 0 (y ~ N(1, s2)) on y in [y0, y1) (a) and y in (-y1, -y0] (b)
    const double a = gauss_tail((y0 - 1.0) / sg) - (std::isinf(y1) ? 0.0 : gauss_tail((y1 - 1.0) / sg));
    const double b = gauss_tail((y0 + 1.0) / sg) - (std::isinf(y1) ? 0.0 : gauss_tail((y1 + 1.0) / sg));
    const double w = a + b;
    out.push_back(Cls{w, w > 0.0 ? b / w : 0.0});
    y0 = y1;
  }
  return out;
}

struct Walk {
  int n;
  size_t M;
  double *pe;
  std::vector<Cls> buf;     // children of every depth: (n + 1) * M
  std::vector<Cls> prod;
  Merger mg;
  Walk(int n_, size_t M_, double *pe_, size_t cap)
      : n(n_), M(M_), pe(pe_), buf((size_t)(n_ + 1) * M_), prod(cap) {}
  // the subtree below the channel c (L classes) at depth d, leaf index base j
  void down(const Cls *c, size_t L, int d, uint64_t j) {
    if (d == n) {
      double e = 0.0;
      for (size_t k = 0; k < L; ++k) e += c[k].w * c[k].z;
      pe[j] = e;
      return;
    }
    Cls *ch = buf.data() + (size_t)(d + 1) * M;
    for (int side = 0; side < 2; ++side) {      // minus child (index bit 0), then plus
      size_t m = combine(c, L, side == 1, prod.data());
      m = mg.run(prod.data(), m, M);
      std::copy(prod.begin(), prod.begin() + m, ch);
      down(ch, m, d + 1, 2 * j + side);
    }
  }
};

}  // namespace

int tv_bit_channel_pe(uint32_t log2n, polar_channel ch, double param, int mu,
                      std::vector<double> &pe) {
  const int n = (int)log2n;
  const size_t M = (size_t)mu / 2, M0 = 4 * M;
  const size_t cap = std::max(M * (M + 1), M0) + 8;
  try {
    pe.assign(size_t(1) << n, 0.0);
  } catch (...) {
    return POLAR_ENOMEM;
  }
  std::vector<Cls> root = start_classes(ch, param, M0);
  Merger mg0;
  root.resize(cap);
  const size_t L0 = mg0.run(root.data(), M0 == 0 || ch == POLAR_BSC ? 1 : M0, M);
  // Expand the first levels breadth first (one list of channels per level),
  // then walk each of those subtrees depth first on its own thread.
  const int top = std::min(n, 6);
  std::vector<std::vector<Cls>> level{std::vector<Cls>(root.begin(), root.begin() + L0)};
  std::vector<Cls> prod(cap);
  for (int d = 0; d < top; ++d) {
    std::vector<std::vector<Cls>> nx;
    nx.reserve(level.size() * 2);
    for (const auto &c : level)
      for (int side = 0; side < 2; ++side) {
        size_t m = combine(c.data(), c.size(), side == 1, prod.data());
        m = mg0.run(prod.data(), m, M);
        nx.emplace_back(prod.begin(), prod.begin() + m);
      }
    level.swap(nx);
  }
  std::atomic<size_t> next{0};
  auto worker = [&] {
    Walk wk(n, M, pe.data(), cap);
    for (;;) {
      const size_t r = next.fetch_add(1);
      if (r >= level.size()) break;
      wk.down(level[r].data(), level[r].size(), top, r);
    }
  };
  const unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  if (n <= 10 || nt == 1) {
    worker();
  } else {
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t) th.emplace_back(worker);
    for (auto &x : th) x.join();
  }
  return POLAR_OK;
}

int build_frozen_set_tv(uint32_t log2n, polar_channel ch, double param, int mu, double rate,
                        double sum_pe_max, polar_frozen_set **out) {
  NvtxRange nv("polar construct (degraded)");
  if (!out || log2n < 1 || log2n > 27 || mu < 2 || mu > 128 || (mu & 1)) return POLAR_EINVAL;
  if (!(rate >= 0.0 && rate <= 1.0) || !(sum_pe_max >= 0.0)) return POLAR_EINVAL;
  if (ch == POLAR_BSC) {
    if (!(param > 0.0 && param < 0.5)) return POLAR_EINVAL;
  } else if (ch == POLAR_BIAWGN) {
    if (!(param > 0.0 && std::isfinite(param))) return POLAR_EINVAL;
  } else {
    return POLAR_EINVAL;
  }
  std::vector<double> pe;
  int rc = tv_bit_channel_pe(log2n, ch, param, mu, pe);
  if (rc) return rc;
  const uint64_t N = uint64_t(1) << log2n;
  // rank: error probability descending, lower index first on ties
  std::vector<uint32_t> idx(N);
  for (uint64_t i = 0; i < N; ++i) idx[i] = (uint32_t)i;
  std::sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) {
    if (pe[a] != pe[b]) return pe[a] > pe[b];
    return a < b;
  });
  uint64_t K;
  if (rate > 0.0) {
    K = std::min<uint64_t>(N, (uint64_t)std::floor(rate * (double)N));
  } else {   // Sec. 3: the largest K whose best channels sum to <= sum_pe_max
    double acc = 0.0;
    K = 0;
    for (uint64_t r = N; r-- > 0;) {
      acc += pe[idx[r]];
      if (acc > sum_pe_max) break;
      ++K;
    }
  }
  polar_frozen_set *fs = new_set(log2n);
  if (!fs) return POLAR_ENOMEM;
  fs->K = K;
  const uint64_t nf = N - K;
  for (uint64_t r = 0; r < nf; ++r) fs->mask[idx[r] >> 5] |= 1u << (idx[r] & 31);
  double s = 0.0;
  for (uint64_t r = N; r-- > nf;) s += pe[idx[r]];
  fs->sum_pe = s;
  *out = fs;
  return POLAR_OK;
}

int frozen_set_from_mask(uint32_t log2n, const uint32_t *mask, polar_frozen_set **out) {
  if (!out || !mask || log2n < 1 || log2n > 27) return POLAR_EINVAL;
  polar_frozen_set *fs = new_set(log2n);
  if (!fs) return POLAR_ENOMEM;
  const uint64_t W = fs->mask.size();
  uint64_t frozen = 0;
  for (uint64_t w = 0; w < W; ++w) {
    uint32_t v = mask[w];
    if (fs->N < 32) v &= (1u << fs->N) - 1u;
    fs->mask[w] = v;
    frozen += (uint64_t)__builtin_popcount(v);
  }
  fs->K = fs->N - frozen;
  fs->sum_pe = std::nan("");
  *out = fs;
  return POLAR_OK;
}

// Class of the node of 2^k leaves starting at leaf o, from the host mask.
NodeClass node_class_host(const polar_frozen_set *fs, int k, uint64_t o) {
  if (k < 5) {
    uint32_t w = fs->mask[o >> 5];
    uint32_t m = (1u << (1u << k)) - 1u;
    uint32_t b = (w >> (o & 31)) & m;
    return b == m ? NODE_RATE0 : (b == 0 ? NODE_RATE1 : NODE_MIXED);
  }
  uint64_t w0 = o >> 5, nw = uint64_t(1) << (k - 5);
  bool all1 = true, all0 = true;
  for (uint64_t w = w0; w < w0 + nw && (all1 || all0); ++w) {
    all1 &= fs->mask[w] == 0xFFFFFFFFu;
    all0 &= fs->mask[w] == 0u;
  }
  return all1 ? NODE_RATE0 : (all0 ? NODE_RATE1 : NODE_MIXED);
}

// Streamed schedule of the SC recursion above level t.  Rate-0 nodes of any
// size become one OP_R0 (their partial sums are the encoded frozen values,
// independent of the LLRs); the f feeding a rate-0 left child is skipped.
// Every unit (subtree or rate-0 node) records how many levels it is a right
// child for: that many partial-sum combines follow it.
static void plan_visit(const polar_frozen_set *fs, Plan &p, int k, uint64_t o) {
  const int n = (int)fs->log2n;
  auto unit_r = [&](int ku, uint64_t ou) {
    uint64_t pos = ou >> ku;
    int r = 0;
    while (ku + r < n && ((pos >> r) & 1)) ++r;
    return r;
  };
  auto rate0 = [&](int kk, uint64_t oo) {
    return p.shortcuts && kk >= 5 && node_class_host(fs, kk, oo) == NODE_RATE0;
  };
  if (rate0(k, o)) {
    p.ops.push_back(Op{OP_R0, (uint8_t)k, (uint8_t)unit_r(k, o), 0, o});
    p.n_r0++;
    return;
  }
  if (k == p.t) {
    p.ops.push_back(Op{OP_ST, (uint8_t)k, (uint8_t)unit_r(k, o), 0, o});
    p.n_st++;
    return;
  }
  if (k == p.split) {
    p.ops.push_back(Op{OP_NODE, (uint8_t)k, (uint8_t)unit_r(k, o), 0, o});
    p.n_node++;
    return;
  }
  uint64_t h = uint64_t(1) << (k - 1);
  if (!rate0(k - 1, o)) {
    p.ops.push_back(Op{OP_F, (uint8_t)k, 0, 0, o});
    p.n_f++;
  }
  plan_visit(fs, p, k - 1, o);
  if (!rate0(k - 1, o + h)) {          // a rate-0 right child needs no LLRs
    p.ops.push_back(Op{OP_G, (uint8_t)k, 0, 0, o});
    p.n_g++;
  }
  plan_visit(fs, p, k - 1, o + h);
}

// Give each subtree the step that produces its input when that step comes
// right before it: an f (left child) or g (right child) at level t + 1 is
// done by the subtree kernel itself while it loads the parent's LLRs
// (pad = 1 / 2), instead of by a separate launch that writes level t.
static void plan_prologue(Plan &p) {
  std::vector<Op> out;
  out.reserve(p.ops.size());
  const uint64_t T = uint64_t(1) << p.t;
  for (size_t i = 0; i < p.ops.size(); ++i) {
    const Op &a = p.ops[i];
    if ((a.kind == OP_F || a.kind == OP_G) && a.k == p.t + 1 && i + 1 < p.ops.size()) {
      const Op &b = p.ops[i + 1];
      const uint64_t child = a.kind == OP_F ? a.o : a.o + T;
      if (b.kind == OP_ST && b.o == child) {
        Op m = b;
        m.pad = a.kind == OP_F ? 1 : 2;
        out.push_back(m);
        if (a.kind == OP_F) p.n_f--;
        else p.n_g--;
        ++i;
        continue;
      }
    }
    out.push_back(a);
  }
  p.ops.swap(out);
}

// Merge each f or g step with the f steps that directly continue it (level
// by level down the left edge) into one fused chain of at most 7 levels.
static void plan_fuse(Plan &p) {
  std::vector<Op> out;
  out.reserve(p.ops.size());
  for (size_t i = 0; i < p.ops.size();) {
    const Op &a = p.ops[i];
    if (a.kind != OP_F && a.kind != OP_G) {
      out.push_back(a);
      ++i;
      continue;
    }
    size_t j = i + 1;
    int levels = 1;
    while (j < p.ops.size() && levels < 7 && p.ops[j].kind == OP_F &&
           p.ops[j].k == a.k - levels) {
      ++levels;
      ++j;
    }
    out.push_back(Op{OP_CHAIN, a.k, (uint8_t)levels, (uint8_t)(a.kind == OP_G ? 1 : 0), a.o});
    p.n_chain++;
    i = j;
  }
  p.ops.swap(out);
}

std::shared_ptr<Plan> get_plan(polar_frozen_set *fs, int t, bool shortcuts, bool fuse,
                               bool prologue, int split) {
  std::lock_guard<std::mutex> g(fs->mu);
  // nodes need the class tables and word-aligned units; none at or above the root
  if (!shortcuts || t < 5 || split <= t || split >= (int)fs->log2n) split = 0;
  auto key = std::make_pair(t, (shortcuts ? 1 : 0) | (fuse ? 2 : 0) | (prologue ? 4 : 0) |
                                   (split << 8));
  auto it = fs->plans.find(key);
  if (it != fs->plans.end()) return it->second;
  auto p = std::make_shared<Plan>();
  p->t = t;
  p->split = split;
  p->shortcuts = shortcuts;
  plan_visit(fs, *p, (int)fs->log2n, 0);
  if (prologue && shortcuts && t >= 5) plan_prologue(*p);   // word-aligned subtrees
  if (fuse) plan_fuse(*p);
  fs->plans[key] = p;
  return p;
}

const uint32_t *device_mask(polar_frozen_set *fs, int device, cudaError_t *err) {
  std::lock_guard<std::mutex> g(fs->mu);
  *err = cudaSuccess;
  auto it = fs->dmask.find(device);
  if (it != fs->dmask.end()) return it->second;
  uint32_t *d = nullptr;
  size_t bytes = fs->mask.size() * sizeof(uint32_t);
  *err = cudaMalloc(&d, bytes);
  if (*err != cudaSuccess) return nullptr;
  *err = cudaMemcpy(d, fs->mask.data(), bytes, cudaMemcpyHostToDevice);
  if (*err != cudaSuccess) {
    cudaFree(d);
    return nullptr;
  }
  fs->dmask[device] = d;
  return d;
}

static std::vector<uint32_t> build_class_table(const polar_frozen_set *fs, int t) {
  const int n = (int)fs->log2n;
  const uint32_t CW = class_words(t);
  const uint64_t nsub = t <= n ? (uint64_t(1) << (n - t)) : 1;
  std::vector<uint32_t> tab(nsub * 2 * CW, 0u);
  if (t < 5) return tab;
  for (uint64_t j = 0; j < nsub; ++j) {
    uint32_t *r0 = tab.data() + j * 2 * CW, *r1 = r0 + CW;
    for (int k = 5; k <= t; ++k) {
      for (uint64_t q = 0; q < (uint64_t(1) << (t - k)); ++q) {
        const NodeClass c = node_class_host(fs, k, (j << t) + (q << k));
        const uint64_t i = (uint64_t(1) << (t - k)) + q;
        if (c == NODE_RATE0) r0[i >> 5] |= 1u << (i & 31);
        if (c == NODE_RATE1) r1[i >> 5] |= 1u << (i & 31);
      }
    }
  }
  return tab;
}

std::shared_ptr<std::vector<uint32_t>> class_table_host(polar_frozen_set *fs, int t) {
  std::lock_guard<std::mutex> g(fs->mu);
  auto it = fs->hclass.find(t);
  if (it != fs->hclass.end()) return it->second;
  auto tab = std::make_shared<std::vector<uint32_t>>(build_class_table(fs, t));
  fs->hclass[t] = tab;
  return tab;
}

const uint32_t *device_class_table(polar_frozen_set *fs, int device, int t, cudaError_t *err) {
  *err = cudaSuccess;
  {
    std::lock_guard<std::mutex> g(fs->mu);
    auto it = fs->dclass.find({device, t});
    if (it != fs->dclass.end()) return it->second;
  }
  std::shared_ptr<std::vector<uint32_t>> tab = class_table_host(fs, t);
  uint32_t *d = nullptr;
  *err = cudaMalloc(&d, tab->size() * sizeof(uint32_t));
  if (*err != cudaSuccess) return nullptr;
  *err = cudaMemcpy(d, tab->data(), tab->size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (*err != cudaSuccess) {
    cudaFree(d);
    return nullptr;
  }
  std::lock_guard<std::mutex> g(fs->mu);
  auto it = fs->dclass.find({device, t});
  if (it != fs->dclass.end()) {
    cudaFree(d);
    return it->second;
  }
  fs->dclass[{device, t}] = d;
  return d;
}

// Upper levels from the subtree roots up: a node is rate 0 (rate 1) when
// both children are.
static std::vector<uint32_t> build_upper_class_table(const polar_frozen_set *fs, int t) {
  const int n = (int)fs->log2n;
  const uint32_t UW = upper_class_words(n, t);
  std::vector<uint32_t> tab(2 * (size_t)UW, 0u);
  std::vector<uint8_t> cur(size_t(1) << (n - t)), nxt;
  for (uint64_t q = 0; q < cur.size(); ++q) cur[q] = node_class_host(fs, t, q << t);
  for (int k = t;; ++k) {
    for (uint64_t q = 0; q < cur.size(); ++q) {
      const uint64_t i = (uint64_t(1) << (n - k)) + q;
      if (cur[q] == NODE_RATE0) tab[i >> 5] |= 1u << (i & 31);
      if (cur[q] == NODE_RATE1) tab[UW + (i >> 5)] |= 1u << (i & 31);
    }
    if (k == n) break;
    nxt.assign(cur.size() / 2, NODE_MIXED);
    for (uint64_t q = 0; q < nxt.size(); ++q)
      if (cur[2 * q] == cur[2 * q + 1]) nxt[q] = cur[2 * q];
    cur.swap(nxt);
  }
  return tab;
}

const uint32_t *device_upper_class_table(polar_frozen_set *fs, int device, int t,
                                         cudaError_t *err) {
  *err = cudaSuccess;
  if ((int)fs->log2n <= t) return nullptr;
  {
    std::lock_guard<std::mutex> g(fs->mu);
    auto it = fs->ducls.find({device, t});
    if (it != fs->ducls.end()) return it->second;
  }
  const std::vector<uint32_t> tab = build_upper_class_table(fs, t);
  uint32_t *d = nullptr;
  *err = cudaMalloc(&d, tab.size() * sizeof(uint32_t));
  if (*err != cudaSuccess) return nullptr;
  *err = cudaMemcpy(d, tab.data(), tab.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (*err != cudaSuccess) {
    cudaFree(d);
    return nullptr;
  }
  std::lock_guard<std::mutex> g(fs->mu);
  auto it = fs->ducls.find({device, t});
  if (it != fs->ducls.end()) {
    cudaFree(d);
    return it->second;
  }
  fs->ducls[{device, t}] = d;
  return d;
}

}  // namespace polar
