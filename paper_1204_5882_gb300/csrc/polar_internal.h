// Internal declarations of the GB300 SC polar decoder library (not part of
// the C ABI).  The public contract is include/polar.h.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "polar.h"

#include <nvtx3/nvToolsExt.h>

// Small index helpers used by host and device code.
#ifdef __CUDACC__
#define POLAR_HD __host__ __device__
#else
#define POLAR_HD
#endif

namespace polar {

// Node classes of the SC tree, read from the frozen mask (Sec. 3 / Sec. 4):
// all positions frozen (rate 0), all information (rate 1) or mixed.
enum NodeClass : uint8_t { NODE_MIXED = 0, NODE_RATE0 = 1, NODE_RATE1 = 2 };

// One step of the streamed (upper) part of the SC recursion.  Levels are
// counted from the leaves: level k holds nodes of 2^k leaves; the root is at
// level n.  `o` is the first leaf (bit offset) of the node the op touches.
enum OpKind : uint8_t {
  OP_F = 0,   // level k -> k-1, left child LLRs  L'[j] = f(L[j], L[j+h])
  OP_G = 1,   // level k -> k-1, right child LLRs L'[j] = g(L[j], L[j+h], b[o+j])
  OP_ST = 2,  // decode the subtree of 2^t leaves at o in one CTA
  OP_R0 = 3,  // rate-0 node of 2^k leaves at o: partial sums = fv F^{(x)k}
  OP_CHAIN = 4,  // fused steps level k -> k - r: first g (pad = 1) or f, then f
  OP_NODE = 5,   // node of 2^k leaves (k > t) at o decoded by one CTA per frame
};

struct Op {
  uint8_t kind;
  uint8_t k;
  uint8_t r;   // partial-sum combine levels done after a unit (ST / R0)
  uint8_t pad;   // OP_CHAIN: 1 = the first step is g; OP_ST: 1 / 2 = the subtree
                 // computes its input itself by f / g from level t + 1
  uint64_t o;
};

struct Plan {
  int t = 0;
  int split = 0;          // level of the OP_NODE units (0: none)
  bool shortcuts = true;
  std::vector<Op> ops;
  int n_st = 0, n_f = 0, n_g = 0, n_r0 = 0, n_chain = 0, n_node = 0;
};

}  // namespace polar

struct polar_frozen_set {
  uint64_t id = 0;
  uint32_t log2n = 0;
  uint64_t N = 0, K = 0;
  double sum_pe = 0.0;
  std::vector<uint32_t> mask;   // max(1, N/32) words, bit set = frozen
  std::mutex mu;
  std::map<int, uint32_t *> dmask;                        // device -> mask copy
  std::map<std::pair<int, int>, uint32_t *> dclass;       // (device, t) -> class table
  std::map<std::pair<int, int>, uint32_t *> ducls;        // (device, t) -> upper class table
  std::map<int, std::shared_ptr<std::vector<uint32_t>>> hclass;   // t -> host class table
  std::map<std::pair<int, int>, std::shared_ptr<polar::Plan>> plans;  // (t, flags)
};

namespace polar {

// --- construction (construct.cpp) -----------------------------------------
int build_frozen_set(uint32_t log2n, polar_channel ch, double param, double rate,
                     polar_frozen_set **out);
int build_frozen_set_sum(uint32_t log2n, polar_channel ch, double param, double sum_pe_max,
                         polar_frozen_set **out);
int frozen_set_from_mask(uint32_t log2n, const uint32_t *mask, polar_frozen_set **out);
// Degraded-channel (Tal-Vardy) construction: bit-channel error bounds, and
// the frozen set they give (K = floor(rate N), or by the sum rule if rate = 0).
int tv_bit_channel_pe(uint32_t log2n, polar_channel ch, double param, int mu,
                      std::vector<double> &pe);
int build_frozen_set_tv(uint32_t log2n, polar_channel ch, double param, int mu, double rate,
                        double sum_pe_max, polar_frozen_set **out);
NodeClass node_class_host(const polar_frozen_set *fs, int k, uint64_t o);
// Bhattacharyya (BSC) / GA (BI-AWGN) set built on the current device in
// double precision (construct_dev.cu): K = floor(rate N), or with rate = 0
// the largest K whose most reliable channels have sum P_e <= sum_max.
int build_frozen_set_device(uint32_t log2n, polar_channel ch, double param, double rate,
                            double sum_max, cudaStream_t s, polar_frozen_set **out);
// fuse: chain kernels for runs of streamed steps; prologue: the subtree
// kernel performs the streamed step that produces its input; split > t: every
// node of 2^split leaves that is not rate 0 is one OP_NODE unit (the levels
// split .. t + 1 then run inside its CTAs instead of as streamed launches).
std::shared_ptr<Plan> get_plan(polar_frozen_set *fs, int t, bool shortcuts, bool fuse,
                               bool prologue, int split = 0);
const uint32_t *device_mask(polar_frozen_set *fs, int device, cudaError_t *err);
// Node-class table of every subtree of 2^t leaves (levels 5..t): per subtree
// class_words(t) words of "rate 0" bits then as many of "rate 1" bits; node
// (k, q) of a subtree is bit 2^(t-k) + q.
POLAR_HD inline uint32_t class_words(int t) { return t >= 9 ? (1u << (t - 9)) : 1u; }
std::shared_ptr<std::vector<uint32_t>> class_table_host(polar_frozen_set *fs, int t);
const uint32_t *device_class_table(polar_frozen_set *fs, int device, int t, cudaError_t *err);
// Node-class table of the levels t..n of the whole code (n > t): node (k, q)
// is bit 2^(n-k) + q of upper_class_words(n, t) "rate 0" words, followed by
// as many "rate 1" words.
POLAR_HD inline uint32_t upper_class_words(int n, int t) {
  return n - t + 1 >= 5 ? (1u << (n - t + 1 - 5)) : 1u;
}
const uint32_t *device_upper_class_table(polar_frozen_set *fs, int device, int t,
                                         cudaError_t *err);

// --- kernels (stream_kernels.cu, subtree.cu) --------------------------------
cudaError_t launch_llr_bsc(const uint32_t *y, float *llr, size_t n_total, float c,
                           cudaStream_t s);
cudaError_t launch_llr_biawgn(const double *y, float *llr, size_t n_total, double scale,
                              cudaStream_t s);
// In-place transform of nframes regions of 2^log2len bits; region f starts at
// words + f * stride_w + off_w (word-aligned, log2len >= 5) or is the low
// 2^log2len bits of words[f * stride_w] (log2len < 5).
cudaError_t launch_encode_regions(uint32_t *words, size_t stride_w, size_t off_w,
                                  int log2len, int nframes, cudaStream_t s);
cudaError_t launch_copy_regions(const uint32_t *src, uint32_t *dst, size_t stride_w,
                                size_t off_w, size_t nwords, int nframes,
                                const uint32_t *and_mask, cudaStream_t s);
cudaError_t launch_cascade(uint32_t *xhat, size_t stride_w, int k_unit, uint64_t o_unit,
                           int r, int nframes, cudaStream_t s);

// Streamed f / g for levels above the subtree size (templated on storage).
// Level-n inputs (in_is_llr) are the float channel LLRs; they are scaled
// (int8) and rounded to the storage format on load.
cudaError_t launch_stream_f(int prec, int fkind, const void *in, size_t in_stride,
                            bool in_is_llr, void *out, size_t out_stride, uint64_t h,
                            int nframes, const float *scale, cudaStream_t s);
cudaError_t launch_stream_g(int prec, const void *in, size_t in_stride, bool in_is_llr,
                            void *out, size_t out_stride, uint64_t h,
                            const uint32_t *xhat, size_t xhat_stride_w, uint64_t o,
                            int nframes, const float *scale, cudaStream_t s);
// Fused run of streamed steps kt -> kb (first step g if first_g, then f);
// lv_base = start of the level buffers (level k of frame f at
// F * (2^k - 2^t) + f * 2^k elements).  kt - kb <= 7.
cudaError_t launch_chain(int prec, int fkind, bool first_g, const void *in, size_t in_stride,
                         bool in_is_llr, void *lv_base, int t, int nframes, int kt, int kb,
                         const uint32_t *xhat, size_t xhat_stride_w, uint64_t o_left,
                         const float *scale, cudaStream_t s);
// Per-frame int8 scale 2^round(log2(target / mean|L|)) (1 if all L = 0).
cudaError_t launch_int8_scale(const float *llr, size_t n, int nframes, double target,
                              float *scale, cudaStream_t s);

struct SubtreeArgs {
  const void *in;        // level-t LLRs of every frame (or the channel LLRs)
  size_t in_stride;      // elements between frames
  bool in_is_llr;        // in is the float channel LLR array (level n == t)
  const uint32_t *cls;   // device class table of this subtree (levels 5..t) or null
  const float *scale;    // per-frame int8 scale (null = 1)
  const uint32_t *mask;  // device frozen mask (whole code)
  const uint32_t *fv;
  uint32_t *xhat;
  uint32_t *uhat;
  size_t w_stride;       // words per frame
  uint64_t o;            // first leaf of the subtree
  int t;                 // subtree log2 size
  int r;                 // combine levels after the subtree
  int pre;               // 0: in is level t; 1 / 2: in is the parent at level t + 1
                         // and level t is its f / g (g reads the left child's bits)
  int nframes;
  int fkind;
  int prec;
  bool shortcuts;
};
cudaError_t launch_subtree(const SubtreeArgs &a, cudaStream_t s);

// A node of 2^s leaves (s > t) decoded by one CTA per frame: the levels
// s .. t + 1 inside the CTA over the frame's workspace rows, then its subtrees
// (node_impl.cuh).  Bit-identical to the streamed schedule of those levels.
struct NodeArgs {
  const void *lv;          // workspace level t (storage prec); level k at nframes (2^k - 2^t)
  const uint32_t *mask;    // device frozen mask (whole code)
  const uint32_t *cls;     // subtree class table (whole code) or null (no shortcuts)
  const uint32_t *ucls;    // upper class table of levels t..n
  const float *scale;      // per-frame int8 scale (null = 1)
  const uint32_t *fv;
  uint32_t *xhat;
  uint32_t *uhat;
  size_t w_stride;         // words per frame
  uint64_t o;              // first leaf of the node
  int s, t, n;             // node level, subtree level, code level
  int r;                   // combine levels after the node
  int nframes;
  int fkind;
  int prec;
};
cudaError_t launch_node(const NodeArgs &a, cudaStream_t s);
size_t node_smem_bytes_host(int t);

size_t storage_bytes(int prec);

// Keyed hash of each frame's packed words (verification of decoded blocks).
cudaError_t launch_frame_hash(const uint32_t *words, size_t stride_w, size_t nwords,
                              int nframes, uint64_t key, uint64_t *out, cudaStream_t s);

// --- persistent decoder (persist.cu) ------------------------------------------
// One frame of a persistent launch.  Levels t..n-1 of the frame being decoded
// live in the scratch of the CTA that claimed it.
struct PFrame {
  const float *llr;        // [2^log2n] channel LLRs, 16-byte aligned
  const uint32_t *fv;      // frozen values, packed
  uint32_t *xhat;          // x_hat, packed
  uint32_t *uhat;          // u_hat, packed, or null
  const uint32_t *mask;    // frozen mask of the code (device)
  const uint32_t *cls;     // subtree class tables (levels 5..t, t >= 5) or null
  const uint32_t *ucls;    // class table of the levels t..n (n > t) or null
  uint32_t log2n;
  uint32_t t;              // subtree size of this frame: min(log2n, the launch's t)
};
// Threads of a persistent CTA.
constexpr int kPersistThreads = 128;
// Dynamic shared memory of a persistent CTA for subtrees of up to 2^t leaves.
size_t persistent_smem_bytes(int t);
// Resident CTAs per SM of the persistent kernel (0 on error).
int persistent_ctas_per_sm(int prec, int fkind, bool uhat, int t);
// Frames [0, count) of `frames` (device) are claimed in order through *head
// (device, zero on entry) by `grid` CTAs; CTA c keeps its levels (stored as
// prec: float, half or int8) at scratch + c * cta_floats floats; int8 frames
// take the per-frame scale of the "int8_target" option.
cudaError_t launch_persistent(int prec, int fkind, bool uhat, const PFrame *frames,
                              uint32_t count, uint32_t *head, float *scratch,
                              uint64_t cta_floats, int t, int grid, double int8_target,
                              cudaStream_t s);

// Serving launch: frames come from a ring in host-mapped memory that the
// host fills while the launch runs (see persist.cu).
struct ServeArgs {
  const PFrame *ring;      // host-mapped, rmask + 1 entries (a power of two)
  uint32_t rmask;
  const uint32_t *tail;    // host-mapped: frames published so far
  const uint32_t *stop;    // host-mapped: 1 = leave once nothing is published
  uint32_t *done;          // host-mapped: done[i & rmask] = i + 1 once frame i is decoded
  uint32_t *head;          // device: frames claimed so far (kept across launches)
  float *scratch;          // grid * cta_floats floats
  uint64_t cta_floats;
  uint64_t idle_ns;        // a CTA leaves after this long without a frame
  double int8_target;      // int8 storage: target of the per-frame scale
  uint32_t smem;           // set by launch_serve
};
int serve_ctas_per_sm(int prec, int fkind, int t);
// Make a frozen set resident on `dev` for decodes at subtree size t: its
// mask, the node-class table of the subtrees (t >= 5) and, with `upper`, the
// class table of the levels above t that the persistent decoder reads.
// Switches to `dev` for the uploads and back.  OK, ENOMEM or ECUDA.
int prepare_tables(polar_frozen_set *fs, int dev, int t, bool upper);
cudaError_t launch_serve(int prec, int fkind, ServeArgs a, int t, int grid, cudaStream_t s);

// api.cu: decoding with caller-provided device mask and level scratch.
size_t level_scratch_bytes(const polar_frozen_set *fs, int nframes, int prec, int *t_out);
// One read of the decode options for a scratch-supplied decode (subtree size
// t, autotuned when cached; shortcuts; fused streamed steps; prologue).
struct ScratchOpts {
  int t;
  bool shortcuts, fuse, prologue;
};
ScratchOpts scratch_opts(const polar_frozen_set *fs, int nframes, int fkind, int prec);
// Level scratch (and int8 scales) of nframes frames at subtree size t, bytes.
size_t scratch_level_bytes(const polar_frozen_set *fs, int nframes, int prec, int t);
int decode_with_scratch(const polar_frozen_set *fs, int nframes, const float *llr,
                        const uint32_t *fv, uint32_t *xhat, uint32_t *uhat, int fkind, int prec,
                        const ScratchOpts &o, const uint32_t *dmask, const uint32_t *dclass,
                        void *scratch, size_t scratch_bytes, cudaStream_t s);
void set_last_error(const char *msg);
// Diagnostics on stderr ("[polar] ..." lines) when the environment variable
// POLAR_LOG is set to anything but "" or "0" (read once): frozen-set
// construction, autotune choices, tune-cache files, server launches.
bool log_on();
void log_msg(const char *fmt, ...) __attribute__((format(printf, 1, 2)));
int decode_eager(const polar_frozen_set *fs, int nframes, const float *llr, const uint32_t *fv,
                 uint32_t *xhat, uint32_t *uhat, int fkind, int prec, cudaStream_t s);
size_t decode_scratch_bytes(const polar_frozen_set *fs, int nframes, int prec);
void release_stream_workspace(int dev, cudaStream_t s);

// NVTX range over a host-side stage (a no-op unless a profiler is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Kernels launched by this library (graph replays included).
extern std::atomic<uint64_t> g_kernel_launches;
// 1 = decode kernels are launched with programmatic dependent launch.
extern std::atomic<int> g_pdl;
inline cudaError_t counted(cudaError_t e, uint64_t kernels) {
  if (e == cudaSuccess) g_kernel_launches.fetch_add(kernels, std::memory_order_relaxed);
  return e;
}

}  // namespace polar
