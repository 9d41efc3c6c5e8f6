// C ABI of the GB300 SC polar decoder (include/polar.h): argument checks,
// per-stream scratch, the streamed schedule of the SC recursion and its
// replay as CUDA graphs.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <list>
#include <tuple>

#include "polar_internal.h"

using namespace polar;

namespace {

thread_local std::string g_last_error;

struct Config {
  std::atomic<long> subtree_log2{14};
  std::atomic<long> persist_log2{13};
  std::atomic<long> shortcuts{1};
  std::atomic<long> graphs{1};
  std::atomic<long> plain{0};
  std::atomic<long> profile{0};
  std::atomic<long> int8_target{8};
  std::atomic<long> fuse{1};
  std::atomic<long> prologue{0};
  std::atomic<long> autotune{1};
  std::atomic<long> persistent{1};
  std::atomic<long> guard{0};
  std::atomic<long> split_log2{0};   // level of node units (0: none), see get_plan
};

// ---------------------------------------------------------------- autotuning
// Best (subtree size, schedule flags: 1 = fused streamed steps, 2 = the
// subtree kernel takes its parent's step) per batch shape, found by
// polar_autotune; used by later decodes of that shape while "autotune" is 1.
struct TuneKey {
  int dev, log2n, nframes, fkind, prec;
  bool operator<(const TuneKey &o) const {
    return std::tie(dev, log2n, nframes, fkind, prec) <
           std::tie(o.dev, o.log2n, o.nframes, o.fkind, o.prec);
  }
};
struct TuneVal {
  int t;
  int fuse;
  double ms;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;
Config g_cfg;

// ---------------------------------------------------------------- profiling
struct ProfRec {
  int kind;
  cudaEvent_t a, b;
  double bytes;
};
const char *const kKinds[] = {"llr",   "stream_f", "stream_g", "subtree",
                              "rate0", "chain",    "persist",  "node"};
constexpr int kNumKinds = 8;
std::mutex g_prof_mu;
std::vector<ProfRec> g_prof_pending;
double g_prof_ms[kNumKinds];
uint64_t g_prof_n[kNumKinds];
double g_prof_bytes[kNumKinds];

struct ProfScope {
  bool on;
  int kind;
  double bytes;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  bool captured = false;   // inside a stream capture: record as event nodes of the graph
  ProfScope(bool enable, int k, double by, cudaStream_t st) : on(enable), kind(k), bytes(by), s(st) {
    if (!on) return;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      cudaGetLastError();
      on = false;
      return;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    captured = cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
    record(a);
  }
  void record(cudaEvent_t e) {
    if (captured) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else cudaEventRecord(e, s);
  }
  ~ProfScope() {
    if (!on) return;
    record(b);
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof_pending.push_back({kind, a, b, bytes});
  }
};

void prof_drain() {
  std::lock_guard<std::mutex> g(g_prof_mu);
  for (auto &r : g_prof_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      g_prof_ms[r.kind] += ms;
      g_prof_n[r.kind] += 1;
      g_prof_bytes[r.kind] += r.bytes;
    } else {
      cudaGetLastError();                 // not the caller's error to see later
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_prof_pending.clear();
}

int cuda_fail(cudaError_t e) {
  g_last_error = cudaGetErrorString(e);
  cudaGetLastError();                     // reported here; leave no stale error behind
  return POLAR_ECUDA;
}

#define CK(expr)                                   \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_);   \
  } while (0)

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// ---------------------------------------------------------------- workspace
// One scratch workspace per (device, stream), grown on demand.  In guard mode
// ("guard" = 1, a debugging aid) the allocation carries kGuard bytes of a
// fixed pattern before the workspace and again right after the bytes the
// current decode asked for; the synchronous decode entry points check both
// zones afterwards, so a kernel writing past either end of its scratch is
// reported as POLAR_EFAULT instead of passing silently.
constexpr size_t kGuard = 64 * 1024;
constexpr unsigned char kGuardByte = 0xA5;
struct Workspace {
  void *ptr = nullptr;        // workspace (after the leading guard zone, if any)
  size_t bytes = 0;           // capacity
  char *base = nullptr;       // allocation
  bool guarded = false;
  size_t last_req = 0;        // bytes of the latest request (trailing zone follows them)
};
std::mutex g_ws_mu;
std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;

int get_workspace(int dev, cudaStream_t s, size_t bytes, void **out) {
  std::lock_guard<std::mutex> g(g_ws_mu);
  Workspace &w = g_ws[{dev, s}];
  const bool guard = g_cfg.guard.load() != 0;
  bool fresh = false;
  if (w.bytes < bytes || w.guarded != guard) {
    fresh = true;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) {
      g_last_error = "scratch workspace must grow, but the stream is being captured";
      return POLAR_EINVAL;
    }
    if (w.base) {
      CK(cudaStreamSynchronize(s));
      cudaFree(w.base);
      w = Workspace{};
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes + (guard ? 2 * kGuard : 0));
    if (e != cudaSuccess) {
      cudaGetLastError();
      g_last_error = cudaGetErrorString(e);
      return POLAR_ENOMEM;
    }
    w.base = static_cast<char *>(p);
    w.ptr = w.base + (guard ? kGuard : 0);
    w.bytes = bytes;
    w.guarded = guard;
    if (guard) CK(cudaMemsetAsync(w.base, kGuardByte, kGuard, s));
  }
  if (w.guarded && (fresh || w.last_req != bytes)) {
    // the trailing zone follows the bytes this decode uses; it is written
    // when it moves and otherwise left as the last check found (or restored) it
    CK(cudaMemsetAsync(static_cast<char *>(w.ptr) + bytes, kGuardByte, kGuard, s));
    w.last_req = bytes;
  }
  *out = w.ptr;
  return POLAR_OK;
}

// Guard mode: wait for the stream, then check both guard zones of its
// workspace.  POLAR_EFAULT (with the first changed offset in the error text)
// if a kernel wrote outside its scratch.
int check_guard(cudaStream_t s) {
  if (g_cfg.guard.load() == 0) return POLAR_OK;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaStreamSynchronize(s));
  std::lock_guard<std::mutex> g(g_ws_mu);
  auto it = g_ws.find({dev, s});
  if (it == g_ws.end() || !it->second.guarded) return POLAR_OK;
  const Workspace &w = it->second;
  std::vector<unsigned char> h(kGuard);
  const char *zones[2] = {w.base, static_cast<const char *>(w.ptr) + w.last_req};
  const char *names[2] = {"before", "after"};
  for (int z = 0; z < 2; ++z) {
    CK(cudaMemcpy(h.data(), zones[z], kGuard, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < kGuard; ++i) {
      if (h[i] != kGuardByte) {
        char msg[160];
        std::snprintf(msg, sizeof msg,
                      "guard zone %s the scratch workspace overwritten at byte %zu (of %zu)",
                      names[z], i, kGuard);
        g_last_error = msg;
        CK(cudaMemset(const_cast<char *>(zones[z]), kGuardByte, kGuard));
        return POLAR_EFAULT;
      }
    }
  }
  return POLAR_OK;
}

// ---------------------------------------------------------------- graphs
using GraphKey = std::tuple<uint64_t, int, const void *, const void *, const void *, const void *,
                            int, int, int, int, cudaStream_t, int, const void *>;
struct GraphEntry {
  cudaGraphExec_t exec;
  uint64_t kernels;
};
std::mutex g_graph_mu;
std::list<std::pair<GraphKey, GraphEntry>> g_graphs;   // most recent first
constexpr size_t kMaxGraphs = 32;

// ---------------------------------------------------------------- decoding
struct Group {
  polar_frozen_set *fs;
  int nframes;
  const float *llr;
  const uint32_t *fv;
  uint32_t *xhat;
  uint32_t *uhat;
  int fkind, prec;
};

struct Exec {
  const Plan *plan;
  const Group *g;
  const uint32_t *dmask;
  void *ws;
  int n, t;
  const uint32_t *dclass;   // class table (shortcuts, t >= 5) or null
  const uint32_t *ducls = nullptr;   // upper class table (plans with node units)
};

// Workspace: [int8 scales, F floats rounded up to 256 B][levels t..n-1].
inline size_t scale_region(int nframes, int prec) {
  return prec == POLAR_INT8 ? ((size_t)nframes * sizeof(float) + 255) & ~size_t(255) : 0;
}

inline float *scale_ptr(const Exec &x) {
  return x.g->prec == POLAR_INT8 ? static_cast<float *>(x.ws) : nullptr;
}

inline void *level_ptr(const Exec &x, int k) {
  // levels t .. n-1 of all frames: level k at F * (2^k - 2^t) elements
  size_t off = (size_t)x.g->nframes * ((size_t(1) << k) - (size_t(1) << x.t));
  return static_cast<char *>(x.ws) + scale_region(x.g->nframes, x.g->prec) +
         off * storage_bytes(x.g->prec);
}

inline size_t workspace_bytes(int n, int t, int nframes, int prec) {
  size_t lv = n > t ? (size_t)nframes * ((size_t(1) << n) - (size_t(1) << t)) * storage_bytes(prec)
                    : 0;
  return scale_region(nframes, prec) + lv;
}

// One streamed f or g step (level op.k -> op.k - 1) over every frame.
int run_step(const Exec &x, const Op &op, cudaStream_t s, bool prof) {
  const Group &g = *x.g;
  const int n = x.n, k = op.k;
  const uint64_t N = uint64_t(1) << n;
  const size_t W = N >= 32 ? N / 32 : 1;
  const double F = g.nframes, sb = (double)storage_bytes(g.prec);
  float *scale = scale_ptr(x);
  const bool top = (k == n);
  const void *in = top ? static_cast<const void *>(g.llr) : level_ptr(x, k);
  const size_t ins = top ? N : (size_t(1) << k);
  void *out = level_ptr(x, k - 1);
  const uint64_t h = uint64_t(1) << (k - 1);
  const double inb = top ? 4.0 : sb;
  ProfScope ps(prof, op.kind == OP_F ? 1 : 2,
               F * (2.0 * h * inb + h * sb + (op.kind == OP_G ? h / 8.0 : 0.0)), s);
  if (op.kind == OP_F) {
    CK(launch_stream_f(g.prec, g.fkind, in, ins, top, out, h, h, g.nframes, scale, s));
  } else {
    CK(launch_stream_g(g.prec, in, ins, top, out, h, h, g.xhat, W, op.o, g.nframes, scale, s));
  }
  return POLAR_OK;
}

int run_ops(const Exec &x, cudaStream_t s, bool prof) {
  const Group &g = *x.g;
  const int n = x.n, t = x.t;
  const uint64_t N = uint64_t(1) << n;
  const size_t W = N >= 32 ? N / 32 : 1;
  const double F = g.nframes, sb = (double)storage_bytes(g.prec);
  float *scale = scale_ptr(x);
  if (scale) CK(launch_int8_scale(g.llr, N, g.nframes, (double)g_cfg.int8_target.load(), scale, s));
  for (const Op &op0 : x.plan->ops) {
    Op op = op0;
    if (op.kind == OP_ST && op.pad && g.prec != POLAR_FP32) {
      // reduced storage: the parent's step stays a streamed launch
      const Op step{(uint8_t)(op.pad == 1 ? OP_F : OP_G), (uint8_t)(t + 1), 0, 0,
                    op.pad == 1 ? op.o : op.o - (uint64_t(1) << t)};
      const int rc = run_step(x, step, s, prof);
      if (rc) return rc;
      op.pad = 0;
    }
    switch (op.kind) {
      case OP_F:
      case OP_G: {
        const int rc = run_step(x, op, s, prof);
        if (rc) return rc;
        break;
      }
      case OP_ST: {
        SubtreeArgs a;
        a.pre = op.pad;
        const int kin = op.pad ? t + 1 : t;   // level the kernel reads
        a.in_is_llr = (n == kin);
        a.in = a.in_is_llr ? static_cast<const void *>(g.llr) : level_ptr(x, kin);
        a.in_stride = a.in_is_llr ? N : (size_t(1) << kin);
        a.mask = x.dmask;
        a.cls = x.dclass ? x.dclass + (op.o >> t) * 2 * class_words(t) : nullptr;
        a.scale = scale;
        a.fv = g.fv;
        a.xhat = g.xhat;
        a.uhat = g.uhat;
        a.w_stride = W;
        a.o = op.o;
        a.t = t;
        a.r = op.r;
        a.nframes = g.nframes;
        a.fkind = g.fkind;
        a.prec = g.prec;
        a.shortcuts = x.plan->shortcuts;
        const double T = double(uint64_t(1) << t);
        double cb = 0;
        for (int m = 0; m < op.r; ++m) cb += 3.0 * double(uint64_t(1) << (t + m)) / 8.0;
        ProfScope ps(prof, 3,
                     F * ((op.pad ? 2.0 : 1.0) * T * (a.in_is_llr ? 4.0 : sb) +
                          T / 8.0 * (g.uhat ? 4 : 3) + (op.pad == 2 ? T / 8.0 : 0.0) + cb),
                     s);
        CK(launch_subtree(a, s));
        break;
      }
      case OP_CHAIN: {
        const int kt = op.k, kb = op.k - op.r;
        const bool top = (kt == n);
        const void *in = top ? static_cast<const void *>(g.llr) : level_ptr(x, kt);
        const size_t ins = top ? N : (size_t(1) << kt);
        const double inb = top ? 4.0 : sb;
        double outb = 0;
        for (int k = kb; k < kt; ++k) outb += double(uint64_t(1) << k) * sb;
        ProfScope ps(prof, 5,
                     F * (double(uint64_t(1) << kt) * inb + outb +
                          (op.pad ? double(uint64_t(1) << (kt - 1)) / 8.0 : 0.0)),
                     s);
        CK(launch_chain(g.prec, g.fkind, op.pad != 0, in, ins, top, level_ptr(x, t), t,
                        g.nframes, kt, kb, g.xhat, W, op.o, scale, s));
        break;
      }
      case OP_NODE: {
        NodeArgs a;
        a.lv = level_ptr(x, t);
        a.mask = x.dmask;
        a.cls = x.dclass;
        a.ucls = x.ducls;
        a.scale = scale;
        a.fv = g.fv;
        a.xhat = g.xhat;
        a.uhat = g.uhat;
        a.w_stride = W;
        a.o = op.o;
        a.s = op.k;
        a.t = t;
        a.n = n;
        a.r = op.r;
        a.nframes = g.nframes;
        a.fkind = g.fkind;
        a.prec = g.prec;
        if (!a.ucls || !a.cls) return POLAR_EINVAL;
        // per frame: the node's steps (each level read twice -- f and g --
        // and written once per node below it) and its subtrees' traffic
        const double S2 = double(uint64_t(1) << op.k), T = double(uint64_t(1) << t);
        double steps = 0;
        for (int k = t + 1; k <= op.k; ++k) steps += S2 * sb * 1.5 + (S2 / 2) / 8.0;
        double cb = 0;
        for (int m = 0; m < op.r; ++m) cb += 3.0 * double(uint64_t(1) << (op.k + m)) / 8.0;
        ProfScope ps(prof, 7, F * (steps + S2 / T * (T * sb + T / 8.0 * (g.uhat ? 4 : 3)) + cb),
                     s);
        CK(launch_node(a, s));
        break;
      }
      case OP_R0: {
        const size_t off = op.o >> 5, nw = size_t(1) << (op.k - 5);
        double cb = 0;
        for (int m = 0; m < op.r; ++m) cb += 3.0 * double(uint64_t(1) << (op.k + m)) / 8.0;
        ProfScope ps(prof, 4, F * (nw * 4.0 * (g.uhat ? 3 : 2) + cb), s);
        CK(launch_copy_regions(g.fv, g.xhat, W, off, nw, g.nframes, nullptr, s));
        if (g.uhat) CK(launch_copy_regions(g.fv, g.uhat, W, off, nw, g.nframes, nullptr, s));
        CK(launch_encode_regions(g.xhat, W, off, op.k, g.nframes, s));
        CK(launch_cascade(g.xhat, W, op.k, op.o, op.r, g.nframes, s));
        break;
      }
    }
  }
  return POLAR_OK;
}

int current_device(int *dev) {
  cudaError_t e = cudaGetDevice(dev);
  if (e != cudaSuccess) return cuda_fail(e);
  return POLAR_OK;
}

struct Opts {
  bool plain, shortcuts, graphs, profile, fuse, prologue;
  int subtree_log2;
  int split;                 // node-unit level (0: none)
};

Opts current_opts() {
  Opts o;
  o.plain = g_cfg.plain.load() != 0;
  o.shortcuts = !o.plain && g_cfg.shortcuts.load() != 0;
  o.graphs = !o.plain && g_cfg.graphs.load() != 0;
  o.profile = g_cfg.profile.load() != 0;
  o.fuse = !o.plain && g_cfg.fuse.load() != 0;
  o.prologue = !o.plain && g_cfg.prologue.load() != 0;
  o.subtree_log2 = (int)g_cfg.subtree_log2.load();
  o.split = o.plain ? 0 : (int)g_cfg.split_log2.load();
  return o;
}

// Options for one batch: the tuned (t, fuse) of its shape when autotuning is on.
Opts opts_for(const polar_frozen_set *fs, int nframes, int fkind, int prec) {
  Opts o = current_opts();
  if (o.plain || g_cfg.autotune.load() == 0) return o;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return o;
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_tune.find(TuneKey{dev, (int)fs->log2n, nframes, fkind, prec});
  if (it != g_tune.end()) {
    o.subtree_log2 = it->second.t;
    o.fuse = (it->second.fuse & 1) != 0;
    o.prologue = (it->second.fuse & 2) != 0;
    o.split = (it->second.fuse >> 8) & 0xFF;
  }
  return o;
}

int decode_group(const Group &g, cudaStream_t s, const Opts &opt) {
  NvtxRange nv("polar decode batch");
  polar_frozen_set *fs = g.fs;
  const int n = (int)fs->log2n;
  const bool plain = opt.plain;
  const bool shortcuts = opt.shortcuts;
  const bool graphs = opt.graphs;
  const int t = std::min<int>(n, opt.subtree_log2);
  int dev = 0;
  int rc = current_device(&dev);
  if (rc) return rc;
  cudaError_t e;
  const uint32_t *dmask = device_mask(fs, dev, &e);
  if (!dmask) return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : cuda_fail(e);
  std::shared_ptr<Plan> plan =
      get_plan(fs, t, shortcuts, opt.fuse, opt.prologue, plain ? 0 : opt.split);
  const uint32_t *dclass = nullptr;
  if (shortcuts && t >= 5) {
    dclass = device_class_table(fs, dev, t, &e);
    if (!dclass) return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : cuda_fail(e);
  }
  const uint32_t *ducls = nullptr;
  if (plan->n_node > 0) {
    ducls = device_upper_class_table(fs, dev, t, &e);
    if (!ducls) return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : cuda_fail(e);
  }
  const int F = plain ? 1 : g.nframes;
  size_t ws_bytes = workspace_bytes(n, t, F, g.prec);
  void *ws = nullptr;
  if (ws_bytes) {
    rc = get_workspace(dev, s, ws_bytes, &ws);
    if (rc) return rc;
  }
  if (plain) {
    const uint64_t N = uint64_t(1) << n;
    const size_t W = N >= 32 ? N / 32 : 1;
    for (int f = 0; f < g.nframes; ++f) {
      Group one = g;
      one.nframes = 1;
      one.llr = g.llr + (size_t)f * N;
      one.fv = g.fv + (size_t)f * W;
      one.xhat = g.xhat + (size_t)f * W;
      one.uhat = g.uhat ? g.uhat + (size_t)f * W : nullptr;
      Exec x{plan.get(), &one, dmask, ws, n, t, dclass, ducls};
      rc = run_ops(x, s, opt.profile);
      if (rc) return rc;
    }
    return POLAR_OK;
  }
  Exec x{plan.get(), &g, dmask, ws, n, t, dclass, ducls};
  const bool prof = opt.profile;
  bool use_graph = graphs && s != nullptr;
  if (use_graph) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) use_graph = false;   // caller is capturing
  }
  if (prof && use_graph && g_cfg.profile.load() == 1) {
    // One-off replay of the same schedule with an event-record node around
    // every kernel group, so that the per-kind times are the graph's device
    // times, without the host's launch gaps.
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    const uint64_t before = g_kernel_launches.load();
    rc = run_ops(x, s, true);
    const uint64_t kernels = g_kernel_launches.load() - before;
    g_kernel_launches.fetch_sub(kernels);
    cudaGraph_t graph = nullptr;
    cudaError_t ee = cudaStreamEndCapture(s, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ee != cudaSuccess) return cuda_fail(ee);
    cudaGraphExec_t exec = nullptr;
    ee = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ee != cudaSuccess) return cuda_fail(ee);
    ee = cudaGraphLaunch(exec, s);
    cudaGraphExecDestroy(exec);             // the launched replay still completes
    if (ee != cudaSuccess) return cuda_fail(ee);
    g_kernel_launches.fetch_add(kernels);
    return POLAR_OK;
  }
  if (prof || !use_graph) return run_ops(x, s, prof);

  GraphKey key{fs->id, g.nframes, g.llr, g.fv, g.xhat, g.uhat, g.fkind, g.prec, t,
               (shortcuts ? 1 : 0) | (opt.fuse ? 2 : 0) | (g_pdl.load() ? 4 : 0) |
                   (opt.prologue ? 8 : 0) | (plan->split << 8),
               s, dev, ws};
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;
  {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it) {
      if (it->first == key) {
        exec = it->second.exec;
        kernels = it->second.kernels;
        g_graphs.splice(g_graphs.begin(), g_graphs, it);
        break;
      }
    }
  }
  if (!exec) {
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    const uint64_t before = g_kernel_launches.load();
    rc = run_ops(x, s, false);
    kernels = g_kernel_launches.load() - before;
    g_kernel_launches.fetch_sub(kernels);   // captured, not yet run
    cudaGraph_t graph = nullptr;
    cudaError_t ee = cudaStreamEndCapture(s, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ee != cudaSuccess) return cuda_fail(ee);
    ee = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ee != cudaSuccess) return cuda_fail(ee);
    std::lock_guard<std::mutex> lk(g_graph_mu);
    g_graphs.emplace_front(key, GraphEntry{exec, kernels});
    if (g_graphs.size() > kMaxGraphs) {
      cudaGraphExecDestroy(g_graphs.back().second.exec);
      g_graphs.pop_back();
    }
  }
  CK(cudaGraphLaunch(exec, s));
  g_kernel_launches.fetch_add(kernels);
  return POLAR_OK;
}

int check_group(const Group &g) {
  if (!g.fs || g.nframes < 1 || !g.llr || !g.fv || !g.xhat) return POLAR_EINVAL;
  if (g.fkind != POLAR_F_MINSUM && g.fkind != POLAR_F_EXACT) return POLAR_EINVAL;
  if (g.prec != POLAR_FP32 && g.prec != POLAR_FP16 && g.prec != POLAR_INT8) return POLAR_EINVAL;
  if (!aligned(g.llr, 16) || !aligned(g.fv, 4) || !aligned(g.xhat, 4)) return POLAR_EINVAL;
  if (g.uhat && !aligned(g.uhat, 4)) return POLAR_EINVAL;
  return POLAR_OK;
}

int check_frames(int nframes, const polar_frame_desc *frames, int fkind, int prec) {
  if (nframes < 1 || !frames) return POLAR_EINVAL;
  for (int i = 0; i < nframes; ++i) {
    Group one{const_cast<polar_frozen_set *>(frames[i].fs), 1, frames[i].llr,
              frames[i].frozen_vals, frames[i].xhat, frames[i].uhat, fkind, prec};
    int rc = check_group(one);
    if (rc) return rc;
  }
  return POLAR_OK;
}

// Whole frames per CTA from a device queue (persist.cu).  The queue is
// ordered longest first so that the long frames start early and the short
// ones fill in behind them.
int decode_persistent(int nframes, const polar_frame_desc *frames, int fkind, int prec,
                      cudaStream_t s) {
  NvtxRange nv("polar decode persistent");
  if (prec != POLAR_FP32 && prec != POLAR_FP16 && prec != POLAR_INT8) return POLAR_EINVAL;
  int dev = 0;
  int rc = current_device(&dev);
  if (rc) return rc;
  const int tc = (int)g_cfg.persist_log2.load();
  std::vector<int> order(nframes);
  for (int i = 0; i < nframes; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return frames[a].fs->log2n > frames[b].fs->log2n;
  });
  std::vector<PFrame> h(nframes);
  int nmax = 0;
  bool uh = false;
  double alg = 0;
  for (int j = 0; j < nframes; ++j) {
    const polar_frame_desc &d = frames[order[j]];
    polar_frozen_set *fs = const_cast<polar_frozen_set *>(d.fs);
    const int n = (int)fs->log2n, t = std::min(n, tc);
    cudaError_t e = cudaSuccess;
    PFrame &p = h[j];
    p.llr = d.llr;
    p.fv = d.frozen_vals;
    p.xhat = d.xhat;
    p.uhat = d.uhat;
    p.log2n = (uint32_t)n;
    p.t = (uint32_t)t;
    p.mask = device_mask(fs, dev, &e);
    if (!p.mask) return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : cuda_fail(e);
    p.cls = nullptr;
    if (t >= 5) {
      p.cls = device_class_table(fs, dev, t, &e);
      if (!p.cls) return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : cuda_fail(e);
    }
    p.ucls = nullptr;
    if (n > t) {
      p.ucls = device_upper_class_table(fs, dev, t, &e);
      if (!p.ucls) return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : cuda_fail(e);
    }
    nmax = std::max(nmax, n);
    uh |= d.uhat != nullptr;
    const double N = double(uint64_t(1) << n), sl = n - t;
    alg += (3.0 * sl + 1.0) * N * (double)storage_bytes(prec) + (0.3125 * sl + 0.375) * N;
  }
  const int per_sm = persistent_ctas_per_sm(prec, fkind, uh, tc);
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (per_sm < 1 || sms < 1) {
    g_last_error = "persistent decoder: no resident CTA fits on an SM";
    return POLAR_ECUDA;
  }
  const int grid = std::min(nframes, per_sm * sms);
  uint64_t cta_floats = nmax > tc ? (uint64_t(1) << nmax) - (uint64_t(1) << tc) : 0;
  cta_floats = (cta_floats + 63) & ~uint64_t(63);
  const size_t tab = ((size_t)nframes * sizeof(PFrame) + 255) & ~size_t(255);
  const size_t bytes = 256 + tab + (size_t)grid * cta_floats * sizeof(float);
  void *ws = nullptr;
  rc = get_workspace(dev, s, bytes, &ws);
  if (rc) return rc;
  uint32_t *head = static_cast<uint32_t *>(ws);
  PFrame *ftab = reinterpret_cast<PFrame *>(static_cast<char *>(ws) + 256);
  float *scratch = reinterpret_cast<float *>(static_cast<char *>(ws) + 256 + tab);
  CK(cudaMemsetAsync(head, 0, sizeof(uint32_t), s));
  CK(cudaMemcpyAsync(ftab, h.data(), (size_t)nframes * sizeof(PFrame), cudaMemcpyHostToDevice,
                     s));
  ProfScope ps(g_cfg.profile.load() != 0, 6, alg, s);
  CK(launch_persistent(prec, fkind, uh, ftab, (uint32_t)nframes, head, scratch, cta_floats, tc,
                       grid, (double)g_cfg.int8_target.load(), s));
  return POLAR_OK;
}

}  // namespace

namespace polar {

// Levels t..n-1 of nframes frames at the current "subtree_log2", in bytes.
size_t level_scratch_bytes(const polar_frozen_set *fs, int nframes, int prec, int *t_out) {
  const int n = (int)fs->log2n;
  const int t = std::min<int>(n, (int)g_cfg.subtree_log2.load());
  if (t_out) *t_out = t;
  return workspace_bytes(n, t, nframes, prec);
}

// Options of a decode that runs in caller-supplied scratch, read once so
// that the sizing and the launches see the same subtree size and shortcut
// setting even if another thread changes the configuration in between.  The
// subtree size is the autotuned one for this batch shape when the tuner has
// an entry, as in polar_sc_decode_many.
ScratchOpts scratch_opts(const polar_frozen_set *fs, int nframes, int fkind, int prec) {
  const Opts o = opts_for(fs, nframes, fkind, prec);
  ScratchOpts so;
  so.t = std::min<int>((int)fs->log2n, o.subtree_log2);
  so.shortcuts = o.shortcuts;
  so.fuse = o.fuse;
  so.prologue = o.prologue;
  return so;
}

size_t scratch_level_bytes(const polar_frozen_set *fs, int nframes, int prec, int t) {
  return workspace_bytes((int)fs->log2n, t, nframes, prec);
}

// One batch decoded with launches only: the caller supplies the device mask
// and the level scratch, so no device memory is allocated and no graph is
// built.  Host-side the cached schedule of the frozen set is reused.
int decode_with_scratch(const polar_frozen_set *fs_c, int nframes, const float *llr,
                        const uint32_t *fv, uint32_t *xhat, uint32_t *uhat, int fkind, int prec,
                        const ScratchOpts &o, const uint32_t *dmask, const uint32_t *dclass,
                        void *scratch, size_t scratch_bytes, cudaStream_t s) {
  polar_frozen_set *fs = const_cast<polar_frozen_set *>(fs_c);
  Group g{fs, nframes, llr, fv, xhat, uhat, fkind, prec};
  int rc = check_group(g);
  if (rc) return rc;
  const int t = o.t;
  if (t < 1 || t > (int)fs->log2n) return POLAR_EINVAL;
  if (scratch_level_bytes(fs, nframes, prec, t) > scratch_bytes) return POLAR_EINVAL;
  if (o.shortcuts && t >= 5 && !dclass) return POLAR_EINVAL;
  std::shared_ptr<Plan> plan = get_plan(fs, t, o.shortcuts, o.fuse, o.prologue);
  Exec x{plan.get(), &g, dmask, scratch, (int)fs->log2n, t,
         o.shortcuts && t >= 5 ? dclass : nullptr};
  return run_ops(x, s, false);
}

void set_last_error(const char *msg) { g_last_error = msg; }

int prepare_tables(polar_frozen_set *fs, int dev, int t, bool upper) {
  int prev = 0;
  CK(cudaGetDevice(&prev));
  if (prev != dev) CK(cudaSetDevice(dev));
  const int n = (int)fs->log2n, tt = std::min(n, t);
  cudaError_t e = cudaSuccess;
  bool ok = device_mask(fs, dev, &e) != nullptr;
  if (ok && tt >= 5) ok = device_class_table(fs, dev, tt, &e) != nullptr;
  if (ok && upper && n > tt) ok = device_upper_class_table(fs, dev, tt, &e) != nullptr;
  if (prev != dev) cudaSetDevice(prev);
  if (ok) return POLAR_OK;
  return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : cuda_fail(e);
}

bool log_on() {
  static const bool on = [] {
    const char *v = std::getenv("POLAR_LOG");
    return v && *v && std::strcmp(v, "0") != 0;
  }();
  return on;
}

void log_msg(const char *fmt, ...) {
  if (!log_on()) return;
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  std::fprintf(stderr, "[polar] %s\n", buf);
}

// Eager decode (no graphs, no plain mode) for callers that launch many
// unrelated small batches, such as the request server.
int decode_eager(const polar_frozen_set *fs, int nframes, const float *llr, const uint32_t *fv,
                 uint32_t *xhat, uint32_t *uhat, int fkind, int prec, cudaStream_t s) {
  Group g{const_cast<polar_frozen_set *>(fs), nframes, llr, fv, xhat, uhat, fkind, prec};
  int rc = check_group(g);
  if (rc) return rc;
  Opts o = current_opts();
  o.plain = false;
  o.graphs = false;
  o.profile = false;
  o.shortcuts = g_cfg.shortcuts.load() != 0;
  return decode_group(g, s, o);
}

void release_stream_workspace(int dev, cudaStream_t s) {
  std::lock_guard<std::mutex> g(g_ws_mu);
  auto it = g_ws.find({dev, s});
  if (it == g_ws.end()) return;
  if (it->second.base) cudaFree(it->second.base);
  g_ws.erase(it);
}

size_t decode_scratch_bytes(const polar_frozen_set *fs, int nframes, int prec) {
  return level_scratch_bytes(fs, nframes, prec, nullptr);
}

}  // namespace polar

// ====================================================================== ABI
extern "C" {

const char *polar_strerror(int status) {
  switch (status) {
    case POLAR_OK: return "ok";
    case POLAR_EINVAL: return "invalid argument";
    case POLAR_ENOMEM: return "out of memory";
    case POLAR_ECUDA: return "CUDA error";
    case POLAR_ETIMEDOUT: return "device wait timed out";
    case POLAR_EBUSY: return "admission refused";
    case POLAR_ENOTFOUND: return "not found";
    case POLAR_ECANCELED: return "cancelled";
    case POLAR_EFAULT: return "out-of-range write detected (guard mode)";
    case POLAR_PENDING: return "pending";
    default: return "unknown status";
  }
}

const char *polar_last_error_string(void) { return g_last_error.c_str(); }

int polar_config_set(const char *key, long value) {
  if (!key) return POLAR_EINVAL;
  if (!strcmp(key, "subtree_log2")) {
    if (value < 5 || value > 14) return POLAR_EINVAL;
    g_cfg.subtree_log2 = value;
  } else if (!strcmp(key, "shortcuts")) {
    g_cfg.shortcuts = value ? 1 : 0;
  } else if (!strcmp(key, "graphs")) {
    g_cfg.graphs = value ? 1 : 0;
  } else if (!strcmp(key, "plain")) {
    g_cfg.plain = value ? 1 : 0;
  } else if (!strcmp(key, "profile")) {
    if (value < 0 || value > 2) return POLAR_EINVAL;
    g_cfg.profile = value;
  } else if (!strcmp(key, "fuse")) {
    g_cfg.fuse = value ? 1 : 0;
  } else if (!strcmp(key, "prologue")) {
    g_cfg.prologue = value ? 1 : 0;
  } else if (!strcmp(key, "autotune")) {
    g_cfg.autotune = value ? 1 : 0;
  } else if (!strcmp(key, "int8_target")) {
    if (value < 1 || value > 64) return POLAR_EINVAL;
    g_cfg.int8_target = value;
  } else if (!strcmp(key, "pdl")) {
    g_pdl = value ? 1 : 0;
  } else if (!strcmp(key, "persist_log2")) {
    if (value < 5 || value > 14) return POLAR_EINVAL;
    g_cfg.persist_log2 = value;
  } else if (!strcmp(key, "persistent")) {
    if (value < 0 || value > 2) return POLAR_EINVAL;
    g_cfg.persistent = value;
  } else if (!strcmp(key, "guard")) {
    g_cfg.guard = value ? 1 : 0;
  } else if (!strcmp(key, "split_log2")) {
    if (value != 0 && (value < 6 || value > 27)) return POLAR_EINVAL;
    g_cfg.split_log2 = value;
  } else {
    return POLAR_ENOTFOUND;
  }
  return POLAR_OK;
}

int polar_config_get(const char *key, long *value) {
  if (!key || !value) return POLAR_EINVAL;
  if (!strcmp(key, "subtree_log2")) *value = g_cfg.subtree_log2;
  else if (!strcmp(key, "shortcuts")) *value = g_cfg.shortcuts;
  else if (!strcmp(key, "graphs")) *value = g_cfg.graphs;
  else if (!strcmp(key, "plain")) *value = g_cfg.plain;
  else if (!strcmp(key, "profile")) *value = g_cfg.profile;
  else if (!strcmp(key, "int8_target")) *value = g_cfg.int8_target;
  else if (!strcmp(key, "fuse")) *value = g_cfg.fuse;
  else if (!strcmp(key, "prologue")) *value = g_cfg.prologue;
  else if (!strcmp(key, "autotune")) *value = g_cfg.autotune;
  else if (!strcmp(key, "persistent")) *value = g_cfg.persistent;
  else if (!strcmp(key, "persist_log2")) *value = g_cfg.persist_log2;
  else if (!strcmp(key, "pdl")) *value = g_pdl.load();
  else if (!strcmp(key, "guard")) *value = g_cfg.guard;
  else if (!strcmp(key, "split_log2")) *value = g_cfg.split_log2;
  else return POLAR_ENOTFOUND;
  return POLAR_OK;
}

uint64_t polar_kernel_launches(void) { return g_kernel_launches.load(); }

int polar_profile_read(const char *kind, double *total_ms, uint64_t *launches,
                       double *alg_bytes) {
  if (!kind) return POLAR_EINVAL;
  prof_drain();
  for (int i = 0; i < kNumKinds; ++i) {
    if (!strcmp(kind, kKinds[i])) {
      std::lock_guard<std::mutex> g(g_prof_mu);
      if (total_ms) *total_ms = g_prof_ms[i];
      if (launches) *launches = g_prof_n[i];
      if (alg_bytes) *alg_bytes = g_prof_bytes[i];
      return POLAR_OK;
    }
  }
  return POLAR_ENOTFOUND;
}

void polar_profile_reset(void) {
  prof_drain();
  std::lock_guard<std::mutex> g(g_prof_mu);
  for (int i = 0; i < kNumKinds; ++i) {
    g_prof_ms[i] = 0;
    g_prof_n[i] = 0;
    g_prof_bytes[i] = 0;
  }
}

namespace {
// Logs one construction: what was asked, the resulting K and the time taken.
int logged_build(const char *what, uint32_t log2n, polar_channel ch, double param,
                 polar_frozen_set **out, int rc, std::chrono::steady_clock::time_point t0) {
  if (polar::log_on()) {
    const double s =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    polar::log_msg("frozen set (%s): log2n %u, %s %.6g -> status %d, K %llu, %.3f s", what,
                   log2n, ch == POLAR_BSC ? "bsc" : "biawgn", param, rc,
                   rc == POLAR_OK && out && *out ? (unsigned long long)(*out)->K : 0ull, s);
  }
  return rc;
}
}  // namespace

int polar_build_frozen_set(uint32_t log2n, polar_channel ch, double param, double rate,
                           polar_frozen_set **out) {
  const auto t0 = std::chrono::steady_clock::now();
  return logged_build("rate", log2n, ch, param, out,
                      build_frozen_set(log2n, ch, param, rate, out), t0);
}

int polar_build_frozen_set_sum(uint32_t log2n, polar_channel ch, double param,
                               double sum_pe_max, polar_frozen_set **out) {
  const auto t0 = std::chrono::steady_clock::now();
  return logged_build("sum rule", log2n, ch, param, out,
                      build_frozen_set_sum(log2n, ch, param, sum_pe_max, out), t0);
}

int polar_build_frozen_set_tv(uint32_t log2n, polar_channel ch, double param, int mu,
                              double rate, double sum_pe_max, polar_frozen_set **out) {
  const auto t0 = std::chrono::steady_clock::now();
  return logged_build("degraded", log2n, ch, param, out,
                      build_frozen_set_tv(log2n, ch, param, mu, rate, sum_pe_max, out), t0);
}

int polar_frozen_set_from_mask(uint32_t log2n, const uint32_t *mask_host,
                               polar_frozen_set **out) {
  return frozen_set_from_mask(log2n, mask_host, out);
}

int polar_frozen_set_upload(const polar_frozen_set *fs_c, int device) {
  if (!fs_c || device < 0) return POLAR_EINVAL;
  int count = 0;
  CK(cudaGetDeviceCount(&count));
  if (device >= count) return POLAR_EINVAL;
  polar_frozen_set *fs = const_cast<polar_frozen_set *>(fs_c);
  const int ts[] = {(int)g_cfg.subtree_log2.load(), 12, 13, 14};
  for (int t : ts) {
    const int rc = prepare_tables(fs, device, t, false);
    if (rc) return rc;
  }
  return prepare_tables(fs, device, (int)g_cfg.persist_log2.load(), true);
}

int polar_frozen_set_query(const polar_frozen_set *fs, uint32_t *log2n, uint64_t *k,
                           uint32_t *mask_host, double *sum_pe_info) {
  if (!fs) return POLAR_EINVAL;
  if (log2n) *log2n = fs->log2n;
  if (k) *k = fs->K;
  if (mask_host) std::memcpy(mask_host, fs->mask.data(), fs->mask.size() * sizeof(uint32_t));
  if (sum_pe_info) *sum_pe_info = fs->sum_pe;
  return POLAR_OK;
}

void polar_frozen_set_free(polar_frozen_set *fs) {
  if (!fs) return;
  {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end();) {
      if (std::get<0>(it->first) == fs->id) {
        cudaGraphExecDestroy(it->second.exec);
        it = g_graphs.erase(it);
      } else {
        ++it;
      }
    }
  }
  for (auto &kv : fs->dmask) cudaFree(kv.second);
  for (auto &kv : fs->dclass) cudaFree(kv.second);
  for (auto &kv : fs->ducls) cudaFree(kv.second);
  delete fs;
}

int polar_llr_from_channel(polar_channel ch, double param, const void *y_dev, int y_is_bits,
                           float *llr_dev, size_t n_total, void *stream) {
  if (!y_dev || !llr_dev) return POLAR_EINVAL;
  if (n_total == 0) return POLAR_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (ch == POLAR_BSC) {
    if (!y_is_bits || !(param > 0.0 && param < 0.5) || n_total % 32) return POLAR_EINVAL;
    if (!aligned(y_dev, 4) || !aligned(llr_dev, 16)) return POLAR_EINVAL;
    const float c = (float)std::log((1.0 - param) / param);
    ProfScope ps(g_cfg.profile.load() != 0, 0, n_total / 8.0 + 4.0 * n_total, s);
    CK(launch_llr_bsc(static_cast<const uint32_t *>(y_dev), llr_dev, n_total, c, s));
    return POLAR_OK;
  }
  if (ch == POLAR_BIAWGN) {
    if (y_is_bits || !(param > 0.0 && std::isfinite(param))) return POLAR_EINVAL;
    if (!aligned(y_dev, 16) || !aligned(llr_dev, 8)) return POLAR_EINVAL;
    ProfScope ps(g_cfg.profile.load() != 0, 0, 12.0 * n_total, s);
    CK(launch_llr_biawgn(static_cast<const double *>(y_dev), llr_dev, n_total, 2.0 / param, s));
    return POLAR_OK;
  }
  return POLAR_EINVAL;
}

int polar_frame_hash(uint32_t log2n, int nframes, const uint32_t *words_dev, uint64_t key,
                     uint64_t *hash_dev, void *stream) {
  if (log2n < 1 || log2n > 27 || nframes < 1 || !words_dev || !hash_dev) return POLAR_EINVAL;
  if (!aligned(words_dev, 4) || !aligned(hash_dev, 8)) return POLAR_EINVAL;
  const size_t W = log2n >= 5 ? (size_t(1) << (log2n - 5)) : 1;
  CK(launch_frame_hash(words_dev, W, W, nframes, key, hash_dev,
                       static_cast<cudaStream_t>(stream)));
  return POLAR_OK;
}

double polar_key_rate(double alpha, double fer, double beta, double mutual_info,
                      double eve_info) {
  return alpha * (1.0 - fer) * (beta * mutual_info - eve_info);
}

int polar_encode(uint32_t log2n, int nframes, const uint32_t *in_dev, uint32_t *out_dev,
                 void *stream) {
  if (log2n < 1 || log2n > 27 || nframes < 1 || !in_dev || !out_dev) return POLAR_EINVAL;
  if (!aligned(in_dev, 4) || !aligned(out_dev, 4)) return POLAR_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t W = log2n >= 5 ? (size_t(1) << (log2n - 5)) : 1;
  if (in_dev != out_dev) CK(launch_copy_regions(in_dev, out_dev, W, 0, W, nframes, nullptr, s));
  CK(launch_encode_regions(out_dev, W, 0, (int)log2n, nframes, s));
  return POLAR_OK;
}

int polar_reveal(const polar_frozen_set *fs_c, int nframes, const uint32_t *x_dev,
                 uint32_t *fval_dev, void *stream) {
  if (!fs_c || nframes < 1 || !x_dev || !fval_dev) return POLAR_EINVAL;
  if (!aligned(x_dev, 4) || !aligned(fval_dev, 4)) return POLAR_EINVAL;
  polar_frozen_set *fs = const_cast<polar_frozen_set *>(fs_c);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  int rc = current_device(&dev);
  if (rc) return rc;
  cudaError_t e;
  const uint32_t *dmask = device_mask(fs, dev, &e);
  if (!dmask) return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : cuda_fail(e);
  const size_t W = fs->mask.size();
  if (x_dev != fval_dev) CK(launch_copy_regions(x_dev, fval_dev, W, 0, W, nframes, nullptr, s));
  CK(launch_encode_regions(fval_dev, W, 0, (int)fs->log2n, nframes, s));
  CK(launch_copy_regions(fval_dev, fval_dev, W, 0, W, nframes, dmask, s));
  return POLAR_OK;
}

int polar_build_frozen_set_device(uint32_t log2n, polar_channel ch, double param, double rate,
                                  double sum_pe_max, void *stream, polar_frozen_set **out) {
  return build_frozen_set_device(log2n, ch, param, rate, sum_pe_max,
                                 static_cast<cudaStream_t>(stream), out);
}

int polar_sc_decode_many(const polar_frozen_set *fs, int nframes, const float *llr_dev,
                         const uint32_t *frozen_vals_dev, uint32_t *xhat_dev, uint32_t *uhat_dev,
                         polar_fkind fkind, polar_prec prec, void *stream) {
  Group g{const_cast<polar_frozen_set *>(fs), nframes, llr_dev, frozen_vals_dev, xhat_dev,
          uhat_dev, (int)fkind, (int)prec};
  int rc = check_group(g);
  if (rc) return rc;
  rc = decode_group(g, static_cast<cudaStream_t>(stream),
                    opts_for(g.fs, g.nframes, g.fkind, g.prec));
  return rc ? rc : check_guard(static_cast<cudaStream_t>(stream));
}

int polar_sc_decode(const polar_frozen_set *fs, const float *llr_dev,
                    const uint32_t *frozen_vals_dev, uint32_t *xhat_dev, uint32_t *uhat_dev,
                    polar_fkind fkind, polar_prec prec, void *stream) {
  return polar_sc_decode_many(fs, 1, llr_dev, frozen_vals_dev, xhat_dev, uhat_dev, fkind, prec,
                              stream);
}

int polar_autotune(const polar_frozen_set *fs_c, int nframes, const float *llr_dev,
                   const uint32_t *frozen_vals_dev, uint32_t *xhat_dev, polar_fkind fkind,
                   polar_prec prec, void *stream, int *best_t, int *best_fuse, double *best_ms) {
  NvtxRange nv("polar autotune");
  Group g{const_cast<polar_frozen_set *>(fs_c), nframes, llr_dev, frozen_vals_dev, xhat_dev,
          nullptr, (int)fkind, (int)prec};
  int rc = check_group(g);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n = (int)g.fs->log2n;
  // FP16 / INT8 round the levels >= t, so t changes their results: tune only
  // the fused / unfused streamed steps there.
  std::vector<int> ts;
  if (prec == POLAR_FP32 && n > 12) {
    for (int t = 12; t <= 14 && t <= n; ++t) ts.push_back(t);
  } else {
    ts.push_back(std::min<int>(n, (int)g_cfg.subtree_log2.load()));
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // schedule flags: bit 0 = fused streamed steps, bit 1 = the subtree kernel
  // takes its parent's step (float32 only; reduced storage keeps that step
  // streamed, so the flag would change nothing there)
  const int nflags = prec == POLAR_FP32 ? 4 : 2;
  TuneVal best{ts[0], 1, 1e30};
  // Mean device time of one decode with options o over `reps` decodes (after
  // warm-up decodes that build the workspace, plan and graph).
  auto timed = [&](const Opts &o, double *ms_out, int reps = 3) -> int {
    int r = POLAR_OK;
    for (int rep = 0; rep < 2 && !r; ++rep) r = decode_group(g, s, o);
    if (r) return r;
    CK(cudaEventRecord(e0, s));
    for (int rep = 0; rep < reps && !r; ++rep) r = decode_group(g, s, o);
    if (r) return r;
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    *ms_out = ms / reps;
    return POLAR_OK;
  };
  std::vector<TuneVal> tried;   // every schedule timed, for the final round
  auto base_opts = [&](int t) {
    Opts o = current_opts();
    o.plain = false;
    o.profile = false;
    o.subtree_log2 = t;
    o.split = 0;
    return o;
  };
  // phase 1: subtree size and streamed-step flags
  for (int t : ts) {
    for (int flags = 0; flags < nflags && !rc; ++flags) {
      Opts o = base_opts(t);
      o.fuse = (flags & 1) != 0;
      o.prologue = (flags & 2) != 0;
      double ms = 0;
      rc = timed(o, &ms);
      if (!rc) tried.push_back(TuneVal{t, flags, ms});
      if (!rc && ms < best.ms) best = TuneVal{t, flags, ms};
    }
    if (rc) break;
  }
  // phase 2: node units of 2^s leaves at that subtree size (the levels s..t+1
  // inside one CTA per frame; results are the same bits); bits 8..15 of the
  // flags carry s
  if (!rc && g_cfg.shortcuts.load() != 0 && best.t >= 5) {
    for (int sp = best.t + 1; sp <= std::min(n - 1, best.t + 4) && !rc; ++sp) {
      for (int fu = 0; fu < 2 && !rc; ++fu) {
        Opts o = base_opts(best.t);
        o.fuse = fu != 0;
        o.prologue = false;
        o.split = sp;
        double ms = 0;
        rc = timed(o, &ms);
        if (!rc) tried.push_back(TuneVal{best.t, fu | (sp << 8), ms});
        if (!rc && ms < best.ms) best = TuneVal{best.t, fu | (sp << 8), ms};
      }
    }
  }
  // final round: schedules within 4 % of the best are timed again over more
  // decodes (neighbouring schedules often differ by 1-3 %, about the spread
  // of a three-decode mean), and the fastest of that round is kept
  if (!rc && tried.size() > 1) {
    std::vector<TuneVal> close;
    for (const TuneVal &c : tried)
      if (c.ms <= best.ms * 1.04) close.push_back(c);
    if (close.size() > 1) {
      best.ms = 1e30;
      for (const TuneVal &c : close) {
        Opts o = base_opts(c.t);
        o.fuse = (c.fuse & 1) != 0;
        o.prologue = (c.fuse & 2) != 0;
        o.split = (c.fuse >> 8) & 0xFF;
        double ms = 0;
        rc = timed(o, &ms, 8);
        if (rc) break;
        if (ms < best.ms) best = TuneVal{c.t, c.fuse, ms};
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[TuneKey{dev, n, nframes, (int)fkind, (int)prec}] = best;
  }
  log_msg("autotune: log2n %d, %d frames, fkind %d, prec %d -> t %d, fused %d, subtree takes "
          "parent step %d, node units 2^%d, %.3f ms per decode", n, nframes, (int)fkind,
          (int)prec, best.t, best.fuse & 1, (best.fuse >> 1) & 1, (best.fuse >> 8) & 0xFF,
          best.ms);
  if (best_t) *best_t = best.t;
  if (best_fuse) *best_fuse = best.fuse;
  if (best_ms) *best_ms = best.ms;
  return POLAR_OK;
}

int polar_tune_save(const char *path) {
  if (!path) return POLAR_EINVAL;
  FILE *f = fopen(path, "w");
  if (!f) return POLAR_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  fprintf(f, "{\"polar_tune\": [\n");
  size_t i = 0;
  for (auto &kv : g_tune) {
    fprintf(f,
            "  {\"device\": %d, \"log2n\": %d, \"nframes\": %d, \"fkind\": %d, "
            "\"prec\": %d, \"subtree_log2\": %d, \"fuse\": %d, \"ms\": %.6f}%s\n",
            kv.first.dev, kv.first.log2n, kv.first.nframes, kv.first.fkind, kv.first.prec,
            kv.second.t, kv.second.fuse, kv.second.ms, ++i < g_tune.size() ? "," : "");
  }
  fprintf(f, "]}\n");
  fclose(f);
  log_msg("tune cache: saved %zu entries to %s", g_tune.size(), path);
  return POLAR_OK;
}

int polar_tune_load(const char *path) {
  if (!path) return POLAR_EINVAL;
  FILE *f = fopen(path, "r");
  if (!f) return POLAR_ENOTFOUND;
  char line[512];
  int loaded = 0;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  while (fgets(line, sizeof line, f)) {
    TuneKey k;
    TuneVal v;
    if (sscanf(line,
               " {\"device\": %d, \"log2n\": %d, \"nframes\": %d, \"fkind\": %d, "
               "\"prec\": %d, \"subtree_log2\": %d, \"fuse\": %d, \"ms\": %lf",
               &k.dev, &k.log2n, &k.nframes, &k.fkind, &k.prec, &v.t, &v.fuse, &v.ms) == 8) {
      const int split = (v.fuse >> 8) & 0xFF;   // node-unit level (0: none)
      if (v.t < 5 || v.t > 14 || v.fuse < 0 || (v.fuse & ~0xFF03) != 0 ||
          (split != 0 && (split <= v.t || split > 27)))
        continue;
      g_tune[k] = v;
      ++loaded;
    }
  }
  fclose(f);
  log_msg("tune cache: loaded %d entries from %s", loaded, path);
  return loaded > 0 ? POLAR_OK : POLAR_ENOTFOUND;
}

void polar_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
}

// Frames [i, j) that decode_batch runs as one group: same frozen set and
// equally strided buffers.
static int group_end(int nframes, const polar_frame_desc *frames, int i) {
  const polar_frame_desc &a = frames[i];
  const uint64_t N = a.fs->N;
  const size_t W = a.fs->mask.size();
  int j = i + 1;
  while (j < nframes) {
    const polar_frame_desc &b = frames[j];
    const size_t d = (size_t)(j - i);
    if (b.fs != a.fs || b.llr != a.llr + d * N || b.frozen_vals != a.frozen_vals + d * W ||
        b.xhat != a.xhat + d * W || (a.uhat == nullptr) != (b.uhat == nullptr) ||
        (a.uhat && b.uhat != a.uhat + d * W))
      break;
    ++j;
  }
  return j;
}

int polar_sc_decode_persistent(int nframes, const polar_frame_desc *frames, polar_fkind fkind,
                               polar_prec prec, void *stream) {
  int rc = check_frames(nframes, frames, (int)fkind, (int)prec);
  if (rc) return rc;
  rc = decode_persistent(nframes, frames, (int)fkind, (int)prec,
                         static_cast<cudaStream_t>(stream));
  return rc ? rc : check_guard(static_cast<cudaStream_t>(stream));
}

int polar_sc_decode_batch(int nframes, const polar_frame_desc *frames, polar_fkind fkind,
                          polar_prec prec, void *stream) {
  int rc = check_frames(nframes, frames, (int)fkind, (int)prec);
  if (rc) return rc;
  const long pm = g_cfg.persistent.load();
  if (prec == POLAR_FP32 && !g_cfg.plain.load() &&
      (pm == 2 || (pm == 1 && group_end(nframes, frames, 0) < nframes))) {
    rc = decode_persistent(nframes, frames, (int)fkind, (int)prec,
                           static_cast<cudaStream_t>(stream));
    return rc ? rc : check_guard(static_cast<cudaStream_t>(stream));
  }
  int i = 0;
  while (i < nframes) {
    const polar_frame_desc &a = frames[i];
    const int j = group_end(nframes, frames, i);
    Group g{const_cast<polar_frozen_set *>(a.fs), j - i, a.llr, a.frozen_vals, a.xhat, a.uhat,
            (int)fkind, (int)prec};
    int rc = decode_group(g, static_cast<cudaStream_t>(stream),
                          opts_for(g.fs, g.nframes, g.fkind, g.prec));
    if (rc) return rc;
    rc = check_guard(static_cast<cudaStream_t>(stream));
    if (rc) return rc;
    i = j;
  }
  return POLAR_OK;
}

int polar_debug_spoil_guard(void *stream) {
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> g(g_ws_mu);
  auto it = g_ws.find({dev, s});
  if (it == g_ws.end() || !it->second.guarded) return POLAR_ENOTFOUND;
  char *p = static_cast<char *>(it->second.ptr) + it->second.last_req + 100;
  CK(cudaMemsetAsync(p, 0, 1, s));   // inside the allocation: the trailing guard zone
  return POLAR_OK;
}

}  // extern "C"
