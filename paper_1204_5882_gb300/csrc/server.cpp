// Request server: continuous batching of reconciliation frames.
//
// Requests (one or more contiguous frames sharing a frozen set) enter a
// bounded host queue.  Scheduler threads (each owning an equal share of the
// decode slots, so that the host cost of launching is spread over cores)
// serve it; a slot is a non-blocking CUDA stream with its own scratch
// workspace.  Whenever a slot
// is free and the server's scratch budget allows the request's workspace, the
// oldest pending request is launched on that slot; completion is detected
// with a CUDA event and reported through poll / wait.  Requests submitted
// while others run are admitted as soon as a slot and memory free up, so
// their work overlaps on the device.  Admission is by device memory: a slot
// may only grow its workspace while the sum over slots stays within the
// budget (the decode scratch of a frame is about N * bytes(storage)).
//
// Persistent mode keeps one launch of the persistent decoder resident
// instead: the scheduler writes each admitted frame's descriptor into a ring
// in host-mapped memory and publishes it by advancing `tail`; the launch's
// CTAs claim frames in publication order and write one completion word per
// frame back into host-mapped memory.  The scheduler turns those words into
// request completions, recycles ring entries, and relaunches the decoder when
// frames are waiting and the previous launch has ended (its CTAs leave after
// about a millisecond without work).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>

#include "polar_internal.h"

using Clock = std::chrono::steady_clock;

namespace {

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  size_t ws_bytes = 0;   // workspace this slot holds (largest request so far)
  bool busy = false;
  uint64_t ticket = 0;
};

struct Pending {
  uint64_t ticket;
  polar_request req;
  Clock::time_point t_submit;
};

struct Record {
  int status = POLAR_PENDING;
  Clock::time_point t_submit, t_launch, t_done;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

// Persistent-mode state.
struct Ring {
  int t = 13;                   // subtree size of the resident launch
  int grid = 0;                 // resident CTAs
  uint32_t R = 0;               // ring entries (power of two)
  polar::PFrame *ring = nullptr;          // host-mapped
  uint32_t *ctl = nullptr;                // host-mapped: [0] tail, [1] stop, [64..) done
  uint32_t *done = nullptr;
  uint32_t *head = nullptr;               // device
  float *scratch = nullptr;               // device
  uint64_t cta_floats = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  bool running = false;
  bool stopping = false;                  // stop word set for the running launch
  Clock::time_point last_busy;            // last time frames were outstanding
  uint32_t published = 0;                 // frames published (tail)
  std::vector<uint32_t> out;              // published frames not yet complete, any order
  std::vector<uint8_t> seen;              // per entry: free (its last frame completed)
  std::vector<uint64_t> ticket;           // per entry: request ticket
  std::unordered_map<uint64_t, int> left; // ticket -> frames not yet complete
};

struct polar_server {
  polar_server_config cfg;
  Ring pr;
  std::vector<Slot> slots;
  std::deque<Pending> queue;
  std::unordered_map<uint64_t, Record> records;
  std::mutex mu;
  std::condition_variable cv_done;
  std::vector<std::thread> threads;
  bool stop = false;
  uint64_t next_ticket = 1;
  size_t ws_total = 0;
  uint64_t completed = 0, launched = 0, refused = 0;
};

namespace {

int check_request(const polar_request *r) {
  if (!r || !r->fs || r->nframes < 1 || !r->llr || !r->frozen_vals || !r->xhat) return POLAR_EINVAL;
  if (reinterpret_cast<uintptr_t>(r->llr) % 16) return POLAR_EINVAL;
  return POLAR_OK;
}

void finish_slot(polar_server *s, Slot &sl, int status) {
  auto it = s->records.find(sl.ticket);
  if (it != s->records.end()) {
    it->second.status = status;
    it->second.t_done = Clock::now();
  }
  sl.busy = false;
  s->completed++;
  s->cv_done.notify_all();
}

void scheduler(polar_server *s, size_t first, size_t step) {
  cudaSetDevice(s->cfg.device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    bool any_busy = false;
    // 1. completions of this thread's slots
    for (size_t si = first; si < s->slots.size(); si += step) {
      Slot &sl = s->slots[si];
      if (!sl.busy) continue;
      cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaSuccess) {
        finish_slot(s, sl, POLAR_OK);
      } else if (q != cudaErrorNotReady) {
        polar::set_last_error(cudaGetErrorString(q));
        finish_slot(s, sl, POLAR_ECUDA);
      } else {
        any_busy = true;
      }
    }
    // 2. admissions, oldest first, while a slot and memory allow
    while (!s->queue.empty()) {
      Pending &p = s->queue.front();
      const size_t need = polar::decode_scratch_bytes(p.req.fs, p.req.nframes, s->cfg.prec);
      if (need > s->cfg.mem_budget) {                 // can never fit
        auto it = s->records.find(p.ticket);
        if (it != s->records.end()) {
          it->second.status = POLAR_ENOMEM;
          it->second.t_done = Clock::now();
        }
        s->queue.pop_front();
        s->cv_done.notify_all();
        continue;
      }
      Slot *pick = nullptr;
      for (size_t si = first; si < s->slots.size() && !pick; si += step) {
        Slot &sl = s->slots[si];                       // a free slot that fits as is
        if (!sl.busy && sl.ws_bytes >= need) pick = &sl;
      }
      for (size_t si = first; si < s->slots.size() && !pick; si += step) {
        Slot &sl = s->slots[si];                       // or one that may grow
        if (!sl.busy && s->ws_total - sl.ws_bytes + need <= s->cfg.mem_budget) pick = &sl;
      }
      if (!pick) break;
      Pending job = p;
      s->queue.pop_front();
      if (pick->ws_bytes < need) {
        s->ws_total += need - pick->ws_bytes;
        pick->ws_bytes = need;
      }
      pick->busy = true;                               // reserved while launching
      auto it = s->records.find(job.ticket);
      if (it != s->records.end()) it->second.t_launch = Clock::now();
      lk.unlock();
      int rc = polar::decode_eager(job.req.fs, job.req.nframes, job.req.llr, job.req.frozen_vals,
                                   job.req.xhat, job.req.uhat, s->cfg.fkind, s->cfg.prec,
                                   pick->stream);
      if (rc == POLAR_OK && cudaEventRecord(pick->done, pick->stream) != cudaSuccess)
        rc = POLAR_ECUDA;
      lk.lock();
      pick->ticket = job.ticket;
      s->launched++;
      if (rc != POLAR_OK) {
        finish_slot(s, *pick, rc);
      } else {
        any_busy = true;
      }
    }
    if (s->stop && s->queue.empty() && !any_busy) break;
    if (any_busy) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(5));
      lk.lock();
    } else {
      s->cv_done.wait_for(lk, std::chrono::microseconds(200));
    }
  }
}

// ---------------------------------------------------------------- persistent
void finish_ticket(polar_server *s, uint64_t ticket, int status) {
  auto it = s->records.find(ticket);
  if (it != s->records.end()) {
    it->second.status = status;
    it->second.t_done = Clock::now();
  }
  s->completed++;
  s->cv_done.notify_all();
}

// Completions: every published frame whose completion word has arrived.
// Frames finish in any order; each frees its own ring entry.
void ring_collect(polar_server *s) {
  Ring &r = s->pr;
  for (size_t k = 0; k < r.out.size();) {
    const uint32_t idx = r.out[k], e = idx & (r.R - 1);
    if (__atomic_load_n(r.done + e, __ATOMIC_ACQUIRE) != idx + 1) {
      ++k;
      continue;
    }
    r.seen[e] = 1;
    auto it = r.left.find(r.ticket[e]);
    if (it != r.left.end() && --it->second == 0) {
      finish_ticket(s, it->first, POLAR_OK);
      r.left.erase(it);
    }
    r.out[k] = r.out.back();
    r.out.pop_back();
  }
}

// Publishes the oldest pending requests while the ring has room.
void ring_publish(polar_server *s) {
  if (s->queue.empty()) return;
  polar::NvtxRange nv("polar server publish");
  Ring &r = s->pr;
  int dev = s->cfg.device;
  while (!s->queue.empty()) {
    Pending &p = s->queue.front();
    const uint32_t nf = (uint32_t)p.req.nframes;
    bool room = true;                                      // the next nf entries are free
    for (uint32_t f = 0; f < nf && room; ++f) room = r.seen[(r.published + f) & (r.R - 1)];
    if (!room) break;
    polar_frozen_set *fs = const_cast<polar_frozen_set *>(p.req.fs);
    const int n = (int)fs->log2n, t = std::min(n, r.t);
    cudaError_t e = cudaSuccess;
    const uint32_t *mask = polar::device_mask(fs, dev, &e);
    const uint32_t *cls = mask && t >= 5 ? polar::device_class_table(fs, dev, t, &e) : nullptr;
    const uint32_t *ucls =
        mask && n > t ? polar::device_upper_class_table(fs, dev, t, &e) : nullptr;
    if (!mask || (t >= 5 && !cls) || (n > t && !ucls)) {
      polar::set_last_error(cudaGetErrorString(e));
      finish_ticket(s, p.ticket, e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : POLAR_ECUDA);
      s->queue.pop_front();
      continue;
    }
    const uint64_t N = uint64_t(1) << n;
    const size_t W = fs->mask.size();
    for (uint32_t f = 0; f < nf; ++f) {
      const uint32_t idx = r.published + f, ent = idx & (r.R - 1);
      polar::PFrame &d = r.ring[ent];
      d.llr = p.req.llr + f * N;
      d.fv = p.req.frozen_vals + f * W;
      d.xhat = p.req.xhat + f * W;
      d.uhat = p.req.uhat ? p.req.uhat + f * W : nullptr;
      d.mask = mask;
      d.cls = cls;
      d.ucls = ucls;
      d.log2n = (uint32_t)n;
      d.t = (uint32_t)t;
      r.seen[ent] = 0;
      r.ticket[ent] = p.ticket;
      r.out.push_back(idx);
    }
    r.left[p.ticket] = (int)nf;
    r.published += nf;
    __atomic_store_n(r.ctl, r.published, __ATOMIC_RELEASE);   // tail
    auto it = s->records.find(p.ticket);
    if (it != s->records.end()) it->second.t_launch = Clock::now();
    s->launched++;
    s->queue.pop_front();
  }
}

// (Re)launches the decoder when frames wait and no launch is running; asks a
// running launch to end (stop word) once nothing has been outstanding for a
// millisecond.  The launch's own 50 ms idle limit only bounds its waits.
int ring_launch(polar_server *s) {
  Ring &r = s->pr;
  const Clock::time_point now = Clock::now();
  if (!r.out.empty() || !s->queue.empty()) r.last_busy = now;
  if (r.running) {
    const cudaError_t q = cudaEventQuery(r.ev);
    if (q == cudaErrorNotReady) {
      if (!r.stopping && r.out.empty() && s->queue.empty() &&
          now - r.last_busy > std::chrono::milliseconds(1)) {
        __atomic_store_n(r.ctl + 1, 1u, __ATOMIC_RELEASE);
        r.stopping = true;
      }
      return POLAR_OK;
    }
    r.running = false;
    if (q != cudaSuccess) {
      polar::set_last_error(cudaGetErrorString(q));
      return POLAR_ECUDA;
    }
    ring_collect(s);                        // words written by the launch that ended
  }
  if (r.out.empty()) {
    // idle with no launch running: restart the 32-bit frame counters long
    // before they could wrap (the kernel compares claimed < published)
    if (r.published >= (1u << 31)) {
      cudaError_t e = cudaMemsetAsync(r.head, 0, sizeof(uint32_t), r.stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(r.stream);
      if (e != cudaSuccess) {
        polar::set_last_error(cudaGetErrorString(e));
        return POLAR_ECUDA;
      }
      std::memset(r.done, 0, r.R * sizeof(uint32_t));
      r.published = 0;
      __atomic_store_n(r.ctl, 0u, __ATOMIC_RELEASE);
    }
    return POLAR_OK;
  }
  if (r.stopping) {                         // the ended launch no longer reads it
    __atomic_store_n(r.ctl + 1, 0u, __ATOMIC_RELEASE);
    r.stopping = false;
  }
  polar::ServeArgs a;
  a.ring = r.ring;
  a.rmask = r.R - 1;
  a.tail = r.ctl;
  a.stop = r.ctl + 1;
  a.done = r.done;
  a.head = r.head;
  a.scratch = r.scratch;
  a.cta_floats = r.cta_floats;
  a.idle_ns = 50000000;
  long target = 8;
  polar_config_get("int8_target", &target);
  a.int8_target = (double)target;
  a.smem = 0;
  cudaError_t e =
      polar::launch_serve((int)s->cfg.prec, (int)s->cfg.fkind, a, r.t, r.grid, r.stream);
  if (e == cudaSuccess) e = cudaEventRecord(r.ev, r.stream);
  if (e != cudaSuccess) {
    polar::set_last_error(cudaGetErrorString(e));
    return POLAR_ECUDA;
  }
  r.running = true;
  polar::log_msg("server: resident decoder launched, %zu frames outstanding, %u published",
                 r.out.size(), r.published);
  return POLAR_OK;
}

// Every published frame and every pending request fails with `status`.
void ring_fail_all(polar_server *s, int status) {
  Ring &r = s->pr;
  for (auto &kv : r.left) finish_ticket(s, kv.first, status);
  r.left.clear();
  r.out.clear();
  while (!s->queue.empty()) {
    finish_ticket(s, s->queue.front().ticket, status);
    s->queue.pop_front();
  }
}

void ring_scheduler(polar_server *s) {
  cudaSetDevice(s->cfg.device);
  std::unique_lock<std::mutex> lk(s->mu);
  bool failed = false;
  while (true) {
    if (!failed) {
      ring_collect(s);
      ring_publish(s);
      if (ring_launch(s) != POLAR_OK) {
        failed = true;
        ring_fail_all(s, POLAR_ECUDA);
      }
    } else if (!s->queue.empty()) {
      ring_fail_all(s, POLAR_ECUDA);
    }
    const bool busy = !s->pr.out.empty();
    if (s->stop && s->queue.empty() && !busy) break;
    if (busy) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(5));
      lk.lock();
    } else {
      s->cv_done.wait_for(lk, std::chrono::microseconds(200));
    }
  }
  __atomic_store_n(s->pr.ctl + 1, 1u, __ATOMIC_RELEASE);      // stop: idle CTAs leave
}

void ring_release(polar_server *s) {
  Ring &r = s->pr;
  if (r.stream) cudaStreamSynchronize(r.stream);
  if (r.ev) cudaEventDestroy(r.ev);
  if (r.stream) cudaStreamDestroy(r.stream);
  if (r.head) cudaFree(r.head);
  if (r.scratch) cudaFree(r.scratch);
  if (r.ring) cudaFreeHost(r.ring);
  if (r.ctl) cudaFreeHost(r.ctl);
  r = Ring();
}

int ring_create(polar_server *s) {
  Ring &r = s->pr;
  const polar_server_config &c = s->cfg;
  long tcfg = 13;
  polar_config_get("persist_log2", &tcfg);
  r.t = (int)tcfg;
  const int nmax = c.max_log2n ? c.max_log2n : 22;
  const int per_sm = polar::serve_ctas_per_sm((int)c.prec, (int)c.fkind, r.t);
  int sms = 0;
  if (per_sm < 1 || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device) !=
                        cudaSuccess) {
    cudaGetLastError();
    return POLAR_ECUDA;
  }
  r.cta_floats = nmax > r.t ? (uint64_t(1) << nmax) - (uint64_t(1) << r.t) : 0;
  r.cta_floats = (r.cta_floats + 63) & ~uint64_t(63);
  uint64_t fit = r.cta_floats ? c.mem_budget / (r.cta_floats * sizeof(float)) : ~uint64_t(0);
  r.grid = (int)std::min<uint64_t>({(uint64_t)per_sm * sms, (uint64_t)c.max_inflight, fit});
  if (r.grid < 1) return POLAR_ENOMEM;
  // frames are published in order but finish in any order: a generous ring
  // keeps a long frame's entry from holding back the next publications
  r.R = 8192;
  while (r.R < 16u * (uint32_t)r.grid) r.R *= 2;
  r.seen.assign(r.R, 1);
  r.ticket.assign(r.R, 0);
  auto fail = [&](cudaError_t e) {
    polar::set_last_error(cudaGetErrorString(e));
    cudaGetLastError();
    ring_release(s);
    return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : POLAR_ECUDA;
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
  if ((e = cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
  if ((e = cudaHostAlloc(reinterpret_cast<void **>(&r.ring), r.R * sizeof(polar::PFrame),
                         cudaHostAllocMapped | cudaHostAllocPortable)) != cudaSuccess)
    return fail(e);
  if ((e = cudaHostAlloc(reinterpret_cast<void **>(&r.ctl), (64 + r.R) * sizeof(uint32_t),
                         cudaHostAllocMapped | cudaHostAllocPortable)) != cudaSuccess)
    return fail(e);
  std::memset(r.ctl, 0, (64 + r.R) * sizeof(uint32_t));
  r.done = r.ctl + 64;
  if ((e = cudaMalloc(reinterpret_cast<void **>(&r.head), 256)) != cudaSuccess) return fail(e);
  if ((e = cudaMemset(r.head, 0, 256)) != cudaSuccess) return fail(e);
  if (r.cta_floats &&
      (e = cudaMalloc(reinterpret_cast<void **>(&r.scratch),
                      (size_t)r.grid * r.cta_floats * sizeof(float))) != cudaSuccess)
    return fail(e);
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e);
  s->ws_total = (size_t)r.grid * r.cta_floats * sizeof(float);
  polar::log_msg("server: persistent, %d resident CTAs (subtree 2^%d), ring of %u frames, "
                 "%zu bytes of scratch", r.grid, r.t, r.R, s->ws_total);
  return POLAR_OK;
}

}  // namespace

extern "C" {

int polar_server_create(const polar_server_config *cfg, polar_server **out) {
  if (!cfg || !out) return POLAR_EINVAL;
  if (cfg->persistent != 0 && cfg->persistent != 1) return POLAR_EINVAL;
  if (cfg->max_inflight < 1 || cfg->max_inflight > (cfg->persistent ? 4096 : 256) ||
      cfg->max_queue < 1)
    return POLAR_EINVAL;
  if (cfg->persistent && (cfg->max_log2n < 0 || cfg->max_log2n > 27)) return POLAR_EINVAL;
  if (cfg->fkind != POLAR_F_MINSUM && cfg->fkind != POLAR_F_EXACT) return POLAR_EINVAL;
  if (cfg->prec != POLAR_FP32 && cfg->prec != POLAR_FP16 && cfg->prec != POLAR_INT8)
    return POLAR_EINVAL;
  if (cfg->threads < 0 || cfg->threads > 16) return POLAR_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
    cudaGetLastError();
    return POLAR_EINVAL;
  }
  auto *s = new (std::nothrow) polar_server();
  if (!s) return POLAR_ENOMEM;
  s->cfg = *cfg;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(cfg->device);
  if (cfg->persistent) {
    const int rc = ring_create(s);
    cudaSetDevice(prev);
    if (rc != POLAR_OK) {
      delete s;
      return rc;
    }
    s->threads.emplace_back(ring_scheduler, s);
    *out = s;
    return POLAR_OK;
  }
  s->slots.resize(cfg->max_inflight);
  for (auto &sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
      for (auto &x : s->slots) {
        if (x.stream) cudaStreamDestroy(x.stream);
        if (x.done) cudaEventDestroy(x.done);
      }
      cudaSetDevice(prev);
      delete s;
      return POLAR_ECUDA;
    }
  }
  cudaSetDevice(prev);
  size_t nth = cfg->threads ? (size_t)cfg->threads : 4;
  if (nth > s->slots.size()) nth = s->slots.size();
  for (size_t i = 0; i < nth; ++i) s->threads.emplace_back(scheduler, s, i, nth);
  polar::log_msg("server: %zu decode slots, %zu scheduler threads, scratch budget %zu bytes",
                 s->slots.size(), nth, cfg->mem_budget);
  *out = s;
  return POLAR_OK;
}

int polar_server_submit(polar_server *s, const polar_request *req, uint64_t *ticket) {
  if (!s || !ticket) return POLAR_EINVAL;
  int rc = check_request(req);
  if (rc) return rc;
  if (s->cfg.persistent) {
    const int nmax = s->cfg.max_log2n ? s->cfg.max_log2n : 22;
    if ((int)req->fs->log2n > nmax || (uint32_t)req->nframes > s->pr.R / 2) return POLAR_EINVAL;
    // A code's first request uploads its tables here, on the caller's
    // thread, rather than in the scheduler, where it would hold up the
    // publication of every other frame.
    rc = polar::prepare_tables(const_cast<polar_frozen_set *>(req->fs), s->cfg.device, s->pr.t,
                               true);
    if (rc) return rc;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return POLAR_EINVAL;
  if ((int)s->queue.size() >= s->cfg.max_queue) {
    s->refused++;
    return POLAR_EBUSY;
  }
  const uint64_t t = s->next_ticket++;
  Record r;
  r.t_submit = Clock::now();
  s->records.emplace(t, r);
  s->queue.push_back(Pending{t, *req, r.t_submit});
  *ticket = t;
  return POLAR_OK;
}

static int fill_result(polar_server *s, uint64_t ticket, polar_result *out) {
  auto it = s->records.find(ticket);
  if (it == s->records.end()) return POLAR_ENOTFOUND;
  const Record &r = it->second;
  if (r.status == POLAR_PENDING) return POLAR_PENDING;
  if (out) {
    out->status = r.status;
    out->queue_ms = r.t_launch.time_since_epoch().count() ? ms_between(r.t_submit, r.t_launch)
                                                           : ms_between(r.t_submit, r.t_done);
    out->latency_ms = ms_between(r.t_submit, r.t_done);
  }
  int st = r.status;
  s->records.erase(it);
  return st == POLAR_OK ? POLAR_OK : st;
}

int polar_server_poll(polar_server *s, uint64_t ticket, polar_result *out) {
  if (!s) return POLAR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  return fill_result(s, ticket, out);
}

int polar_server_wait(polar_server *s, uint64_t ticket, double timeout_ms, polar_result *out) {
  if (!s) return POLAR_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = Clock::now() + std::chrono::microseconds((int64_t)(timeout_ms * 1e3));
  for (;;) {
    int rc = fill_result(s, ticket, out);
    if (rc != POLAR_PENDING) return rc;
    if (Clock::now() >= deadline) return POLAR_ETIMEDOUT;
    s->cv_done.wait_until(lk, deadline);
  }
}

int polar_server_cancel(polar_server *s, uint64_t ticket) {
  if (!s) return POLAR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto rec = s->records.find(ticket);
  if (rec == s->records.end()) return POLAR_ENOTFOUND;
  if (rec->second.status != POLAR_PENDING) return POLAR_EBUSY;   // finished, not yet reported
  // The schedulers take requests off the queue under this lock (and copy
  // them before unlocking), so a request found here has not started.
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    if (it->ticket != ticket) continue;
    s->queue.erase(it);
    rec->second.status = POLAR_ECANCELED;
    rec->second.t_done = Clock::now();
    s->cv_done.notify_all();
    return POLAR_OK;
  }
  return POLAR_EBUSY;                                              // launched or published
}

int polar_server_stats(polar_server *s, uint64_t *launched, uint64_t *completed,
                       uint64_t *refused, size_t *scratch_bytes) {
  if (!s) return POLAR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (launched) *launched = s->launched;
  if (completed) *completed = s->completed;
  if (refused) *refused = s->refused;
  if (scratch_bytes) *scratch_bytes = s->ws_total;
  return POLAR_OK;
}

void polar_server_destroy(polar_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_done.notify_all();
  for (auto &th : s->threads)
    if (th.joinable()) th.join();
  if (s->cfg.persistent) ring_release(s);
  for (auto &sl : s->slots) {
    cudaStreamSynchronize(sl.stream);
    polar::release_stream_workspace(s->cfg.device, sl.stream);
    cudaStreamDestroy(sl.stream);
    cudaEventDestroy(sl.done);
  }
  delete s;
}

}  // extern "C"
