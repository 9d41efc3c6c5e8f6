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
#include <chrono>
#include <condition_variable>
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

struct polar_server {
  polar_server_config cfg;
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

}  // namespace

extern "C" {

int polar_server_create(const polar_server_config *cfg, polar_server **out) {
  if (!cfg || !out) return POLAR_EINVAL;
  if (cfg->max_inflight < 1 || cfg->max_inflight > 256 || cfg->max_queue < 1) return POLAR_EINVAL;
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
  *out = s;
  return POLAR_OK;
}

int polar_server_submit(polar_server *s, const polar_request *req, uint64_t *ticket) {
  if (!s || !ticket) return POLAR_EINVAL;
  int rc = check_request(req);
  if (rc) return rc;
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
  for (auto &sl : s->slots) {
    cudaStreamSynchronize(sl.stream);
    polar::release_stream_workspace(s->cfg.device, sl.stream);
    cudaStreamDestroy(sl.stream);
    cudaEventDestroy(sl.done);
  }
  delete s;
}

}  // extern "C"
