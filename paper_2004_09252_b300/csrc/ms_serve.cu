// Served form: continuous batching of encrypt / decrypt requests on pages of
// a host working set, through pinned staging and a two-direction copy
// pipeline.  Stands in for the paper's server + data thread (Sec. 4.2-4.4).
//
// Threads: callers submit requests (any thread); one server thread admits
// them in arrival order, forms waves, gathers pages into pinned staging,
// issues copies + kernel, and completes waves; a small pool of copy workers
// shares the gather / scatter memcpys of large waves.
//
// Staging is a ring of S page slots (pinned host) mirrored on the device,
// with one 16-byte kernel entry per slot.  A wave occupies a contiguous run
// of slots; waves are freed in issue order.
//
// In-place lane (continuous mode, working set in pinned mapped memory,
// zero_copy_max_pages = N > 0): while everything queued fits in N pages (64
// while a longer wave is in flight), the server forms the wave without
// staging slots and runs it in place on the working set: one launch of the
// host-link page kernel (a bounded grid, ms_link.cu) with the entries in the
// kernel's parameters -- no gather, no copies, no scatter.  Such waves
// complete as soon as their kernel does (up to kInplaceDepth at once, one
// while a longer wave is in flight).  Under load the queue outgrows N, and
// the longer waves run in place as well: their entries take staging slots
// (copied to the device), their pages do not.  Only a pageable working set,
// or N = 0, has its pages gathered, copied both ways and scattered.
#include <sys/prctl.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "ms_admission.h"
#include "ms_internal.h"

using namespace ms;

namespace {

using clk = std::chrono::steady_clock;

inline uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(clk::now().time_since_epoch()).count();
}

// Short naps must stay short: the first nap on a thread (the server's, a
// replay's or a caller of ms_server_wait) drops its timer slack (default
// 50 us, which would stretch a 1 us nap to about 50 us) to 1 us.
inline void nap_ns(long ns) {
  thread_local bool slack_set = false;
  if (!slack_set) {
    prctl(PR_SET_TIMERSLACK, 1000UL, 0, 0, 0);
    slack_set = true;
  }
  struct timespec ts = {ns / 1000000000L, ns % 1000000000L};
  nanosleep(&ts, nullptr);
}

enum ReqState : int { kFree = 0, kQueued = 1, kAdmitted = 2, kDone = 3, kClaiming = 4 };

struct Req {
  std::atomic<int> state{kFree};
  std::atomic<int> error{0};
  std::atomic<uint64_t> ticket{~0ull};
  int op = 0;
  uint32_t domain = 0;         // nonce word 15 of this request's pages
  std::vector<uint64_t> pages;
  uint64_t t_sched_ns = 0;     // arrival time latency is measured from
  std::atomic<uint64_t> t_done_ns{0};
  double *lat_out = nullptr;   // replay: where to write the latency, seconds
};

// Parallel-for over page indices for the gather / scatter memcpys.
class CopyPool {
 public:
  explicit CopyPool(int n) {
    for (int i = 0; i < n; ++i) th_.emplace_back([this] { worker(); });
  }
  ~CopyPool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
      stop_flag_.store(true);
    }
    cv_.notify_all();
    for (auto &t : th_) t.join();
  }
  // Runs fn(i) for i in [0, n); the calling thread takes part.
  void run(size_t n, const std::function<void(size_t)> &fn) {
    // Below 512 KiB one thread does it: a hand-off costs wake-ups.  (A
    // threshold of 2 MiB measured worse: 532k-pages/s p99 1.3 -> 2.5-3.5 ms.)
    if (th_.empty() || n < 128) {
      for (size_t i = 0; i < n; ++i) fn(i);
      return;
    }
    {
      std::lock_guard<std::mutex> lk(mu_);
      job_ = &fn;
      n_ = n;
      next_.store(0);
      active_ = (int)th_.size();
      ++gen_;
      pub_gen_.store(gen_, std::memory_order_release);
    }
    cv_.notify_all();
    drain(fn, n);
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return active_ == 0; });
    job_ = nullptr;
  }

 private:
  void drain(const std::function<void(size_t)> &fn, size_t n) {
    for (;;) {
      const size_t a = next_.fetch_add(16);
      if (a >= n) break;
      const size_t b = std::min(n, a + 16);
      for (size_t i = a; i < b; ++i) fn(i);
    }
  }
  void worker() {
    prctl(PR_SET_TIMERSLACK, 1000UL, 0, 0, 0);
    uint64_t seen = 0;
    for (;;) {
      const std::function<void(size_t)> *job;
      size_t n;
      // poll for a new job for ~100 us before sleeping: waves come in bursts
      for (int i = 0; i < 100 && pub_gen_.load(std::memory_order_acquire) == seen && !stop_flag_.load(); ++i)
        nap_ns(1000);
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
        job = job_;
        n = n_;
      }
      drain(*job, n);
      {
        std::lock_guard<std::mutex> lk(mu_);
        if (--active_ == 0) done_cv_.notify_all();
      }
    }
  }
  std::vector<std::thread> th_;
  std::mutex mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(size_t)> *job_ = nullptr;
  size_t n_ = 0;
  std::atomic<size_t> next_{0};
  int active_ = 0;
  uint64_t gen_ = 0;
  std::atomic<uint64_t> pub_gen_{0};
  std::atomic<bool> stop_flag_{false};
  bool stop_ = false;
};

struct Wave : ms::AdmittedWave {
  cudaEvent_t ev_h2d = nullptr, ev_done = nullptr;
  bool zc = false;  // run in place on the working set (no staging copies)
};

constexpr size_t kInplaceDepth = 4;        // in-place waves in flight at most
constexpr uint32_t kInplaceBusyPages = 64;  // lane wave size while a longer wave is in flight

}  // namespace

struct ms_server {
  ms_ctx *ctx = nullptr;
  uint8_t *host = nullptr;
  uint64_t n_pages = 0;
  ms_server_config cfg{};
  uint32_t S = 0;  // staging slots
  uint8_t *h_stage = nullptr, *d_stage = nullptr;
  ms_page_dom *h_ent = nullptr, *d_ent = nullptr;
  cudaStream_t s_in = nullptr, s_work[2] = {nullptr, nullptr};
  // Kernels that work on the mapped working set itself (in-place lane,
  // zero-copy waves) run on this one stream: one such kernel at a time, so the
  // host link sees at most one bounded grid of SM-issued accesses.
  cudaStream_t s_link = nullptr;
  uint32_t inplace_max = 0;       // pages of an in-place wave at most (0: lane off)
  std::vector<Req> reqs;
  // Submitters hold inmu only to claim a request slot and append its ticket
  // to the inbox; the server thread moves the inbox into `incoming` (its
  // own queue) at each pass.  So forming and completing waves, however long
  // under load, never hold up a submission.
  std::mutex inmu;
  std::condition_variable qcv;       // with inmu: wakes an idle server thread
  std::vector<uint64_t> inbox;       // submitted tickets, in submission order (guarded by inmu)
  std::vector<uint64_t> inbox_spare; // the server thread's swap buffer for the inbox
  uint64_t taken_upto = 0;           // next_ticket as of the last take of the inbox (server thread)
  std::mutex qmu;
  std::deque<uint64_t> incoming;     // server thread only
  std::atomic<uint64_t> next_ticket{0};
  ms::Admission *adm = nullptr;  // staging ring and in-flight pages (guarded by qmu)
  std::deque<Wave> inflight;
  std::deque<Wave> inflight_inplace;  // completed in any order
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  uint64_t wave_seq = 0;
  std::thread th;
  std::atomic<bool> stop{false};
  std::atomic<bool> exited{false};
  std::atomic<int> error{0};
  CopyPool *pool = nullptr;
  std::mutex done_mu;
  std::condition_variable done_cv;
  std::atomic<uint64_t> st_req{0}, st_pages{0}, st_waves{0}, st_maxreq{0}, st_maxpages{0}, st_conflict{0},
      st_budget{0}, st_maxstaged{0}, st_gather_ns{0}, st_scatter_ns{0}, st_inplace{0}, st_staged{0}, st_max_pass{0},
      st_replay_lag{0}, st_replay_late{0};
  uint64_t d_host = 0;  // device address of host_base (zero-copy mode)
  uint64_t idle_spin_ns = 0;

  Req &slot(uint64_t t) { return reqs[t % reqs.size()]; }
  void loop();
  bool take_inbox(bool wait);
  bool form_wave(Wave &w);
  bool form_inplace(Wave &w, uint32_t max_pages);
  int issue(Wave &w);
  int issue_inplace(Wave &w);
  bool take_events(Wave &w);
  void complete(Wave &w);
  void fail_all(int code);
};

namespace {

void atomic_max(std::atomic<uint64_t> &a, uint64_t v) {
  uint64_t cur = a.load();
  while (v > cur && !a.compare_exchange_weak(cur, v)) {
  }
}

}  // namespace

// Admission (see ms_admission.h): at most kScanWindow queued requests are
// considered per wave.
constexpr size_t kScanWindow = 4096;

// wait = false (a serving pass): leave the inbox for the next pass if a
// submitter holds its lock, so that a submitting thread that is descheduled
// inside its short critical section never holds up the server thread.
// Returns false when it left the inbox so (the caller must not go idle).
bool ms_server::take_inbox(bool wait) {
  {
    std::unique_lock<std::mutex> lk(inmu, std::defer_lock);
    if (wait) {
      lk.lock();
    } else if (!lk.try_lock()) {
      return false;
    }
    taken_upto = next_ticket.load();  // every ticket below this is in `incoming` or beyond
    if (inbox.empty()) return true;
    inbox.swap(inbox_spare);  // the inbox keeps the spare's (empty) buffer
  }
  incoming.insert(incoming.end(), inbox_spare.begin(), inbox_spare.end());
  inbox_spare.clear();
  return true;
}

bool ms_server::form_wave(Wave &w) {
  std::lock_guard<std::mutex> lk(qmu);
  const bool ok = adm->form(incoming, [&](uint64_t t) -> const std::vector<uint64_t> & { return slot(t).pages; }, w);
  st_budget.store(adm->budget_waits);
  st_conflict.store(adm->conflict_waits);
  if (ok) atomic_max(st_maxstaged, adm->used());
  return ok;
}

bool ms_server::form_inplace(Wave &w, uint32_t max_pages) {
  std::lock_guard<std::mutex> lk(qmu);
  const bool ok = adm->form_inplace(incoming, [&](uint64_t t) -> const std::vector<uint64_t> & { return slot(t).pages; },
                                    w, max_pages);
  st_conflict.store(adm->conflict_waits);
  return ok;
}

bool ms_server::take_events(Wave &w) {
  if (ev_pool.empty()) {
    cudaEvent_t a, b;
    if (cudaEventCreateWithFlags(&a, cudaEventDisableTiming) != cudaSuccess) return false;
    if (cudaEventCreateWithFlags(&b, cudaEventDisableTiming) != cudaSuccess) {
      cudaEventDestroy(a);
      return false;
    }
    ev_pool.push_back({a, b});
  }
  w.ev_h2d = ev_pool.back().first;
  w.ev_done = ev_pool.back().second;
  ev_pool.pop_back();
  return true;
}

// An in-place wave: one launch with the entries in the kernel's parameters.
int ms_server::issue_inplace(Wave &w) {
  if (!take_events(w)) return cuda_fail(ctx, cudaGetLastError());
  ms_page_dom ent[512];
  uint32_t k = 0;
  for (uint64_t t : w.tickets) {
    Req &r = slot(t);
    r.state.store(kAdmitted, std::memory_order_release);
    for (uint64_t pg : r.pages) {
      ent[k].addr = d_host + pg * MS_PAGE_BYTES;
      ent[k].page_id = pg;
      ent[k].domain = r.domain;
      ent[k].reserved0 = 0;
      ent[k].reserved1 = 0;
      ++k;
    }
  }
  w.zc = true;
  cudaError_t e = injected(MS_FAULT_SERVER);
  if (e == cudaSuccess) e = launch_pages_link(ctx, ent, k, s_link);
  if (e == cudaSuccess) e = cudaEventRecord(w.ev_done, s_link);
  if (e != cudaSuccess) return cuda_fail(ctx, e);
  st_waves.fetch_add(1);
  st_inplace.fetch_add(1);
  atomic_max(st_maxreq, w.tickets.size());
  atomic_max(st_maxpages, w.len);
  return MS_OK;
}

int ms_server::issue(Wave &w) {
  if (!take_events(w)) return cuda_fail(ctx, cudaGetLastError());
  // Zero-copy mode, and continuous mode whenever its in-place lane is on (a
  // pinned, mapped working set): the kernel works on the working set itself,
  // on the link stream, and only the entries use the wave's staging slots
  // (short queues of continuous mode take the lane instead, issue_inplace).
  // Otherwise the pages are gathered into staging and copied both ways.
  const bool zc = cfg.mode == MS_SERVE_ZERO_COPY || inplace_max != 0;
  w.zc = zc;
  const uint64_t tg = now_ns();
  uint32_t k = w.pos;
  if (zc) {  // entries point at the working set: no per-page map, no copies
    for (uint64_t t : w.tickets) {
      Req &r = slot(t);
      r.state.store(kAdmitted, std::memory_order_release);
      for (uint64_t pg : r.pages) {
        h_ent[k].addr = d_host + pg * MS_PAGE_BYTES;
        h_ent[k].page_id = pg;
        h_ent[k].domain = r.domain;
        ++k;
      }
    }
  } else {
    // slot index of every page of the wave, in order
    std::vector<std::pair<uint64_t, uint32_t>> map;  // (working-set page, staging slot)
    map.reserve(w.len);
    for (uint64_t t : w.tickets) {
      Req &r = slot(t);
      r.state.store(kAdmitted, std::memory_order_release);
      for (uint64_t pg : r.pages) {
        h_ent[k].domain = r.domain;
        map.push_back({pg, k++});
      }
    }
    pool->run(map.size(), [&](size_t i) {
      const uint64_t pg = map[i].first;
      const uint32_t sl = map[i].second;
      std::memcpy(h_stage + (size_t)sl * MS_PAGE_BYTES, host + pg * MS_PAGE_BYTES, MS_PAGE_BYTES);
      h_ent[sl].addr = (uint64_t)(d_stage + (size_t)sl * MS_PAGE_BYTES);
      h_ent[sl].page_id = pg;
    });
  }
  st_gather_ns.fetch_add(now_ns() - tg);
  const size_t off = (size_t)w.pos * MS_PAGE_BYTES, bytes = (size_t)w.len * MS_PAGE_BYTES;
  cudaStream_t sw = zc ? s_link : s_work[wave_seq++ & 1];
  cudaError_t e = injected(MS_FAULT_SERVER);
  if (e == cudaSuccess && !zc) e = cudaMemcpyAsync(d_stage + off, h_stage + off, bytes, cudaMemcpyHostToDevice, s_in);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_ent + w.pos, h_ent + w.pos, sizeof(ms_page_dom) * w.len, cudaMemcpyHostToDevice, s_in);
  if (e == cudaSuccess) e = cudaEventRecord(w.ev_h2d, s_in);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(sw, w.ev_h2d, 0);
  if (e == cudaSuccess && zc) e = launch_pages_link_dev(ctx, d_ent + w.pos, w.len, sw);
  if (e == cudaSuccess && !zc) {
    PageArgs a = make_args(ctx);
    a.dpages = d_ent + w.pos;
    a.n_pages = w.len;
    e = launch_pages(ctx, a, sw);
  }
  if (e == cudaSuccess && !zc) e = cudaMemcpyAsync(h_stage + off, d_stage + off, bytes, cudaMemcpyDeviceToHost, sw);
  if (e == cudaSuccess && cfg.zero_staging && !zc) e = cudaMemsetAsync(d_stage + off, 0, bytes, sw);
  if (e == cudaSuccess) e = cudaEventRecord(w.ev_done, sw);
  if (e != cudaSuccess) return cuda_fail(ctx, e);
  st_waves.fetch_add(1);
  if (!zc) st_staged.fetch_add(1);
  atomic_max(st_maxreq, w.tickets.size());
  atomic_max(st_maxpages, w.len);
  return MS_OK;
}

void ms_server::complete(Wave &w) {
  const bool wipe = cfg.zero_staging != 0;
  const uint64_t ts = now_ns();
  if (!w.zc) {  // a staged wave: its pages go back into the working set
    std::vector<std::pair<uint64_t, uint32_t>> map;
    map.reserve(w.len);
    uint32_t k = w.pos;
    for (uint64_t t : w.tickets)
      for (uint64_t pg : slot(t).pages) map.push_back({pg, k++});
    pool->run(map.size(), [&](size_t i) {
      uint8_t *src = h_stage + (size_t)map[i].second * MS_PAGE_BYTES;
      std::memcpy(host + map[i].first * MS_PAGE_BYTES, src, MS_PAGE_BYTES);
      if (wipe) std::memset(src, 0, MS_PAGE_BYTES);
    });
  }
  const uint64_t t = now_ns();
  st_scatter_ns.fetch_add(t - ts);
  uint64_t pages = 0;
  {
    // qmu guards the admission state (shared with form_wave) and lat_out
    // (a replay that gives up detaches its outstanding requests under it)
    std::lock_guard<std::mutex> lk(qmu);
    adm->release(w, [&](uint64_t t) -> const std::vector<uint64_t> & { return slot(t).pages; });
    for (uint64_t tk : w.tickets) {
      Req &r = slot(tk);
      if (r.lat_out) *r.lat_out = (double)((int64_t)(t - r.t_sched_ns)) * 1e-9;
      r.lat_out = nullptr;
    }
  }
  for (uint64_t tk : w.tickets) {
    Req &r = slot(tk);
    pages += r.pages.size();
    r.t_done_ns.store(t);
    r.state.store(kDone, std::memory_order_release);
  }
  ev_pool.push_back({w.ev_h2d, w.ev_done});
  st_req.fetch_add(w.tickets.size());
  st_pages.fetch_add(pages);
  {
    std::lock_guard<std::mutex> lk(done_mu);
  }
  done_cv.notify_all();
}

void ms_server::fail_all(int code) {
  error.store(code);
  take_inbox(true);  // a submission that saw no error under inmu is in the inbox by now
  std::lock_guard<std::mutex> lk(qmu);
  for (auto *set : {&inflight, &inflight_inplace})
    for (Wave &w : *set)
      for (uint64_t t : w.tickets) {
        slot(t).error.store(code);
        slot(t).state.store(kDone);
      }
  for (uint64_t t : incoming) {
    slot(t).error.store(code);
    slot(t).state.store(kDone);
  }
  incoming.clear();
  {
    std::lock_guard<std::mutex> lk2(done_mu);
  }
  done_cv.notify_all();
}

void ms_server::loop() {
  DeviceGuard g(ctx->device);
  // short naps must stay short: drop this thread's timer slack (default 50 us)
  prctl(PR_SET_TIMERSLACK, 1000UL, 0, 0, 0);
  uint64_t stop_deadline = 0;
  uint64_t idle_since = 0;
  for (;;) {
    bool progress = false;
    const uint64_t t_pass = now_ns();
    while (!inflight.empty()) {
      cudaError_t q = cudaEventQuery(inflight.front().ev_done);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) {
        cuda_fail(ctx, q);
        fail_all(MS_ECUDA);
        exited.store(true);
        return;
      }
      complete(inflight.front());
      inflight.pop_front();
      progress = true;
    }
    for (auto it = inflight_inplace.begin(); it != inflight_inplace.end();) {
      cudaError_t q = cudaEventQuery(it->ev_done);
      if (q == cudaErrorNotReady) {
        ++it;
        continue;
      }
      if (q != cudaSuccess) {
        cuda_fail(ctx, q);
        fail_all(MS_ECUDA);
        exited.store(true);
        return;
      }
      complete(*it);
      it = inflight_inplace.erase(it);
      progress = true;
    }
    const bool stopping = stop.load();
    const bool missed = !take_inbox(stopping);  // stopping: every request submitted so far must be seen
    if (stopping) {
      const bool empty = incoming.empty();
      if (empty && inflight.empty() && inflight_inplace.empty()) break;
      if (!stop_deadline) stop_deadline = now_ns() + (uint64_t)ctx->cfg.timeout_ms * 1000000ull;
      if (now_ns() > stop_deadline) {
        fail_all(MS_ETIMEDOUT);
        break;
      }
    }
    // While a longer wave is in flight (the load outgrew the lane), the lane
    // narrows to one wave of at most kInplaceBusyPages pages: the longer
    // waves carry the bulk, and a short queue between them still goes
    // through the lane.
    const bool long_busy = !inflight.empty();
    const uint32_t lane_pages = long_busy ? std::min(inplace_max, kInplaceBusyPages) : inplace_max;
    const size_t lane_depth = long_busy ? 1 : kInplaceDepth;
    bool formed = false;
    if (inplace_max && inflight_inplace.size() < lane_depth && error.load() == 0) {
      Wave w;
      if (form_inplace(w, lane_pages)) {
        int rc = issue_inplace(w);
        if (rc != MS_OK) {
          inflight_inplace.push_back(w);
          fail_all(rc);
          exited.store(true);
          return;
        }
        inflight_inplace.push_back(std::move(w));
        progress = formed = true;
      }
    }
    if (!formed && inflight.size() < cfg.waves_in_flight && error.load() == 0) {
      Wave w;
      if (form_wave(w)) {
        int rc = issue(w);
        if (rc != MS_OK) {
          inflight.push_back(w);
          fail_all(rc);
          exited.store(true);
          return;
        }
        inflight.push_back(std::move(w));
        progress = true;
      }
    }
    atomic_max(st_max_pass, now_ns() - t_pass);  // this pass's work, without its idle waits
    if (progress || missed) {  // missed: a submission is in the inbox, take it next pass
      idle_since = 0;
      continue;
    }
    if (inflight.empty() && inflight_inplace.empty()) {
      // idle: watch the ticket counter for a while before blocking, so a
      // request that arrives soon is picked up without a wake-up delay (a
      // request submitted since the last take of the inbox ends the wait
      // at once)
      const uint64_t seen = taken_upto, t_idle = now_ns();
      while (next_ticket.load() == seen && !stop.load() && now_ns() - t_idle < idle_spin_ns) nap_ns(1000);
      if (next_ticket.load() == seen && !stop.load()) {
        std::unique_lock<std::mutex> lk(inmu);
        qcv.wait_for(lk, std::chrono::milliseconds(1), [&] { return !inbox.empty() || stop.load(); });
      }
    } else {
      // a wave is on the GPU: poll, spinning briefly before napping
      const uint64_t t = now_ns();
      if (!idle_since) idle_since = t;
      if (t - idle_since > 20000) nap_ns(2000);
    }
  }
  exited.store(true);
}

extern "C" {

void ms_server_config_default(ms_server_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->staging_bytes = (uint64_t)256 << 20;
  cfg->waves_in_flight = 2;
  cfg->copy_threads = 4;
  cfg->max_pending = 1u << 18;
  cfg->mode = MS_SERVE_CONTINUOUS;
  cfg->max_request_pages = 4096;
  cfg->idle_spin_us = 20000;
  cfg->zero_copy_max_pages = 512;  // the in-place lane: queues of up to 512 pages (its parameter limit)
}

static void free_server(ms_server *s) {
  if (s->pool) delete s->pool;
  if (s->adm) delete s->adm;
  for (auto &p : s->ev_pool) {
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  if (s->s_in) cudaStreamDestroy(s->s_in);
  if (s->s_link) cudaStreamDestroy(s->s_link);
  for (auto &w : s->s_work)
    if (w) cudaStreamDestroy(w);
  if (s->h_stage) cudaFreeHost(s->h_stage);
  if (s->h_ent) cudaFreeHost(s->h_ent);
  if (s->d_stage) cudaFree(s->d_stage);
  if (s->d_ent) cudaFree(s->d_ent);
  delete s;
}

int ms_server_create(ms_ctx *c, void *host_base, uint64_t n_pages, const ms_server_config *cfg_in,
                     ms_server **out) {
  if (!out) return MS_EINVAL;
  *out = nullptr;
  if (!c || !c->alive) return MS_ENOTINIT;
  if (!host_base || n_pages == 0) return MS_EINVAL;
  ms_server_config cfg;
  if (cfg_in) cfg = *cfg_in; else ms_server_config_default(&cfg);
  if (cfg.staging_bytes == 0) cfg.staging_bytes = (uint64_t)256 << 20;
  if (cfg.staging_bytes % MS_PAGE_BYTES || cfg.staging_bytes / MS_PAGE_BYTES > (1u << 24)) return MS_EINVAL;
  if (cfg.waves_in_flight == 0) cfg.waves_in_flight = 2;
  if (cfg.waves_in_flight > 8 || cfg.copy_threads > 32) return MS_EINVAL;
  if (cfg.max_pending == 0) cfg.max_pending = 1u << 18;
  if (cfg.max_pending > (1u << 24)) return MS_EINVAL;
  if (cfg.mode != MS_SERVE_CONTINUOUS && cfg.mode != MS_SERVE_ONE_PER_LAUNCH && cfg.mode != MS_SERVE_ZERO_COPY)
    return MS_EINVAL;
  const uint32_t S = (uint32_t)(cfg.staging_bytes / MS_PAGE_BYTES);
  if (cfg.max_wave_pages == 0) cfg.max_wave_pages = std::max<uint32_t>(1, S / cfg.waves_in_flight);
  if (cfg.max_request_pages == 0) cfg.max_request_pages = 4096;
  if (cfg.max_request_pages > S || cfg.max_request_pages > cfg.max_wave_pages) return MS_EINVAL;
  if (cfg.zero_copy_max_pages > 512) return MS_EINVAL;  // an in-place wave's entries fit the kernel parameters

  ms_server *s = new (std::nothrow) ms_server();
  if (!s) return MS_ENOMEM;
  s->ctx = c;
  s->host = (uint8_t *)host_base;
  s->n_pages = n_pages;
  s->cfg = cfg;
  s->S = S;
  s->idle_spin_ns = (uint64_t)cfg.idle_spin_us * 1000ull;
  DeviceGuard g(c->device);
  if (cfg.mode == MS_SERVE_ZERO_COPY || (cfg.mode == MS_SERVE_CONTINUOUS && cfg.zero_copy_max_pages)) {
    void *dp = nullptr;
    if (cudaHostGetDevicePointer(&dp, host_base, 0) != cudaSuccess || !dp) {
      cudaGetLastError();
      if (cfg.mode == MS_SERVE_ZERO_COPY) {
        delete s;
        return MS_EINVAL;  // the working set is not pinned, mapped host memory
      }
      s->cfg.zero_copy_max_pages = 0;  // pageable working set: every wave is staged
    } else {
      s->d_host = (uint64_t)dp;
      if (cfg.mode == MS_SERVE_CONTINUOUS) s->inplace_max = std::min(cfg.zero_copy_max_pages, cfg.max_wave_pages);
    }
  }
  cudaError_t e = cudaHostAlloc(&s->h_stage, (size_t)S * MS_PAGE_BYTES, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaHostAlloc(&s->h_ent, (size_t)S * sizeof(ms_page_dom), cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_stage, (size_t)S * MS_PAGE_BYTES);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_ent, (size_t)S * sizeof(ms_page_dom));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_work[0], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_work[1], cudaStreamNonBlocking);
  if (e == cudaSuccess && (s->inplace_max || cfg.mode == MS_SERVE_ZERO_COPY)) {
    int lo = 0, hi = 0;  // the link stream at the highest priority: a fault waits on it
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    e = cudaStreamCreateWithPriority(&s->s_link, cudaStreamNonBlocking, hi);
  }
  if (e != cudaSuccess) {
    free_server(s);
    return alloc_fail(c, e);
  }
  try {
    s->reqs = std::vector<Req>(cfg.max_pending);
    s->adm = new ms::Admission(S, cfg.max_wave_pages, cfg.mode == MS_SERVE_ONE_PER_LAUNCH, n_pages, kScanWindow);
    s->pool = new CopyPool((int)cfg.copy_threads);
    s->th = std::thread([s] { s->loop(); });
  } catch (...) {
    free_server(s);
    return MS_ENOMEM;
  }
  c->children.fetch_add(1);
  *out = s;
  return MS_OK;
}

// `checked`: the request was validated already (a replay checks every
// request before its first submission).
static int submit_internal(ms_server *s, int op, uint32_t domain, const uint64_t *page_index, uint32_t n,
                           uint64_t *ticket, uint64_t t_sched, double *lat_out, bool checked = false) {
  if (!s) return MS_EINVAL;
  if (!checked) {
    if (op != MS_ENCRYPT && op != MS_DECRYPT) return MS_EINVAL;
    if (n == 0 || !page_index) return MS_EINVAL;
    if (n > s->cfg.max_request_pages) return MS_ERANGE;
    for (uint32_t i = 0; i < n; ++i)
      if (page_index[i] >= s->n_pages) return MS_EINVAL;
    // distinct pages within a request (two in-place updates of one page in one wave would race)
    if (n > 1) {
      std::vector<uint64_t> tmp(page_index, page_index + n);
      std::sort(tmp.begin(), tmp.end());
      if (std::adjacent_find(tmp.begin(), tmp.end()) != tmp.end()) return MS_EINVAL;
    }
  }
  std::unique_lock<std::mutex> lk(s->inmu);
  if (s->error.load()) return s->error.load();  // under inmu: fail_all drains the inbox after setting it
  if (s->stop.load()) return MS_ENOTINIT;
  const uint64_t t = s->next_ticket.load();
  Req &r = s->slot(t);
  int st = r.state.load();
  if (st == kQueued || st == kAdmitted || st == kClaiming) return MS_EBUSY;
  r.state.store(kClaiming);
  r.ticket.store(t);  // before next_ticket: a poll that sees ticket t valid finds the slot claimed
  s->next_ticket.store(t + 1);
  r.op = op;
  r.domain = domain;
  r.pages.assign(page_index, page_index + n);
  r.error.store(0);
  r.t_done_ns.store(0);
  r.t_sched_ns = t_sched ? t_sched : now_ns();
  r.lat_out = lat_out;
  r.state.store(kQueued, std::memory_order_release);
  s->inbox.push_back(t);
  if (ticket) *ticket = t;
  lk.unlock();
  s->qcv.notify_one();  // after the unlock: the server thread wakes to a free lock
  return MS_OK;
}

int ms_server_submit(ms_server *s, int op, const uint64_t *page_index, uint32_t n, uint64_t *ticket) {
  if (!s) return MS_EINVAL;
  return submit_internal(s, op, s->ctx->cfg.domain, page_index, n, ticket, 0, nullptr);
}

int ms_server_submit_dom(ms_server *s, int op, uint32_t domain, const uint64_t *page_index, uint32_t n,
                         uint64_t *ticket) {
  return submit_internal(s, op, domain, page_index, n, ticket, 0, nullptr);
}

int ms_server_poll(ms_server *s, uint64_t ticket) {
  if (!s) return MS_EINVAL;
  if (ticket >= s->next_ticket.load()) return MS_EINVAL;
  Req &r = s->slot(ticket);
  const uint64_t owner = r.ticket.load();
  if (owner != ticket) return owner > ticket && owner != ~0ull ? 1 : 0;  // reused: finished long ago
  const int st = r.state.load(std::memory_order_acquire);
  if (st != kDone) return 0;
  const int err = r.error.load();
  return err ? err : 1;
}

int ms_server_wait(ms_server *s, uint64_t ticket, uint32_t timeout_ms) {
  if (!s) return MS_EINVAL;
  const auto deadline = clk::now() + std::chrono::milliseconds(timeout_ms);
  // poll for ~50 us first: most waits end within a wave's round trip
  const auto spin_end = clk::now() + std::chrono::microseconds(50);
  int p = ms_server_poll(s, ticket);
  while (p == 0 && clk::now() < spin_end && clk::now() < deadline) {
    nap_ns(1000);
    p = ms_server_poll(s, ticket);
  }
  if (p == 0) {
    // the completing thread stores the state, then takes done_mu and notifies:
    // checking the state under done_mu cannot miss that notification
    std::unique_lock<std::mutex> lk(s->done_mu);
    s->done_cv.wait_until(lk, deadline, [&] { return (p = ms_server_poll(s, ticket)) != 0; });
  }
  if (p < 0) return p;
  return p == 1 ? MS_OK : MS_ETIMEDOUT;
}

int ms_server_replay(ms_server *s, size_t n, const double *arrival_s, const int *ops, const uint32_t *domains,
                     const uint64_t *offsets, const uint64_t *page_index, double *latency_s, double *makespan_s,
                     uint32_t timeout_ms) {
  if (!s || (n && (!arrival_s || !ops || !offsets || !page_index || !latency_s))) return MS_EINVAL;
  // every request is checked before the first one is submitted
  for (size_t r = 0; r < n; ++r) {
    if (offsets[r + 1] <= offsets[r] || (ops[r] != MS_ENCRYPT && ops[r] != MS_DECRYPT)) return MS_EINVAL;
    if (offsets[r + 1] - offsets[r] > s->cfg.max_request_pages) return MS_ERANGE;
    for (uint64_t k = offsets[r]; k < offsets[r + 1]; ++k)
      if (page_index[k] >= s->n_pages) return MS_EINVAL;
    if (offsets[r + 1] - offsets[r] > 1) {  // distinct pages within a request
      std::vector<uint64_t> tmp(page_index + offsets[r], page_index + offsets[r + 1]);
      std::sort(tmp.begin(), tmp.end());
      if (std::adjacent_find(tmp.begin(), tmp.end()) != tmp.end()) return MS_EINVAL;
    }
    latency_s[r] = -1.0;
  }
  // precise pacing: short timer slack for this thread while replaying
  const int old_slack = prctl(PR_GET_TIMERSLACK, 0, 0, 0, 0);
  prctl(PR_SET_TIMERSLACK, 1000UL, 0, 0, 0);
  struct SlackRestore {
    int v;
    ~SlackRestore() {
      if (v > 0) prctl(PR_SET_TIMERSLACK, (unsigned long)v, 0, 0, 0);
    }
  } restore{old_slack};
  const uint64_t t0 = now_ns() + 1000000ull;  // start 1 ms from now
  uint64_t max_lag = 0, late = 0;  // how far submissions ran behind their schedule
  s->st_max_pass.store(0);         // the longest server pass is reported per replay
  std::vector<uint64_t> tickets(n);
  size_t issued = 0;
  // On an early return the requests still queued or running must stop
  // pointing into latency_s, which the caller may free once this returns.
  auto detach = [&](int rc) {
    std::lock_guard<std::mutex> lk(s->qmu);
    for (size_t r = 0; r < issued; ++r) {
      Req &q = s->slot(tickets[r]);
      if (q.ticket.load() == tickets[r]) q.lat_out = nullptr;
    }
    return rc;
  };
  for (size_t r = 0; r < n; ++r) {
    const uint64_t target = t0 + (uint64_t)(arrival_s[r] * 1e9);
    for (;;) {
      const uint64_t t = now_ns();
      if (t >= target) break;
      // sleep only through long gaps and wake 1 ms early, spin otherwise: an
      // idle virtual CPU can wake milliseconds late, and a late submission
      // counts as latency (arrivals are scheduled)
      if (target - t > 2000000) nap_ns((long)(target - t - 1000000));
    }
    const uint64_t n_pg = offsets[r + 1] - offsets[r];
    const uint64_t spin_limit = now_ns() + (uint64_t)timeout_ms * 1000000ull;
    for (;;) {
      const uint32_t dom = domains ? domains[r] : s->ctx->cfg.domain;
      int rc = submit_internal(s, ops[r], dom, page_index + offsets[r], (uint32_t)n_pg, &tickets[r], target,
                               &latency_s[r], true);
      if (rc == MS_OK) {
        issued = r + 1;
        const uint64_t lag = now_ns() - target;
        max_lag = std::max(max_lag, lag);
        late += lag > 1000000ull;
        break;
      }
      if (rc != MS_EBUSY) return detach(rc);
      if (now_ns() > spin_limit) return detach(MS_ETIMEDOUT);
      nap_ns(5000);
    }
  }
  s->st_replay_lag.store(max_lag);
  s->st_replay_late.store(late);
  const uint64_t deadline = now_ns() + (uint64_t)timeout_ms * 1000000ull;
  uint64_t last = t0;
  for (size_t r = 0; r < n; ++r) {
    for (;;) {
      int p = ms_server_poll(s, tickets[r]);
      if (p < 0) return detach(p);
      if (p == 1) break;
      if (now_ns() > deadline) return detach(MS_ETIMEDOUT);
      nap_ns(5000);
    }
  }
  for (size_t r = 0; r < n; ++r) {
    const uint64_t target = t0 + (uint64_t)(arrival_s[r] * 1e9);
    last = std::max(last, target + (uint64_t)std::max(0.0, latency_s[r] * 1e9));
  }
  if (makespan_s) *makespan_s = (double)(last - t0) * 1e-9;
  return MS_OK;
}

int ms_server_get_stats(const ms_server *s, ms_server_stats *out) {
  if (!s || !out) return MS_EINVAL;
  out->requests_done = s->st_req.load();
  out->pages_done = s->st_pages.load();
  out->waves = s->st_waves.load();
  out->max_wave_requests = s->st_maxreq.load();
  out->max_wave_pages = s->st_maxpages.load();
  out->conflict_waits = s->st_conflict.load();
  out->budget_waits = s->st_budget.load();
  out->max_staged_pages = s->st_maxstaged.load();
  out->gather_ns = s->st_gather_ns.load();
  out->scatter_ns = s->st_scatter_ns.load();
  out->inplace_waves = s->st_inplace.load();
  out->staged_waves = s->st_staged.load();
  out->max_pass_ns = s->st_max_pass.load();
  out->replay_max_lag_ns = s->st_replay_lag.load();
  out->replay_late = s->st_replay_late.load();
  return MS_OK;
}

int ms_server_destroy(ms_server *s) {
  if (!s) return MS_OK;
  s->stop.store(true);
  s->qcv.notify_all();
  if (s->th.joinable()) s->th.join();
  int rc = s->error.load();
  DeviceGuard g(s->ctx->device);
  // everything the server issued must be finished before its buffers go:
  // the waves still listed, and any copy of a wave whose issue failed midway
  for (auto *set : {&s->inflight, &s->inflight_inplace})
    for (Wave &w : *set) {
      if (!w.ev_done) continue;  // its issue failed before it had events
      int r = wait_event(s->ctx, w.ev_done, s->ctx->cfg.timeout_ms);
      if (r != MS_OK) return r;  // still running on the GPU: leave the buffers allocated
    }
  for (cudaStream_t st : {s->s_in, s->s_work[0], s->s_work[1], s->s_link}) {
    if (!st) continue;
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return cuda_fail(s->ctx, cudaGetLastError());
    cudaError_t e = cudaEventRecord(ev, st);
    int r = e == cudaSuccess ? wait_event(s->ctx, ev, s->ctx->cfg.timeout_ms) : cuda_fail(s->ctx, e);
    cudaEventDestroy(ev);
    if (r != MS_OK) return r;
  }
  for (auto *set : {&s->inflight, &s->inflight_inplace})
    for (Wave &w : *set)
      if (w.ev_done) s->ev_pool.push_back({w.ev_h2d, w.ev_done});
  s->inflight.clear();
  s->inflight_inplace.clear();
  ms_ctx *c = s->ctx;
  free_server(s);
  c->children.fetch_sub(1);
  return rc == MS_ETIMEDOUT ? MS_ETIMEDOUT : (rc ? rc : MS_OK);
}

}  // extern "C"
