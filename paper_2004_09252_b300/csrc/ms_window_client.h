// The sliding-window client and its background evictor (Sec. 4.3 policy,
// background eviction as proposed in the paper's conclusions), written over
// an abstract backend so that the same code drives the GPU backends of
// ms_window.cu and the CPU simulator of the tests.  Plain C++: no CUDA.
//
// A Backend provides, all returning MS_OK or an MS_E* code:
//   fault_submit(domain, page, &ticket)  queue a one-page decrypt
//   fault_wait(ticket)                   wait for it
//   evict(domain, pages, k, background)  queue an encrypt of k pages (not waited for);
//                                        background: called by the evictor thread
//   wait_evicted()                       wait for the client's latest own (overflow)
//                                        eviction (sync_evict)
//   drain()                              wait for every eviction queued
// A page's requests reach the backend in the order of the window's changes
// (fault_submit under the client's window lock; an eviction before any later
// fault on its pages), and the backend must apply them in that order.  The
// background evictor calls evict from its own thread, concurrently with the
// client's calls: a backend's calls must be safe to make from two threads.
#pragma once

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_set>
#include <vector>

#include "memshield.h"

namespace ms {
namespace window {

using clk = std::chrono::steady_clock;

// One client's run: its description, its counters, its fault latencies and
// its window at the end.
struct ClientRun {
  const ms_window_client *cl;
  ms_window_stats st{};
  std::vector<double> lat_us;
  std::vector<uint64_t> final_window;
  int rc = MS_OK;
};

// The window a client shares with its evictor.  Every field but `size` and
// `evictor_asleep` is guarded by mu.
struct Window {
  std::mutex mu;
  std::condition_variable wake;       // wakes an evictor that has gone to sleep
  std::condition_variable submitted;  // an eviction taken out of the window reached the backend
  std::deque<uint64_t> pages;         // working-set page indices in clear, oldest first
  std::unordered_set<uint64_t> members;
  std::vector<uint64_t> evicting;     // taken out by the evictor, eviction not yet submitted
  std::atomic<size_t> size{0};        // pages.size(), read by the evictor without mu
  std::atomic<bool> evictor_asleep{false};
  bool done = false;                  // the client has finished its trace
  int rc = MS_OK;                     // the first error of either thread
};

// Take the oldest k pages out of the window; caller holds w.mu.
inline std::vector<uint64_t> take_oldest(Window &w, size_t k) {
  std::vector<uint64_t> ev(w.pages.begin(), w.pages.begin() + (long)k);
  w.pages.erase(w.pages.begin(), w.pages.begin() + (long)k);
  for (uint64_t e : ev) w.members.erase(e);
  w.size.store(w.pages.size(), std::memory_order_relaxed);
  return ev;
}

inline void count_eviction(ClientRun &cr, size_t k, bool background) {
  cr.st.evictions += k;
  cr.st.evict_requests += 1;
  if (background) {
    cr.st.background_evictions += k;
    cr.st.background_requests += 1;
  }
}

// The background evictor: whenever fewer than T slots are free, take the
// oldest evict_batch pages out of the window and encrypt them by one request,
// again until at least T slots are free.  A batch larger than the shortfall
// evicts ahead of need.  The pages leave the window under the lock but the
// request is submitted outside it, so the client keeps faulting meanwhile; a
// fault on one of those very pages waits until its eviction is submitted
// (Window::evicting), which keeps the per-page order.  Between triggers the
// evictor polls the window's size for a while before it sleeps, so that the
// client rarely pays for a wake-up.
template <typename Backend>
void run_evictor(Backend &be, const ms_window_config &cfg, Window &w, uint32_t domain, ClientRun &cr) {
  const size_t keep = cfg.window_pages - cfg.background_free;  // pages the window may hold at rest
  for (;;) {
    const auto spin_end = clk::now() + std::chrono::microseconds(200);
    while (w.size.load(std::memory_order_relaxed) <= keep && clk::now() < spin_end) std::this_thread::yield();
    std::unique_lock<std::mutex> lk(w.mu);
    if (w.pages.size() <= keep && !w.done && w.rc == MS_OK) {
      w.evictor_asleep.store(true);
      w.wake.wait(lk, [&] { return w.done || w.rc != MS_OK || w.pages.size() > keep; });
      w.evictor_asleep.store(false);
    }
    while (w.rc == MS_OK && w.pages.size() > keep) {
      const size_t k = std::min<size_t>(cfg.evict_batch, w.pages.size());
      std::vector<uint64_t> ev = take_oldest(w, k);
      w.evicting.insert(w.evicting.end(), ev.begin(), ev.end());
      lk.unlock();
      const int rc = be.evict(domain, ev.data(), k, true);
      lk.lock();
      for (uint64_t e : ev) w.evicting.erase(std::find(w.evicting.begin(), w.evicting.end(), e));
      w.submitted.notify_all();
      if (rc != MS_OK) {
        w.rc = rc;
        break;
      }
      count_eviction(cr, k, true);
    }
    if (w.done || w.rc != MS_OK) return;
  }
}

template <typename Backend>
void run_client(Backend &be, const ms_window_config &cfg, ClientRun &cr) {
  const ms_window_client &cl = *cr.cl;
  const bool bg = cfg.background_free != 0;
  const size_t keep = cfg.window_pages - cfg.background_free;
  Window w;
  cr.lat_us.reserve(cl.trace_len / 4 + 16);
  std::thread evictor;
  if (bg) evictor = std::thread([&] { run_evictor(be, cfg, w, cl.domain, cr); });
  const auto t0 = clk::now();
  int rc = MS_OK;
  for (size_t i = 0; i < cl.trace_len && rc == MS_OK; ++i) {
    const uint64_t rel = cl.trace[i];
    if (rel >= cl.n_pages) {
      rc = MS_EINVAL;
      break;
    }
    const uint64_t pg = cl.first_page + rel;
    uint64_t ticket = 0;
    std::chrono::steady_clock::time_point f0;
    {
      std::unique_lock<std::mutex> lk(w.mu);
      if (w.rc != MS_OK) {
        rc = w.rc;
        break;
      }
      cr.st.accesses += 1;
      if (w.members.count(pg)) {
        cr.st.hits += 1;
        continue;
      }
      f0 = clk::now();
      // fault: a page the evictor has just taken out is decrypted only after
      // its eviction is submitted, and the decrypt is submitted under the lock
      w.submitted.wait(lk, [&] {
        return w.rc != MS_OK || std::find(w.evicting.begin(), w.evicting.end(), pg) == w.evicting.end();
      });
      rc = w.rc != MS_OK ? w.rc : be.fault_submit(cl.domain, pg, &ticket);
    }
    if (rc == MS_OK) rc = be.fault_wait(ticket);  // the faulting thread is stalled until it is resolved
    if (rc != MS_OK) break;
    cr.lat_us.push_back(std::chrono::duration<double, std::micro>(clk::now() - f0).count());
    bool evicted = false;
    {
      std::lock_guard<std::mutex> lk(w.mu);
      cr.st.faults += 1;
      w.pages.push_back(pg);
      w.members.insert(pg);
      w.size.store(w.pages.size(), std::memory_order_relaxed);
      if (w.pages.size() > cfg.window_pages) {  // overflow (without an evictor, or one running behind)
        const size_t k = std::min<size_t>(cfg.evict_batch, w.pages.size());
        std::vector<uint64_t> ev = take_oldest(w, k);
        rc = be.evict(cl.domain, ev.data(), k, false);
        if (rc != MS_OK) break;
        count_eviction(cr, k, false);
        evicted = true;
      }
      if (bg && w.pages.size() > keep && w.evictor_asleep.load()) w.wake.notify_one();
    }
    // the paper's server finishes a fault's eviction before it takes the next fault
    if (evicted && cfg.sync_evict) rc = be.wait_evicted();
  }
  if (bg) {
    {
      std::lock_guard<std::mutex> lk(w.mu);
      w.done = true;
      if (rc != MS_OK && w.rc == MS_OK) w.rc = rc;
    }
    w.wake.notify_one();
    evictor.join();  // it brings the window back to T free slots before it leaves
    if (rc == MS_OK) rc = w.rc;
  }
  // the client's evictions complete before it reports
  if (rc == MS_OK) rc = be.drain();
  if (rc != MS_OK) {
    cr.rc = rc;
    return;
  }
  cr.st.elapsed_s = std::chrono::duration<double>(clk::now() - t0).count();
  cr.final_window.assign(w.pages.begin(), w.pages.end());
}

inline double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t lo = (size_t)pos;
  const size_t hi = std::min(v.size() - 1, lo + 1);
  return v[lo] + (v[hi] - v[lo]) * (pos - (double)lo);
}

}  // namespace window
}  // namespace ms
