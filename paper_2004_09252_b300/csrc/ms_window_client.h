// The sliding-window client and its background evictor (Sec. 4.3 policy,
// background eviction as proposed in the paper's conclusions), written over
// an abstract backend so that the same code drives the GPU backends of
// ms_window.cu and the CPU simulator of the tests.  Plain C++: no CUDA.
//
// A Backend provides, all returning MS_OK or an MS_E* code:
//   fault_submit(domain, page, &ticket)  queue a one-page decrypt
//   fault_wait(ticket)                   wait for it
//   evict(domain, pages, k)              queue an encrypt of k pages (not waited for)
//   drain()                              wait for every eviction queued
// fault_submit and evict are only called under the client's window lock, so
// the order in which they reach the backend is the order of the window's
// changes; the backend must apply a page's requests in that order.
#pragma once

#include <algorithm>
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

// The window a client shares with its evictor (all fields under mu).
struct Window {
  std::mutex mu;
  std::condition_variable cv;  // wakes the evictor
  std::deque<uint64_t> pages;  // working-set page indices in clear, oldest first
  std::unordered_set<uint64_t> members;
  bool done = false;           // the client has finished its trace
  int rc = MS_OK;              // the first error of either thread
};

// Encrypt the oldest k pages of the window (one request); caller holds w.mu.
template <typename Backend>
int evict_oldest(Backend &be, Window &w, uint32_t domain, size_t k, ClientRun &cr, bool background) {
  std::vector<uint64_t> ev(w.pages.begin(), w.pages.begin() + (long)k);
  w.pages.erase(w.pages.begin(), w.pages.begin() + (long)k);
  for (uint64_t e : ev) w.members.erase(e);
  const int rc = be.evict(domain, ev.data(), k);
  if (rc != MS_OK) return rc;
  cr.st.evictions += k;
  cr.st.evict_requests += 1;
  if (background) {
    cr.st.background_evictions += k;
    cr.st.background_requests += 1;
  }
  return MS_OK;
}

// The background evictor: whenever fewer than T slots are free, encrypt the
// oldest evict_batch pages in one request, again until at least T are free.
// A batch larger than the shortfall evicts ahead of need: one wake-up and
// one request serve evict_batch faults.
template <typename Backend>
void run_evictor(Backend &be, const ms_window_config &cfg, Window &w, uint32_t domain, ClientRun &cr) {
  const size_t keep = cfg.window_pages - cfg.background_free;  // pages the window may hold at rest
  std::unique_lock<std::mutex> lk(w.mu);
  for (;;) {
    w.cv.wait(lk, [&] { return w.done || w.rc != MS_OK || w.pages.size() > keep; });
    while (w.rc == MS_OK && w.pages.size() > keep) {
      const size_t k = std::min<size_t>(cfg.evict_batch, w.pages.size());
      const int rc = evict_oldest(be, w, domain, k, cr, true);
      if (rc != MS_OK) w.rc = rc;
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
      std::lock_guard<std::mutex> lk(w.mu);
      if (w.rc != MS_OK) {
        rc = w.rc;
        break;
      }
      cr.st.accesses += 1;
      if (w.members.count(pg)) {
        cr.st.hits += 1;
        continue;
      }
      // fault: the decrypt is submitted under the lock, after any eviction of this page
      f0 = clk::now();
      rc = be.fault_submit(cl.domain, pg, &ticket);
    }
    if (rc == MS_OK) rc = be.fault_wait(ticket);  // the faulting thread is stalled until it is resolved
    if (rc != MS_OK) break;
    cr.lat_us.push_back(std::chrono::duration<double, std::micro>(clk::now() - f0).count());
    std::lock_guard<std::mutex> lk(w.mu);
    cr.st.faults += 1;
    w.pages.push_back(pg);
    w.members.insert(pg);
    if (w.pages.size() > cfg.window_pages) {  // overflow (without an evictor, or one running behind)
      rc = evict_oldest(be, w, cl.domain, std::min<size_t>(cfg.evict_batch, w.pages.size()), cr, false);
      if (rc != MS_OK) break;
    }
    if (bg && w.pages.size() > keep) w.cv.notify_one();
  }
  if (bg) {
    {
      std::lock_guard<std::mutex> lk(w.mu);
      w.done = true;
      if (rc != MS_OK && w.rc == MS_OK) w.rc = rc;
    }
    w.cv.notify_one();
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

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t lo = (size_t)pos;
  const size_t hi = std::min(v.size() - 1, lo + 1);
  return v[lo] + (v[hi] - v[lo]) * (pos - (double)lo);
}

}  // namespace window
}  // namespace ms
