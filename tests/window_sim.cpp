// Host-only simulation of the sliding-window clients and their background
// evictors (ms_window_client.h, the code the GPU backends run), served by a
// fake GPU: executor threads that apply each request to a per-page
// encrypted/clear flag after a random delay.  The fake applies a page's
// requests in submission order, as the library's backends do: with one
// executor in stream order, with several under the server's in-flight rule
// (a request waits while an earlier unfinished request shares a page).
//
// Checks:
//   - every decrypt finds its page encrypted and every encrypt finds it
//     clear (no page is decrypted twice, or evicted before its fault);
//   - at the end exactly the pages of each client's final window are clear;
//   - the counters agree: hits + faults = accesses, faults - evictions =
//     final window size, the background counters are part of the totals;
//   - with background eviction the final window holds at most
//     window_pages - background_free pages, and the evictor did evict.
// "reorder" = 1 lets the executors run requests in any order, which must be
// caught (the checks are not vacuous).
// Usage: window_sim seed clients client_pages trace_len window evict_batch background_free executors reorder
//        [sync_evict]
#include <atomic>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <deque>
#include <memory>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "ms_window_client.h"

namespace {

uint64_t mix(uint64_t z) {  // splitmix64 output function
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Job {
  int op;
  std::vector<uint64_t> pages;
  bool running = false, done = false;
};

class FakeGpu {
 public:
  FakeGpu(uint64_t n_pages, int executors, bool reorder, uint64_t seed)
      : enc_(n_pages, 1), reorder_(reorder), seed_(seed) {
    for (int i = 0; i < executors; ++i) th_.emplace_back([this, i] { run(i); });
  }
  ~FakeGpu() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto &t : th_) t.join();
  }
  uint64_t submit(int op, const uint64_t *pages, size_t k) {
    std::lock_guard<std::mutex> lk(mu_);
    auto j = std::make_unique<Job>();
    j->op = op;
    j->pages.assign(pages, pages + k);
    jobs_.push_back(std::move(j));
    pending_.push_back(jobs_.size() - 1);
    cv_.notify_all();
    return jobs_.size() - 1;
  }
  int wait(uint64_t t) {
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return jobs_[t]->done; });
    return MS_OK;
  }
  int violations() const { return violations_.load(); }
  bool encrypted(uint64_t pg) {
    std::lock_guard<std::mutex> lk(mu_);
    return enc_[pg] != 0;
  }

 private:
  // The first pending job that may start: none of its pages belongs to an
  // earlier job that is still pending or running (unless reordering).
  long pick(uint64_t r) {
    if (pending_.empty()) return -1;
    if (reorder_) return (long)(r % pending_.size());
    std::set<uint64_t> blocked(busy_.begin(), busy_.end());
    for (size_t i = 0; i < pending_.size(); ++i) {
      const Job &j = *jobs_[pending_[i]];
      bool ok = true;
      for (uint64_t pg : j.pages)
        if (blocked.count(pg)) ok = false;
      if (ok) return (long)i;
      for (uint64_t pg : j.pages) blocked.insert(pg);
    }
    return -1;
  }
  void run(int id) {
    uint64_t r = mix(seed_ * 977 + (uint64_t)id);
    std::unique_lock<std::mutex> lk(mu_);
    for (;;) {
      long i;
      cv_.wait(lk, [&] { return stop_ || (i = pick(r = mix(r))) >= 0; });
      if (stop_) return;
      const uint64_t t = pending_[(size_t)i];
      pending_.erase(pending_.begin() + i);
      Job &j = *jobs_[t];
      j.running = true;
      for (uint64_t pg : j.pages) busy_.insert(pg);
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(r % 40));
      lk.lock();
      for (uint64_t pg : j.pages) {
        const int want = j.op == MS_DECRYPT ? 1 : 0;  // decrypt needs ciphertext, encrypt needs clear text
        if (enc_[pg] != want) violations_.fetch_add(1);
        enc_[pg] = (uint8_t)(1 - want);
        busy_.erase(busy_.find(pg));
      }
      j.running = false;
      j.done = true;
      done_cv_.notify_all();
      cv_.notify_all();
    }
  }
  std::mutex mu_;
  std::condition_variable cv_, done_cv_;
  std::vector<std::unique_ptr<Job>> jobs_;
  std::deque<uint64_t> pending_;
  std::multiset<uint64_t> busy_;
  std::vector<uint8_t> enc_;
  std::vector<std::thread> th_;
  bool reorder_, stop_ = false;
  uint64_t seed_;
  std::atomic<int> violations_{0};
};

struct FakeBackend {
  FakeGpu *g;
  std::mutex emu;  // the client and its evictor both evict
  std::vector<uint64_t> evicts;
  uint64_t own = ~0ull;  // the client's latest own eviction
  int fault_submit(uint32_t, uint64_t pg, uint64_t *ticket) {
    *ticket = g->submit(MS_DECRYPT, &pg, 1);
    return MS_OK;
  }
  int fault_wait(uint64_t t) { return g->wait(t); }
  int evict(uint32_t, const uint64_t *pages, size_t k, bool background) {
    const uint64_t t = g->submit(MS_ENCRYPT, pages, k);
    std::lock_guard<std::mutex> lk(emu);
    evicts.push_back(t);
    if (!background) own = t;
    return MS_OK;
  }
  int wait_evicted() {
    uint64_t t;
    {
      std::lock_guard<std::mutex> lk(emu);
      if (own == ~0ull) return MS_OK;
      t = own;
    }
    return g->wait(t);
  }
  int drain() {
    for (uint64_t t : evicts) g->wait(t);
    return MS_OK;
  }
};

#define FAIL(...)             \
  do {                        \
    std::printf("FAIL ");     \
    std::printf(__VA_ARGS__); \
    std::printf("\n");        \
    return 1;                 \
  } while (0)

}  // namespace

int main(int argc, char **argv) {
  if (argc != 10 && argc != 11) return 2;
  const uint64_t seed = std::strtoull(argv[1], nullptr, 10);
  const int n_clients = std::atoi(argv[2]);
  const uint64_t per = std::strtoull(argv[3], nullptr, 10);
  const size_t trace_len = std::strtoull(argv[4], nullptr, 10);
  ms_window_config cfg{};
  cfg.window_pages = (uint32_t)std::atoi(argv[5]);
  cfg.evict_batch = (uint32_t)std::atoi(argv[6]);
  cfg.background_free = (uint32_t)std::atoi(argv[7]);
  const int executors = std::atoi(argv[8]);
  const bool reorder = std::atoi(argv[9]) != 0;
  cfg.sync_evict = argc == 11 ? (uint32_t)std::atoi(argv[10]) : 0;

  // traces: a small hot set with a sequential scan mixed in, so that pages
  // leave the window and come back while their evictions may still run
  std::vector<std::vector<uint64_t>> traces(n_clients);
  std::vector<ms_window_client> clients(n_clients);
  for (int c = 0; c < n_clients; ++c) {
    uint64_t r = mix(seed * 131 + (uint64_t)c), scan = 0;
    for (size_t i = 0; i < trace_len; ++i) {
      r = mix(r);
      traces[c].push_back(r % 3 ? r % (cfg.window_pages + 6) : (scan++ % per));
    }
    clients[c] = ms_window_client{(uint32_t)(100 + c), 0, c * per, per, traces[c].data(), trace_len};
  }
  FakeGpu gpu(per * n_clients, executors, reorder, seed);
  std::vector<ms::window::ClientRun> runs(n_clients);
  std::vector<std::thread> th;
  for (int c = 0; c < n_clients; ++c) {
    runs[c].cl = &clients[c];
    th.emplace_back([&, c] {
      FakeBackend be{&gpu, {}, {}, ~0ull};
      ms::window::run_client(be, cfg, runs[c]);
    });
  }
  for (auto &t : th) t.join();

  if (gpu.violations()) FAIL("%d requests found their page in the wrong state", gpu.violations());
  for (int c = 0; c < n_clients; ++c) {
    const ms::window::ClientRun &r = runs[c];
    const ms_window_stats &st = r.st;
    if (r.rc != MS_OK) FAIL("client %d returned %d", c, r.rc);
    if (st.accesses != trace_len || st.hits + st.faults != st.accesses) FAIL("client %d access counts", c);
    if (st.faults - st.evictions != r.final_window.size()) FAIL("client %d: faults - evictions != window", c);
    if (st.background_evictions > st.evictions || st.background_requests > st.evict_requests)
      FAIL("client %d background counters", c);
    const size_t cap = cfg.window_pages - cfg.background_free;
    if (r.final_window.size() > cap) FAIL("client %d final window %zu > %zu", c, r.final_window.size(), cap);
    if (cfg.background_free && st.background_evictions == 0) FAIL("client %d: the evictor never ran", c);
    if (!cfg.background_free && st.background_evictions) FAIL("client %d: background evictions while off", c);
    std::set<uint64_t> win(r.final_window.begin(), r.final_window.end());
    if (win.size() != r.final_window.size()) FAIL("client %d: a page twice in the window", c);
    for (uint64_t p = c * per; p < (c + 1) * per; ++p)
      if (gpu.encrypted(p) == (win.count(p) != 0)) FAIL("client %d page %llu in the wrong final state", c,
                                                          (unsigned long long)p);
  }
  std::printf("OK\n");
  return 0;
}
