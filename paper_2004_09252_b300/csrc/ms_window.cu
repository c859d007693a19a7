// Sliding-window client driver: produces the paper's fault / eviction stream
// (Sec. 4.3) from page-access traces and serves it through an ms_server
// (staged waves), through resident workers (one page per request, in place
// on the pinned working set, as the paper's GPU module does) or through
// ticketed launches on per-client clones of a context.
//
// Each client owns a range of working-set pages, all encrypted at the start,
// and a FIFO window of pages in clear.  An access to a page outside the
// window is a fault: the client submits a one-page decrypt and waits for it
// (the faulting thread is stalled until the page is resolved), then appends
// the page to its window.  When the window grows past its maximum, the
// oldest pages are evicted: one encrypt request for `evict_batch` of them,
// which the client does not wait for (a later fault on one of those pages
// waits for its encryption through the server's in-flight rule).  Clients
// run on their own threads with their own domain (the paper's PID).
//
// With background_free = T > 0 each client also runs an evictor thread that
// keeps T window slots free (the paper's conclusions propose encrypting window
// pages in the background).  The client and evictor logic is in
// ms_window_client.h; this file supplies the three backends.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_set>
#include <vector>

#include "ms_internal.h"
#include "ms_window_client.h"

namespace {

using clk = std::chrono::steady_clock;
using ms::window::ClientRun;
using ms::window::percentile;
using ms::window::run_client;

// Where a client's requests go.  fault_submit / fault_wait: decrypt one page
// and wait for it.  evict: encrypt pages without waiting.  drain: wait for
// every eviction.  fault_submit and evict are called under the client's
// window lock; fault_wait without it.
struct ServerBackend {
  ms_server *srv;
  uint32_t timeout_ms;
  std::mutex emu;  // evict_tickets: the client and its evictor both evict
  std::vector<uint64_t> evict_tickets;
  uint64_t last_own = ~0ull;  // the client's latest own eviction (written and read by the client)
  // MS_EBUSY (every ticket slot pending) is retried until timeout_ms.
  int submit(int op, uint32_t domain, const uint64_t *pages, size_t k, uint64_t *ticket) {
    const auto limit = clk::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
      const int rc = ms_server_submit_dom(srv, op, domain, pages, (uint32_t)k, ticket);
      if (rc != MS_EBUSY) return rc;
      if (clk::now() > limit) return MS_ETIMEDOUT;
      std::this_thread::yield();
    }
  }
  int fault_submit(uint32_t domain, uint64_t pg, uint64_t *ticket) {
    // an eviction of this page still in flight is waited for by the server's in-flight rule
    return submit(MS_DECRYPT, domain, &pg, 1, ticket);
  }
  int fault_wait(uint64_t ticket) { return ms_server_wait(srv, ticket, timeout_ms); }
  int evict(uint32_t domain, const uint64_t *pages, size_t k, bool background) {
    uint64_t ticket;
    const int rc = submit(MS_ENCRYPT, domain, pages, k, &ticket);
    if (rc == MS_OK) {
      std::lock_guard<std::mutex> lk(emu);
      evict_tickets.push_back(ticket);
      if (!background) last_own = ticket;
    }
    return rc;
  }
  int wait_evicted() { return last_own == ~0ull ? MS_OK : ms_server_wait(srv, last_own, timeout_ms); }
  int drain() {
    for (uint64_t t : evict_tickets) {
      const int rc = ms_server_wait(srv, t, timeout_ms);
      if (rc != MS_OK) return rc;
    }
    return MS_OK;
  }
};

struct ResidentBackend {
  ms_resident *res;
  uint64_t dbase;       // device address of the working set
  uint64_t first_page;  // the client's range, for last_ticket
  uint32_t timeout_ms;
  // per client page: its latest eviction, ~0 = none.  An element is written by
  // the thread that evicts the page and read by a later fault on it, which
  // the window's order puts after that eviction's submission.
  std::vector<uint64_t> last_ticket;
  std::mutex emu;  // evict_tickets: the client and its evictor both evict
  std::vector<uint64_t> evict_tickets;
  std::vector<uint64_t> own;  // the client's latest own eviction, one ticket per page (client only)
  int submit(uint32_t domain, uint64_t pg, uint64_t *ticket) {
    ms_page_dom e{};
    e.addr = dbase + pg * MS_PAGE_BYTES;
    e.page_id = pg;
    e.domain = domain;
    const auto limit = clk::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
      const int rc = ms_resident_submit(res, &e, ticket);
      if (rc != MS_EBUSY) return rc;
      if (clk::now() > limit) return MS_ETIMEDOUT;
      std::this_thread::yield();
    }
  }
  int fault_submit(uint32_t domain, uint64_t pg, uint64_t *ticket) {
    uint64_t &last = last_ticket[pg - first_page];
    if (last != ~0ull) {  // its eviction may still be running: a page is never in flight twice
      const int rc = ms_resident_wait(res, last, timeout_ms);
      if (rc != MS_OK) return rc;
      last = ~0ull;
    }
    return submit(domain, pg, ticket);
  }
  int fault_wait(uint64_t ticket) { return ms_resident_wait(res, ticket, timeout_ms); }
  int evict(uint32_t domain, const uint64_t *pages, size_t k, bool background) {
    if (!background) own.clear();
    for (size_t i = 0; i < k; ++i) {
      uint64_t ticket;
      const int rc = submit(domain, pages[i], &ticket);
      if (rc != MS_OK) return rc;
      last_ticket[pages[i] - first_page] = ticket;
      if (!background) own.push_back(ticket);
      std::lock_guard<std::mutex> lk(emu);
      evict_tickets.push_back(ticket);
    }
    return MS_OK;
  }
  int wait_evicted() {
    for (uint64_t t : own) {
      const int rc = ms_resident_wait(res, t, timeout_ms);
      if (rc != MS_OK) return rc;
    }
    return MS_OK;
  }
  int drain() {
    for (uint64_t t : evict_tickets) {
      const int rc = ms_resident_wait(res, t, timeout_ms);
      if (rc != MS_OK) return rc;
    }
    return MS_OK;
  }
};

// One launch per request on a context, each with its own ticket (in place on
// the pinned working set).  The client's context runs its requests in
// submission order, so a fault on a page whose eviction it queued earlier
// runs after it.  The background evictor submits on a second clone (its own
// lock and stream), so its launches neither hold up the client's calls nor
// queue ahead of its faults; a fault on a page whose background eviction is
// still pending waits for that eviction's ticket first.
struct TicketBackend {
  ms_ctx *ctx;      // the client's faults and its own evictions
  ms_ctx *bg_ctx;   // the evictor's evictions (nullptr without background eviction)
  uint64_t dbase;
  uint64_t first_page;
  uint32_t timeout_ms;
  // per client page: its latest background eviction on bg_ctx, ~0 = none.  An
  // element is written by the evictor and read by a later fault on the page,
  // which the window's order puts after that eviction's submission.
  std::vector<uint64_t> bg_ticket;
  std::mutex emu;                  // the two latest eviction tickets
  uint64_t last_evict = ~0ull, last_bg_evict = ~0ull;
  uint64_t last_own = ~0ull;       // the client's latest own eviction (on ctx)
  static int submit(ms_ctx *c, uint64_t dbase, uint32_t timeout_ms, const uint64_t *pages, size_t k,
                    uint64_t *ticket, int op) {
    std::vector<ms_page> ent(k);
    for (size_t i = 0; i < k; ++i) {
      ent[i].addr = dbase + pages[i] * MS_PAGE_BYTES;
      ent[i].page_id = pages[i];
    }
    const auto limit = clk::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
      const int rc = ms_submit_host(c, op, ent.data(), k, ticket);
      if (rc != MS_EBUSY) return rc;
      if (clk::now() > limit) return MS_ETIMEDOUT;
      std::this_thread::yield();
    }
  }
  int fault_submit(uint32_t, uint64_t pg, uint64_t *ticket) {
    if (bg_ctx) {
      uint64_t &t = bg_ticket[pg - first_page];
      if (t != ~0ull) {  // its background eviction may still be pending on the other stream
        const int rc = ms_wait(bg_ctx, t, timeout_ms);
        if (rc != MS_OK) return rc;
        t = ~0ull;
      }
    }
    return submit(ctx, dbase, timeout_ms, &pg, 1, ticket, MS_DECRYPT);
  }
  int fault_wait(uint64_t ticket) { return ms_wait(ctx, ticket, timeout_ms); }
  int evict(uint32_t, const uint64_t *pages, size_t k, bool background) {
    ms_ctx *c = background && bg_ctx ? bg_ctx : ctx;
    uint64_t t;
    const int rc = submit(c, dbase, timeout_ms, pages, k, &t, MS_ENCRYPT);
    if (rc != MS_OK) return rc;
    if (c == bg_ctx)
      for (size_t i = 0; i < k; ++i) bg_ticket[pages[i] - first_page] = t;
    std::lock_guard<std::mutex> lk(emu);  // tickets of one context grow with submission order
    uint64_t &last = c == bg_ctx ? last_bg_evict : last_evict;
    if (last == ~0ull || t > last) last = t;
    if (!background) last_own = t;
    return MS_OK;
  }
  int wait_evicted() { return last_own == ~0ull ? MS_OK : ms_wait(ctx, last_own, timeout_ms); }
  int drain() {
    int rc = last_evict == ~0ull ? MS_OK : ms_wait(ctx, last_evict, timeout_ms);
    if (rc == MS_OK && last_bg_evict != ~0ull) rc = ms_wait(bg_ctx, last_bg_evict, timeout_ms);
    return rc;
  }
};

int check_window_args(const ms_window_config *cfg, const ms_window_client *clients, size_t n_clients,
                      uint64_t n_pages) {
  if (!cfg || (n_clients && !clients)) return MS_EINVAL;
  if (cfg->window_pages == 0 || cfg->evict_batch == 0 || cfg->evict_batch > cfg->window_pages + 1) return MS_EINVAL;
  if (cfg->background_free >= cfg->window_pages) return MS_EINVAL;
  for (size_t c = 0; c < n_clients; ++c) {
    if (!clients[c].trace && clients[c].trace_len) return MS_EINVAL;
    if (clients[c].first_page > n_pages || clients[c].n_pages > n_pages - clients[c].first_page) return MS_EINVAL;
    for (size_t d = 0; d < c; ++d) {  // clients own disjoint page ranges
      const ms_window_client &a = clients[c], &b = clients[d];
      if (a.first_page < b.first_page + b.n_pages && b.first_page < a.first_page + a.n_pages) return MS_EINVAL;
    }
  }
  return MS_OK;
}

// One thread per client, each with its own backend; then the per-client report.
template <typename MakeBackend>
int run_clients(const ms_window_config &cfg, const ms_window_client *clients, size_t n_clients,
                ms_window_stats *stats_out, uint64_t *final_window_out, MakeBackend make) {
  std::vector<ClientRun> runs(n_clients);
  std::vector<std::thread> th;
  for (size_t c = 0; c < n_clients; ++c) {
    runs[c].cl = &clients[c];
    th.emplace_back([&, c] {
      auto be = make(clients[c]);
      run_client(be, cfg, runs[c]);
    });
  }
  for (auto &t : th) t.join();
  int rc = MS_OK;
  for (size_t c = 0; c < n_clients; ++c) {
    ClientRun &r = runs[c];
    if (r.rc != MS_OK && rc == MS_OK) rc = r.rc;
    r.st.fault_p50_us = percentile(r.lat_us, 0.50);
    r.st.fault_p99_us = percentile(r.lat_us, 0.99);
    r.st.fault_max_us = r.lat_us.empty() ? 0.0 : *std::max_element(r.lat_us.begin(), r.lat_us.end());
    r.st.final_window_pages = r.final_window.size();
    if (stats_out) stats_out[c] = r.st;
    if (final_window_out) {
      // client c's final window goes to final_window_out[c * (window_pages + 1) ...], oldest first
      uint64_t *dst = final_window_out + c * ((size_t)cfg.window_pages + 1);
      for (size_t i = 0; i < (size_t)cfg.window_pages + 1; ++i)
        dst[i] = i < r.final_window.size() ? r.final_window[i] : ~0ull;
    }
  }
  return rc;
}

}  // namespace

extern "C" int ms_window_run(ms_server *srv, const ms_window_config *cfg, const ms_window_client *clients,
                             size_t n_clients, ms_window_stats *stats_out, uint64_t *final_window_out,
                             uint32_t timeout_ms) {
  if (!srv) return MS_EINVAL;
  const int rc = check_window_args(cfg, clients, n_clients, ~0ull);
  if (rc != MS_OK) return rc;
  return run_clients(*cfg, clients, n_clients, stats_out, final_window_out, [&](const ms_window_client &) {
    return ServerBackend{srv, timeout_ms, {}, {}};
  });
}

extern "C" int ms_window_run_resident(ms_resident *res, void *host_base, uint64_t n_pages,
                                      const ms_window_config *cfg, const ms_window_client *clients,
                                      size_t n_clients, ms_window_stats *stats_out, uint64_t *final_window_out,
                                      uint32_t timeout_ms) {
  if (!res || !host_base || n_pages == 0) return MS_EINVAL;
  const int rc = check_window_args(cfg, clients, n_clients, n_pages);
  if (rc != MS_OK) return rc;
  void *dbase = nullptr;
  if (cudaHostGetDevicePointer(&dbase, host_base, 0) != cudaSuccess || !dbase) {
    cudaGetLastError();
    return MS_EINVAL;  // the working set must be pinned, mapped memory
  }
  return run_clients(*cfg, clients, n_clients, stats_out, final_window_out, [&](const ms_window_client &cl) {
    return ResidentBackend{res, (uint64_t)dbase, cl.first_page, timeout_ms,
                           std::vector<uint64_t>(cl.n_pages, ~0ull), {}, {}, {}};
  });
}

extern "C" int ms_window_run_ticketed(ms_ctx *ctx, void *host_base, uint64_t n_pages, const ms_window_config *cfg,
                                      const ms_window_client *clients, size_t n_clients, ms_window_stats *stats_out,
                                      uint64_t *final_window_out, uint32_t timeout_ms) {
  if (!ctx || !host_base || n_pages == 0) return MS_EINVAL;
  int rc = check_window_args(cfg, clients, n_clients, n_pages);
  if (rc != MS_OK) return rc;
  uint64_t dbase = 0;
  if (ms_host_device_address(host_base, &dbase) != MS_OK) return MS_EINVAL;
  // one clone per client: its PID as the domain, its own stream; with
  // background eviction a second one for the client's evictor
  const bool bg = cfg->background_free != 0;
  std::vector<ms_ctx *> clones(n_clients, nullptr), bg_clones(n_clients, nullptr);
  for (size_t c = 0; c < n_clients && rc == MS_OK; ++c) {
    rc = ms_clone(ctx, clients[c].domain, &clones[c]);
    if (rc == MS_OK && bg) rc = ms_clone(ctx, clients[c].domain, &bg_clones[c]);
  }
  if (rc == MS_OK) {
    rc = run_clients(*cfg, clients, n_clients, stats_out, final_window_out, [&](const ms_window_client &cl) {
      const size_t c = (size_t)(&cl - clients);
      return TicketBackend{clones[c], bg_clones[c], dbase, cl.first_page, timeout_ms,
                           std::vector<uint64_t>(bg ? cl.n_pages : 0, ~0ull), {}, ~0ull, ~0ull, ~0ull};
    });
  }
  for (auto *set : {&clones, &bg_clones})
    for (ms_ctx *k : *set)
      if (k) ms_shutdown(k);
  return rc;
}
