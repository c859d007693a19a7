// Resident workers: the paper's always-running GPU crypto module (Sec. 4.4)
// with every wait bounded.
//
// Each worker is a one-CTA kernel on its own stream that consumes its own
// ring of requests in pinned, mapped host memory (the paper's per-worker
// queue: many host threads produce, one GPU worker consumes).  A request is
// one page (the fault path).  The host writes the entry and then publishes
// its sequence number with a release store; the worker reads the sequence
// number with a system-scope acquire load, processes the page in place (in
// device memory, or in pinned host memory over the host link), makes its
// writes visible system-wide and publishes a done word per slot.
//
// Bounded waits: a worker leaves after `idle_exit_us` without work, after
// `max_run_ms` in total, or when the stop word is set.  Leaving is a
// handshake: the worker stores EXITING, fences, and looks at its next slot
// once more; the host publishes a request, fences, and reads the worker's
// state.  One of the two sees the other: either the worker stays
// (RUNNING) or the host sees EXITED and launches the worker again on the
// same stream, where the new launch starts after the old one has returned.
#include <sys/prctl.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "ms_internal.h"
#include "ms_link.cuh"

namespace {

enum : uint32_t { kRunning = 1, kExiting = 2, kExited = 3 };
constexpr int kWorkerThreads = 512;          // 8 pages in parallel at 64 threads per page
constexpr int kPagesPerPass = kWorkerThreads / 64;
static_assert(kPagesPerPass <= 32, "one lane of warp 0 per ring slot of a pass");

struct alignas(32) RingEntry {
  uint64_t addr;
  uint64_t page_id;
  uint32_t domain;
  uint32_t pad;
  uint64_t seq;  // local index + 1 once the entry is valid
};

struct WorkerShared {  // mapped host memory, one per worker
  uint32_t state;
  uint32_t stop;
  uint64_t next;       // first local index the next launch consumes
  uint64_t launches;   // kernel-side count of launches, for the stats
  uint32_t timeouts;   // launches that ended by max_run_ms
  uint32_t pad;
};

struct ResidentArgs {
  RingEntry *ring;       // device view of this worker's ring
  uint64_t *done;        // device view of this worker's done words
  WorkerShared *sh;      // device view of the worker's shared words
  uint32_t ring_mask;    // ring entries - 1
  uint64_t idle_ns, max_ns;
  const uint4 *key;
  ms::MulConsts mc;
};

__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint64_t ld_acquire_sys(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(uint64_t *p, uint64_t v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_sys32(uint32_t *p, uint32_t v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One pass: warp 0 looks at the next kPagesPerPass ring slots at once (lane k
// reads slot i + k: its sequence word with a system-scope acquire, then the
// entry), and the pass takes the leading run of published slots; every page
// of the pass is processed by 64 threads in parallel; then lanes 0..n-1
// publish the done words together.  Host-link round trips per pass: one for
// the sequence words, one for the entries, however many pages are taken.
__global__ void __launch_bounds__(kWorkerThreads) k_resident(const ResidentArgs a) {
  __shared__ RingEntry s_e[kPagesPerPass];
  __shared__ int s_n;
  __shared__ uint4 s_rows[kWorkerThreads / 32][128];  // each warp's 2 KiB row transpose
  const uint32_t tid = threadIdx.x;
  const uint32_t lane = tid % 32;
  uint64_t i = a.sh->next;  // written by the previous launch / the host before this launch
  const uint64_t t_start = gtime();
  uint64_t t_last = t_start;
  bool busy = false;  // warp 0: the last pass took a full kPagesPerPass
  ms::BlockSeed s;
  ms::load_key(a.key, s.k);
  for (;;) {
    if (tid < 32) {
      int n = 0;
      // lane 0's clock and stop word decide for the whole warp (the warp-wide
      // vote and shuffles below need every lane on the same path)
      uint64_t now = gtime();
      now = __shfl_sync(0xffffffffu, now, 0);
      int leave = lane == 0 && (ld_volatile_u32(&a.sh->stop) != 0 || now - t_start > a.max_ns);
      leave = __shfl_sync(0xffffffffu, leave, 0);
      if (leave) {
        // stop, or this launch has run long enough: leave even with work
        // queued; the host launches the worker again when it waits or submits
        if (lane == 0) {
          a.sh->next = i;
          if (now - t_start > a.max_ns) a.sh->timeouts += 1;
          __threadfence_system();
          st_release_sys32(&a.sh->state, kExited);
        }
        n = -1;
      } else {
        const RingEntry *e = a.ring + ((i + lane) & a.ring_mask);
        // While the ring was idle only slot i is watched (one 8-byte read per
        // poll over the host link); after a full pass, all slots are read at once.
        const uint32_t watch = busy ? (uint32_t)kPagesPerPass : 1u;
        bool ready = lane < watch && ld_acquire_sys(&e->seq) == i + lane + 1;
        if (!busy && __shfl_sync(0xffffffffu, (int)ready, 0))
          ready = lane == 0 || (lane < (uint32_t)kPagesPerPass && ld_acquire_sys(&e->seq) == i + lane + 1);
        const uint32_t mask = __ballot_sync(0xffffffffu, ready);
        n = __ffs(~mask) - 1;  // the leading run of published slots, in ring order
        busy = n == kPagesPerPass;
        if ((int)lane < n) s_e[lane] = *e;
        if (n > 0) {
          t_last = now;
        } else if (now - t_last > a.idle_ns) {
          int stay = 0;
          if (lane == 0) {
            st_release_sys32(&a.sh->state, kExiting);
            __threadfence_system();
            const RingEntry *e0 = a.ring + (i & a.ring_mask);
            if (ld_acquire_sys(&e0->seq) == i + 1) {
              st_release_sys32(&a.sh->state, kRunning);  // a request raced the exit: stay
              stay = 1;
            } else {
              a.sh->next = i;
              __threadfence_system();
              st_release_sys32(&a.sh->state, kExited);
            }
          }
          stay = __shfl_sync(0xffffffffu, stay, 0);
          if (stay) {
            t_last = now;
          } else {
            n = -1;
          }
        } else if (lane == 0) {
          __nanosleep(256);
        }
      }
      if (lane == 0) s_n = n;
    }
    __syncthreads();
    const int n = s_n;
    if (n < 0) return;
    if (n > 0) {
      // page `slot` of the pass; warp 2 slot + h takes its blocks 32 h .. 32 h + 31
      // as 512-byte rows over the host link (the branch is warp-uniform)
      const uint32_t slot = tid / 64, t = tid % 64;
      if (slot < (uint32_t)n) {
        const RingEntry e = s_e[slot];
        if (ms::entry_ok(e.addr)) {
          s.n0 = (uint32_t)e.page_id;
          s.n1 = (uint32_t)(e.page_id >> 32);
          s.n2 = e.domain;
          uint4 *span = ms::span_of(e.addr, t);
          uint4 row[4], blk[4];
          ms::load_span(row, span, lane);
          ms::rows_to_block(s_rows[tid / 32], row, blk, lane);
          ms::xor_keystream<20>(blk, s, t, a.mc);
          ms::store_block(s_rows[tid / 32], blk, span, lane);
        }
      }
      __threadfence_system();  // this thread's page writes are visible before the done word
      __syncthreads();
      if (tid < (uint32_t)n) st_release_sys(a.done + ((i + tid) & a.ring_mask), i + tid + 1);
      i += n;
    }
    __syncthreads();
  }
}

// Short naps must stay short: the first nap on a thread drops its timer
// slack (default 50 us) to 1 us.
inline void nap_ns(long ns) {
  thread_local bool slack_set = false;
  if (!slack_set) {
    prctl(PR_SET_TIMERSLACK, 1000UL, 0, 0, 0);
    slack_set = true;
  }
  struct timespec ts = {ns / 1000000000L, ns % 1000000000L};
  nanosleep(&ts, nullptr);
}

inline uint64_t load_acq(const uint64_t *p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }
inline uint32_t load_acq32(const uint32_t *p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }

// The fields the submitting thread writes on every request (tail, the
// hint, the lock) sit on a cache line of their own, apart from the pointers
// that completion checks read, so that a completing thread does not pull
// the submitter's line away on every check.
struct Worker {
  RingEntry *h_ring = nullptr, *d_ring = nullptr;
  uint64_t *h_done = nullptr, *d_done = nullptr;
  WorkerShared *h_sh = nullptr, *d_sh = nullptr;
  cudaStream_t stream = nullptr;
  alignas(64) uint64_t tail = 0;  // next local index to fill
  uint64_t done_hint = 0;  // every local index below this is known finished (under mu)
  std::mutex mu;
  uint64_t host_launches = 0;
};

}  // namespace

struct ms_resident {
  ms_ctx *ctx = nullptr;
  ms_resident_config cfg{};
  std::vector<Worker *> w;
  std::atomic<uint64_t> rr{0};
  std::atomic<uint64_t> replay_max_lag_ns{0};
};

using namespace ms;

namespace {

void free_resident(ms_resident *r) {
  for (Worker *w : r->w) {
    if (!w) continue;
    if (w->stream) cudaStreamDestroy(w->stream);
    if (w->h_ring) cudaFreeHost(w->h_ring);
    if (w->h_done) cudaFreeHost(w->h_done);
    if (w->h_sh) cudaFreeHost(w->h_sh);
    delete w;
  }
  delete r;
}

// Make sure worker `wi` is running; called with its mutex held, after the
// request was published.
int ensure_running(ms_resident *r, int wi) {
  Worker &w = *r->w[wi];
  __atomic_thread_fence(__ATOMIC_SEQ_CST);
  uint32_t st = load_acq32(&w.h_sh->state);
  if (st == kRunning) return MS_OK;  // the common case: no clock read
  const auto limit = std::chrono::steady_clock::now() + std::chrono::milliseconds(r->ctx->cfg.timeout_ms);
  while (st == kExiting) {  // the worker is deciding; it resolves within a few microseconds
    if (std::chrono::steady_clock::now() > limit) return MS_ETIMEDOUT;
    nap_ns(1000);
    st = load_acq32(&w.h_sh->state);
  }
  if (st == kRunning) return MS_OK;
  // EXITED (or never started): launch again; stream order puts it after the old launch
  DeviceGuard g(r->ctx->device);  // only a launch needs the device current
  ResidentArgs a{};
  a.ring = w.d_ring;
  a.done = w.d_done;
  a.sh = w.d_sh;
  a.ring_mask = r->cfg.ring_entries - 1;
  a.idle_ns = (uint64_t)r->cfg.idle_exit_us * 1000ull;
  a.max_ns = (uint64_t)r->cfg.max_run_ms * 1000000ull;
  a.key = r->ctx->d_key;
  a.mc.m12 = 1u << 12;
  a.mc.m7 = 1u << 7;
  __atomic_store_n(&w.h_sh->state, (uint32_t)kRunning, __ATOMIC_RELEASE);
  k_resident<<<1, kWorkerThreads, 0, w.stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    __atomic_store_n(&w.h_sh->state, (uint32_t)kExited, __ATOMIC_RELEASE);
    return cuda_fail(r->ctx, e);
  }
  w.host_launches += 1;
  return MS_OK;
}

}  // namespace

extern "C" {

void ms_resident_config_default(ms_resident_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->workers = 4;
  cfg->ring_entries = 4096;
  cfg->idle_exit_us = 200000;
  cfg->max_run_ms = 10000;
}

int ms_resident_create(ms_ctx *c, const ms_resident_config *cfg_in, ms_resident **out) {
  if (!out) return MS_EINVAL;
  *out = nullptr;
  if (!c || !c->alive) return MS_ENOTINIT;
  if (c->cfg.rounds != 20) return MS_EINVAL;  // the resident worker is compiled for ChaCha20 only
  ms_resident_config cfg;
  if (cfg_in) cfg = *cfg_in; else ms_resident_config_default(&cfg);
  if (cfg.workers == 0 || cfg.workers > 64) return MS_EINVAL;
  if (cfg.ring_entries < 4 || (cfg.ring_entries & (cfg.ring_entries - 1)) || cfg.ring_entries > (1u << 20))
    return MS_EINVAL;
  if (cfg.idle_exit_us == 0 || cfg.max_run_ms == 0 || cfg.max_run_ms > 600000) return MS_EINVAL;
  ms_resident *r = new (std::nothrow) ms_resident();
  if (!r) return MS_ENOMEM;
  r->ctx = c;
  r->cfg = cfg;
  DeviceGuard g(c->device);
  for (uint32_t i = 0; i < cfg.workers; ++i) {
    Worker *w = new (std::nothrow) Worker();
    if (!w) {
      free_resident(r);
      return MS_ENOMEM;
    }
    r->w.push_back(w);
    cudaError_t e = cudaHostAlloc(&w->h_ring, sizeof(RingEntry) * cfg.ring_entries, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostAlloc(&w->h_done, sizeof(uint64_t) * cfg.ring_entries, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostAlloc(&w->h_sh, sizeof(WorkerShared), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&w->d_ring, w->h_ring, 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&w->d_done, w->h_done, 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&w->d_sh, w->h_sh, 0);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      free_resident(r);
      return alloc_fail(c, e);
    }
    std::memset(w->h_ring, 0, sizeof(RingEntry) * cfg.ring_entries);
    std::memset(w->h_done, 0, sizeof(uint64_t) * cfg.ring_entries);
    std::memset(w->h_sh, 0, sizeof(WorkerShared));
    w->h_sh->state = kExited;
  }
  c->children.fetch_add(1);
  *out = r;
  return MS_OK;
}

namespace {

// Queue one page on worker wi (MS_EBUSY when its ring slot is still taken).
int submit_to(ms_resident *r, int wi, const ms_page_dom *page, uint64_t *ticket) {
  const uint32_t W = r->cfg.workers;
  Worker &w = *r->w[wi];
  std::lock_guard<std::mutex> lk(w.mu);
  const uint64_t li = w.tail;
  const uint32_t R = r->cfg.ring_entries;
  const uint32_t slot = (uint32_t)(li & (R - 1));
  if (li >= R && w.done_hint < li - R + 1) {
    // The slot's previous request (li - R) must have finished.  A worker
    // finishes in order, so one done word proves every earlier index done:
    // look halfway back first, which keeps these reads of GPU-written words
    // to about two per R / 2 submissions.
    const uint64_t probe = li - R / 2;
    if (load_acq(&w.h_done[probe & (R - 1)]) >= probe + 1) {
      w.done_hint = probe + 1;
    } else if (load_acq(&w.h_done[slot]) >= li - R + 1) {
      w.done_hint = li - R + 1;
    } else {
      return MS_EBUSY;  // the slot's previous request is still being served
    }
  }
  RingEntry &e = w.h_ring[slot];
  e.addr = page->addr;
  e.page_id = page->page_id;
  e.domain = page->domain;
  __atomic_store_n(&e.seq, li + 1, __ATOMIC_RELEASE);
  __atomic_store_n(&w.tail, li + 1, __ATOMIC_RELAXED);  // read without the lock by ms_resident_poll
  const int rc = ensure_running(r, wi);
  if (rc != MS_OK) return rc;
  *ticket = li * W + (uint64_t)wi;
  return MS_OK;
}

bool page_ok(const ms_page_dom *page) { return page->addr != 0 && (page->addr & 15u) == 0; }

}  // namespace

int ms_resident_submit(ms_resident *r, const ms_page_dom *page, uint64_t *ticket) {
  if (!r || !page || !ticket) return MS_EINVAL;
  if (!page_ok(page)) return MS_EINVAL;
  return submit_to(r, (int)(r->rr.fetch_add(1) % r->cfg.workers), page, ticket);
}

int ms_resident_poll(ms_resident *r, uint64_t ticket) {
  if (!r) return MS_EINVAL;
  const uint32_t W = r->cfg.workers;
  Worker &w = *r->w[ticket % W];
  const uint64_t li = ticket / W;
  if (li >= __atomic_load_n(&w.tail, __ATOMIC_RELAXED)) return MS_EINVAL;
  const uint64_t d = load_acq(&w.h_done[li & (r->cfg.ring_entries - 1)]);
  return d >= li + 1 ? 1 : 0;  // a later occupant of the slot means this one finished
}

int ms_resident_wait(ms_resident *r, uint64_t ticket, uint32_t timeout_ms) {
  if (!r) return MS_EINVAL;
  const auto limit = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  const int wi = (int)(ticket % r->cfg.workers);
  Worker &w = *r->w[wi];
  for (int it = 0;; ++it) {
    const int p = ms_resident_poll(r, ticket);
    if (p != 0) return p == 1 ? MS_OK : p;
    if (std::chrono::steady_clock::now() > limit) return MS_ETIMEDOUT;
    // a worker that left with this request queued (max_run_ms) is launched again
    if ((it & 63) == 63 && load_acq32(&w.h_sh->state) == kExited) {
      std::lock_guard<std::mutex> lk(w.mu);
      const int rc = ensure_running(r, wi);
      if (rc != MS_OK) return rc;
    }
    nap_ns(500);
  }
}

int ms_resident_get_stats(const ms_resident *r, ms_resident_stats *out) {
  if (!r || !out) return MS_EINVAL;
  std::memset(out, 0, sizeof(*out));
  for (Worker *w : r->w) {
    out->requests += __atomic_load_n(&w->tail, __ATOMIC_RELAXED);
    out->launches += w->host_launches;
    out->max_run_exits += __atomic_load_n(&w->h_sh->timeouts, __ATOMIC_RELAXED);
    if (__atomic_load_n(&w->h_sh->state, __ATOMIC_ACQUIRE) == kRunning) out->workers_running += 1;
  }
  out->replay_max_lag_ns = r->replay_max_lag_ns.load();
  return MS_OK;
}

int ms_resident_destroy(ms_resident *r) {
  if (!r) return MS_OK;
  DeviceGuard g(r->ctx->device);
  for (Worker *w : r->w) __atomic_store_n(&w->h_sh->stop, 1u, __ATOMIC_RELEASE);
  // Every worker must be known to have left before its rings are freed; if
  // that cannot be established, the memory stays allocated.
  for (Worker *w : r->w) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(r->ctx, e);
    e = cudaEventRecord(ev, w->stream);
    const int r2 = e == cudaSuccess ? wait_event(r->ctx, ev, r->ctx->cfg.timeout_ms) : cuda_fail(r->ctx, e);
    cudaEventDestroy(ev);
    if (r2 != MS_OK) return r2;
  }
  ms_ctx *c = r->ctx;
  free_resident(r);
  c->children.fetch_sub(1);
  return MS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- replay
// Open-loop replay over a host working set: request r (pages
// page_index[offsets[r] .. offsets[r + 1]) of host_base, domain domains[r])
// is submitted at arrival_s[r], one resident request per page; it completes
// when all its pages are done.  A page still in flight from an earlier
// request is waited for first.  Latency counts from the scheduled arrival.
extern "C" int ms_resident_replay(ms_resident *r, void *host_base, uint64_t n_pages, size_t n, const double *arrival_s,
                                  const uint32_t *domains, const uint64_t *offsets, const uint64_t *page_index,
                                  double *latency_s, double *makespan_s, uint32_t timeout_ms) {
  using clk = std::chrono::steady_clock;
  if (!r || !host_base || (n && (!arrival_s || !offsets || !page_index || !latency_s))) return MS_EINVAL;
  void *dbase = nullptr;
  {
    DeviceGuard g(r->ctx->device);
    if (cudaHostGetDevicePointer(&dbase, host_base, 0) != cudaSuccess || !dbase) {
      cudaGetLastError();
      return MS_EINVAL;  // the working set must be pinned, mapped memory
    }
  }
  for (size_t q = 0; q < n; ++q) {
    if (offsets[q + 1] <= offsets[q]) return MS_EINVAL;  // every request has at least one page
    for (uint64_t k = offsets[q]; k < offsets[q + 1]; ++k)
      if (page_index[k] >= n_pages) return MS_EINVAL;
    latency_s[q] = -1.0;
  }
  if (n > UINT32_MAX) return MS_ERANGE;
  const uint32_t W = r->cfg.workers;
  const uint32_t R = r->cfg.ring_entries;
  const uint64_t total = offsets[n];
  // Completion is followed per worker, in ring order (a worker serves its
  // requests in order): each pass advances every worker's frontier over the
  // pages it has finished, which is O(completions), and a request is stamped
  // when its last page finishes.  wmap[w][i] is the request of the i-th page
  // this replay gave worker w; it is written before that page is published.
  std::vector<uint64_t> tickets(total);
  std::vector<uint64_t> sched(n);
  std::vector<uint32_t> remaining(n);
  for (size_t q = 0; q < n; ++q) remaining[q] = (uint32_t)(offsets[q + 1] - offsets[q]);
  std::vector<uint64_t> last_ticket(n_pages, ~0ull);
  std::vector<std::vector<uint32_t>> wmap(W, std::vector<uint32_t>(total / W + 2));
  std::vector<uint64_t> base_li(W);
  for (uint32_t w = 0; w < W; ++w) {
    std::lock_guard<std::mutex> lk(r->w[w]->mu);
    base_li[w] = r->w[w]->tail;
  }
  std::unique_ptr<std::atomic<uint64_t>[]> published(new std::atomic<uint64_t>[W]);
  for (uint32_t w = 0; w < W; ++w) published[w].store(0);
  std::atomic<int> err{0};
  auto now_ns = [] {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(clk::now().time_since_epoch()).count();
  };
  // Start every worker before the clock does, so that no launch (or module
  // load) falls on the first requests.
  for (uint32_t w = 0; w < W; ++w) {
    std::lock_guard<std::mutex> lk(r->w[w]->mu);
    const int rc0 = ensure_running(r, (int)w);
    if (rc0 != MS_OK) return rc0;
  }
  const uint64_t t0 = now_ns() + 1000000ull;
  std::thread comp([&] {
    std::vector<uint64_t> frontier(W, 0);
    size_t completed = 0;
    const uint64_t deadline_pad = (uint64_t)timeout_ms * 1000000ull;
    uint64_t last_progress = now_ns();
    while (completed < n && !err.load()) {
      bool progress = false;
      for (uint32_t w = 0; w < W; ++w) {
        const uint64_t hi = published[w].load(std::memory_order_acquire);
        while (frontier[w] < hi) {
          // the page's done word alone (ms_resident_poll would also read the
          // worker's tail, the submitting thread's hot line); a later occupant
          // of the slot means this one finished
          const uint64_t li = base_li[w] + frontier[w];
          if (load_acq(&r->w[w]->h_done[li & (R - 1)]) < li + 1) break;
          const uint32_t q = wmap[w][frontier[w]];
          if (--remaining[q] == 0) {
            latency_s[q] = (double)(int64_t)(now_ns() - sched[q]) * 1e-9;
            ++completed;
          }
          ++frontier[w];
          progress = true;
        }
      }
      const uint64_t t = now_ns();
      if (progress) {
        // pause briefly even after progress: a completer that re-reads the
        // published counts without pause pulls their cache line away from
        // the submitting thread on every page it publishes
        last_progress = t;
        nap_ns(1000);
        continue;
      }
      if (t - last_progress > deadline_pad) {
        // nothing finished for timeout_ms: let ms_resident_wait relaunch a worker that left
        for (uint32_t w = 0; w < W; ++w)
          if (frontier[w] < published[w].load(std::memory_order_acquire) &&
              ms_resident_wait(r, (base_li[w] + frontier[w]) * W + w, timeout_ms) != MS_OK) {
            err.store(MS_ETIMEDOUT);
            return;
          }
        last_progress = now_ns();
      }
      nap_ns(2000);
    }
  });
  int rc = MS_OK;
  uint64_t max_lag = 0;
  for (size_t q = 0; q < n && rc == MS_OK; ++q) {
    const uint64_t target = t0 + (uint64_t)(arrival_s[q] * 1e9);
    for (;;) {
      const uint64_t t = now_ns();
      if (t >= target) break;
      // sleep only through long gaps and wake 1 ms early, spin otherwise: an
      // idle virtual CPU can wake milliseconds late, and a late submission
      // counts as latency (arrivals are scheduled)
      if (target - t > 2000000) nap_ns((long)(target - t - 1000000));
    }
    sched[q] = target;
    if (q + 1 < n)  // the next request's entries of the page-sized ticket table: hide their cache misses
      for (uint64_t k = offsets[q + 1]; k < offsets[q + 2] && k < offsets[q + 1] + 16; ++k)
        __builtin_prefetch(&last_ticket[page_index[k]]);
    for (uint64_t k = offsets[q]; k < offsets[q + 1] && rc == MS_OK; ++k) {
      const uint64_t pg = page_index[k];
      const uint64_t prev = last_ticket[pg];
      // The page's previous request must be finished.  This thread is the
      // only submitter during a replay, so it may read the done hint that its
      // own submissions keep (no read of a GPU-written word); only a request
      // that the hint does not cover is waited for.
      if (prev != ~0ull && prev / W >= r->w[prev % W]->done_hint) {
        rc = ms_resident_wait(r, prev, timeout_ms);  // the page may still be in flight
        if (rc != MS_OK) break;
      }
      ms_page_dom e{};
      e.addr = (uint64_t)dbase + pg * MS_PAGE_BYTES;
      e.page_id = pg;
      e.domain = domains ? domains[q] : r->ctx->cfg.domain;
      // Pages go to the workers in strict rotation, and a page whose worker
      // has a full ring waits for that worker: passing it to the next one
      // would give some worker more than its share of the replay's pages.
      if (!page_ok(&e)) {
        rc = MS_EINVAL;
        break;
      }
      const int wi = (int)(r->rr.fetch_add(1) % W);
      uint64_t spin_end = 0;  // set on the first MS_EBUSY: a full ring is rare
      for (;;) {
        rc = submit_to(r, wi, &e, &tickets[k]);
        if (rc != MS_EBUSY) break;
        if (!spin_end) spin_end = now_ns() + (uint64_t)timeout_ms * 1000000ull;
        if (now_ns() > spin_end) {
          rc = MS_ETIMEDOUT;
          break;
        }
        nap_ns(2000);
      }
      if (rc == MS_OK) {
        last_ticket[pg] = tickets[k];
        const uint32_t w = (uint32_t)(tickets[k] % W);
        const uint64_t idx = tickets[k] / W - base_li[w];
        if (idx >= wmap[w].size() || idx != published[w].load(std::memory_order_relaxed)) {
          rc = MS_EBUSY;  // another thread submitted to these workers during the replay
          break;
        }
        wmap[w][idx] = (uint32_t)q;
        published[w].store(idx + 1, std::memory_order_release);
      }
    }
    if (rc == MS_OK) max_lag = std::max(max_lag, now_ns() - target);
  }
  r->replay_max_lag_ns.store(max_lag);
  if (rc != MS_OK) err.store(rc);
  comp.join();
  if (rc != MS_OK) return rc;
  if (err.load()) return err.load();
  uint64_t last = t0;
  for (size_t q = 0; q < n; ++q) last = std::max(last, sched[q] + (uint64_t)std::max(0.0, latency_s[q] * 1e9));
  if (makespan_s) *makespan_s = (double)(last - t0) * 1e-9;
  return MS_OK;
}
