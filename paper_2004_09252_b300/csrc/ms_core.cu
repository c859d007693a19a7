// Context lifecycle, key placement, the one-launch entry points, ms_sync and
// the streamed host-page form.
#include <errno.h>
#include <sys/random.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>
#include <unordered_set>

#include "ms_internal.h"

namespace ms {

int cuda_fail(ms_ctx *c, cudaError_t e) {
  if (c) c->last_cuda.store((int)e);
  cudaGetLastError();  // a non-sticky error must not be reported again by the next launch check
  return MS_ECUDA;
}

int alloc_fail(ms_ctx *c, cudaError_t e) {
  if (e != cudaErrorMemoryAllocation) return cuda_fail(c, e);
  cudaGetLastError();  // out of memory is not sticky: clear it for the next launch check
  return MS_ENOMEM;
}

// Moves the device status word to the mapped host word and clears it: one
// launch where a copy and a memset would be two operations on the stream.
__global__ void k_status_take(unsigned int *d_status, unsigned int *h_status) {
  const unsigned int v = *d_status;
  *d_status = 0;
  *(volatile unsigned int *)h_status = v;
}

namespace {
std::atomic<int> g_fault_mask{0};
std::atomic<int> g_fault_countdown{0};
std::atomic<int> g_fault_error{0};
}  // namespace

cudaError_t injected(int site) {
  if (!(g_fault_mask.load(std::memory_order_relaxed) & site)) return cudaSuccess;
  if (g_fault_countdown.fetch_sub(1) != 0) return cudaSuccess;
  g_fault_mask.store(0);  // one shot
  return (cudaError_t)g_fault_error.load();
}

// Bounded wait on an event: poll, spinning for the first 50 us and then
// sleeping 20 us between polls, until it completes or `timeout_ms` passes.
int wait_event(ms_ctx *c, cudaEvent_t ev, uint32_t timeout_ms) {
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  const auto limit = std::chrono::milliseconds(timeout_ms);
  for (;;) {
    cudaError_t r = cudaEventQuery(ev);
    if (r == cudaSuccess) return MS_OK;
    if (r != cudaErrorNotReady) return cuda_fail(c, r);
    const auto el = clk::now() - t0;
    if (el > limit) return MS_ETIMEDOUT;
    if (el > std::chrono::microseconds(50)) {
      struct timespec ts = {0, 20000};
      nanosleep(&ts, nullptr);
    }
  }
}

PageArgs make_args(const ms_ctx *c) {
  PageArgs a{};
  a.key = c->d_key;
  a.domain = c->cfg.domain;
  a.status = c->d_status;
  a.mc.m12 = 1u << 12;
  a.mc.m7 = 1u << 7;
  return a;
}

// Entry lists of either layout: ms_page (context domain) or ms_page_dom.
template <typename E>
void set_list(PageArgs &a, const E *p);
template <>
void set_list<ms_page>(PageArgs &a, const ms_page *p) { a.pages = p; }
template <>
void set_list<ms_page_dom>(PageArgs &a, const ms_page_dom *p) { a.dpages = p; }

// Host-side entry checks of a host list (addresses; duplicates if configured).
template <typename E>
int check_list_host(const ms_ctx *c, const E *pages, size_t n) {
  if (!pages) return MS_EINVAL;
  for (size_t i = 0; i < n; ++i)
    if (pages[i].addr == 0 || (pages[i].addr & 15u)) return MS_EINVAL;
  if (c->cfg.check_duplicates) {
    std::unordered_set<uint64_t> seen;
    seen.reserve(n * 2);
    for (size_t i = 0; i < n; ++i)
      if (!seen.insert(pages[i].addr).second) return MS_EINVAL;
  }
  return MS_OK;
}

// Queue a checked host list on the context stream; the caller holds c->mu.
template <typename E>
int submit_list_host_locked(ms_ctx *c, const E *pages, size_t n);

template <typename E>
int submit_list_host(ms_ctx *c, const E *pages, size_t n) {
  if (!c || !c->alive) return MS_ENOTINIT;
  if (n == 0) return MS_OK;
  const int rc = check_list_host(c, pages, n);
  if (rc != MS_OK) return rc;
  std::lock_guard<std::mutex> lk(c->mu);
  return submit_list_host_locked(c, pages, n);
}

template <typename E>
int submit_list_host_locked(ms_ctx *c, const E *pages, size_t n) {
  DeviceGuard g(c->device);
  // A short list goes in the kernel parameters: one launch, no copies.  A
  // shape the caller chose is kept, so such contexts take the staged path.
  if (n <= inline_max_pages<E>() && !c->shape_explicit) {
    const cudaError_t e = launch_pages_inline(c, pages, n, c->stream);
    return e == cudaSuccess ? MS_OK : cuda_fail(c, e);
  }
  const size_t cap = c->cfg.list_capacity;  // slots hold cap entries of the larger layout
  for (size_t off = 0; off < n; off += cap) {
    const size_t cnt = std::min(cap, n - off);
    ListSlot &s = c->slots[c->next_slot];
    c->next_slot = (c->next_slot + 1) % kListSlots;
    if (s.used) {
      int rc = wait_event(c, s.done, c->cfg.timeout_ms);
      if (rc != MS_OK) return rc;
    }
    std::memcpy(s.h, pages + off, cnt * sizeof(E));
    cudaError_t e = injected(MS_FAULT_COPY);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.d, s.h, cnt * sizeof(E), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    PageArgs a = make_args(c);
    set_list<E>(a, static_cast<const E *>(s.d));
    a.n_pages = cnt;
    e = launch_pages(c, a, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    e = cudaEventRecord(s.done, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    s.used = true;
  }
  return MS_OK;
}

template <typename E>
int submit_list_dev(ms_ctx *c, const E *d_pages, size_t n) {
  if (!c || !c->alive) return MS_ENOTINIT;
  if (n == 0) return MS_OK;
  if (!d_pages || ((uintptr_t)d_pages & 15u)) return MS_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  PageArgs a = make_args(c);
  set_list<E>(a, d_pages);
  a.n_pages = n;
  c->status_dirty = true;  // set even if the launch fails: a read costs only time
  cudaError_t e = launch_pages(c, a, c->stream);
  return e == cudaSuccess ? MS_OK : cuda_fail(c, e);
}

}  // namespace ms

using namespace ms;

extern "C" {

void ms_config_default(ms_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->device = -1;
  cfg->stream = nullptr;
  cfg->domain = 0;
  cfg->rounds = 20;
  cfg->list_capacity = 65536;
  cfg->timeout_ms = 10000;
}

const char *ms_strerror(int code) {
  switch (code) {
    case MS_OK: return "success";
    case MS_EINVAL: return "invalid argument";
    case MS_ENOTINIT: return "context not initialised";
    case MS_ENOMEM: return "out of memory";
    case MS_ECUDA: return "CUDA runtime error";
    case MS_ETIMEDOUT: return "bounded wait timed out";
    case MS_EBUSY: return "busy: admission refused";
    case MS_ERANGE: return "size beyond the stated maximum";
    case MS_ESTARVED: return "a fed kernel waited for entries that never came";
    default: return "unknown error";
  }
}

int ms_last_cuda_error(const ms_ctx *ctx) { return ctx ? ctx->last_cuda.load() : 0; }

int ms_debug_inject_fault(int site_mask, int countdown, int cuda_error) {
  if (site_mask & ~(MS_FAULT_LAUNCH | MS_FAULT_COPY | MS_FAULT_GRAPH | MS_FAULT_SERVER)) return MS_EINVAL;
  if (countdown < 0 || (site_mask && cuda_error == 0)) return MS_EINVAL;
  g_fault_mask.store(0);
  g_fault_error.store(cuda_error);
  g_fault_countdown.store(countdown);
  g_fault_mask.store(site_mask);
  return MS_OK;
}

static void release(ms_ctx *c) {
  for (auto &s : c->slots) {
    if (s.done) cudaEventDestroy(s.done);
    if (s.h) cudaFreeHost(s.h);
    if (s.d) cudaFree(s.d);
  }
  for (int i = 0; i < kMaxHostStreams; ++i) {
    if (c->hs_ev[i]) cudaEventDestroy(c->hs_ev[i]);
    if (c->hs[i]) cudaStreamDestroy(c->hs[i]);
    if (c->hs_buf[i]) cudaFree(c->hs_buf[i]);
  }
  for (cudaEvent_t &ev : c->tk_ev)
    if (ev) cudaEventDestroy(ev);
  if (c->sync_ev) cudaEventDestroy(c->sync_ev);
  if (c->status_ev) cudaEventDestroy(c->status_ev);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->d_status) cudaFree(c->d_status);
  if (c->d_key) cudaFree(c->d_key);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

namespace {

// Context creation; the key comes from host memory (key, NULL = the OS
// CSPRNG) or, for a clone, from another context's device copy (key_dev).
int init_ctx(ms_ctx **out, const uint8_t *key, const uint4 *key_dev, const ms_config *cfg_in) {
  if (!out) return MS_EINVAL;
  *out = nullptr;
  ms_config cfg;
  if (cfg_in) cfg = *cfg_in; else ms_config_default(&cfg);
  if (cfg.rounds == 0) cfg.rounds = 20;
  if (cfg.rounds != 20 && cfg.rounds != 12 && cfg.rounds != 8) return MS_EINVAL;
  if (cfg.list_capacity == 0) cfg.list_capacity = 65536;
  if (cfg.timeout_ms == 0) cfg.timeout_ms = 10000;

  int dev = cfg.device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return MS_ECUDA;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || dev >= ndev) return MS_ECUDA;

  ms_ctx *c = new (std::nothrow) ms_ctx();
  if (!c) return MS_ENOMEM;
  c->device = dev;
  c->cfg = cfg;
  c->cfg.device = dev;
  DeviceGuard g(dev);
  cudaError_t e;
#define MS_TRY(call)                 \
  do {                               \
    e = (call);                      \
    if (e != cudaSuccess) {          \
      int rc = (e == cudaErrorMemoryAllocation) ? MS_ENOMEM : MS_ECUDA; \
      cudaGetLastError();            \
      release(c);                    \
      return rc;                     \
    }                                \
  } while (0)

  MS_TRY(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev));
  if (cfg.stream || cfg.use_stream) {
    c->stream = (cudaStream_t)cfg.stream;
  } else {
    MS_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    c->own_stream = true;
  }
  MS_TRY(cudaEventCreateWithFlags(&c->sync_ev, cudaEventDisableTiming));
  MS_TRY(cudaEventCreateWithFlags(&c->status_ev, cudaEventDisableTiming));
  MS_TRY(cudaMalloc(&c->d_status, sizeof(unsigned int)));
  MS_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned int), c->stream));
  MS_TRY(cudaHostAlloc(&c->h_status, sizeof(unsigned int), cudaHostAllocMapped));
  MS_TRY(cudaHostGetDevicePointer((void **)&c->h_status_dev, c->h_status, 0));
  for (auto &s : c->slots) {
    MS_TRY(cudaHostAlloc(&s.h, sizeof(ms_page_dom) * cfg.list_capacity, cudaHostAllocDefault));
    MS_TRY(cudaMalloc(&s.d, sizeof(ms_page_dom) * cfg.list_capacity));
    MS_TRY(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
  }

  // Key placement (Sec. 4.4: the key is drawn from the OS CSPRNG, handed to
  // the GPU and purged from host memory).  The pinned bounce buffer is the
  // only host copy the library makes; it is wiped before ms_init returns.
  MS_TRY(cudaMalloc(&c->d_key, MS_KEY_BYTES));
  if (key_dev) {  // a clone: device to device, the key never passes through host memory
    MS_TRY(cudaMemcpyAsync(c->d_key, key_dev, MS_KEY_BYTES, cudaMemcpyDeviceToDevice, c->stream));
    MS_TRY(cudaEventRecord(c->sync_ev, c->stream));
    const int krc = wait_event(c, c->sync_ev, std::max<uint32_t>(cfg.timeout_ms, 1000));
    if (krc != MS_OK) {
      release(c);
      return krc;
    }
  }
  uint8_t *bounce = nullptr;
  if (!key_dev) MS_TRY(cudaHostAlloc(&bounce, MS_KEY_BYTES, cudaHostAllocDefault));
  if (key_dev) {
    // nothing to place
  } else if (key) {
    std::memcpy(bounce, key, MS_KEY_BYTES);
  } else {
    size_t got = 0;
    while (got < MS_KEY_BYTES) {
      ssize_t r = getrandom(bounce + got, MS_KEY_BYTES - got, 0);
      if (r < 0 && errno == EINTR) continue;
      if (r < 0) {
        explicit_bzero(bounce, MS_KEY_BYTES);
        cudaFreeHost(bounce);
        release(c);
        return MS_EINVAL;
      }
      got += (size_t)r;
    }
  }
  if (!key_dev) {
    e = cudaMemcpyAsync(c->d_key, bounce, MS_KEY_BYTES, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->sync_ev, c->stream);
    int rc = (e == cudaSuccess) ? wait_event(c, c->sync_ev, std::max<uint32_t>(cfg.timeout_ms, 1000)) : MS_ECUDA;
    explicit_bzero(bounce, MS_KEY_BYTES);
    cudaFreeHost(bounce);
    if (rc != MS_OK) {
      release(c);
      return rc;
    }
  }
#undef MS_TRY

  c->shape_explicit = cfg.blocks_per_thread || cfg.threads_per_cta || cfg.dr_unroll;
  if (cfg.blocks_per_thread) c->tune.bpt = (int)cfg.blocks_per_thread;
  if (cfg.threads_per_cta) c->tune.tpc = (int)cfg.threads_per_cta;
  if (cfg.dr_unroll) c->tune.unr = (int)cfg.dr_unroll;
  if (cfg.rounds != 20 && !cfg.dr_unroll) c->tune.unr = (int)cfg.rounds / 2;
  // the shared prelude needs >= 2 blocks per thread and a full unroll
  if (c->tune.bpt < 2 || c->tune.unr != (int)cfg.rounds / 2) c->tune.hoist = 0;
  if (!shape_available((int)cfg.rounds, c->tune)) c->tune.hoist = 0;
  if (!shape_available((int)cfg.rounds, c->tune)) {
    release(c);
    return MS_EINVAL;
  }
  c->alive = true;
  *out = c;
  return MS_OK;
}

}  // namespace

int ms_init(ms_ctx **out, const uint8_t *key, const ms_config *cfg) { return init_ctx(out, key, nullptr, cfg); }

int ms_clone(ms_ctx *parent, uint32_t domain, ms_ctx **out) {
  if (!out) return MS_EINVAL;
  *out = nullptr;
  if (!parent || !parent->alive) return MS_ENOTINIT;
  ms_config cfg = parent->cfg;
  cfg.domain = domain;
  cfg.stream = nullptr;  // its own stream
  cfg.use_stream = 0;
  // the parent's shape, explicit or tuned, is taken over below
  cfg.blocks_per_thread = cfg.threads_per_cta = cfg.dr_unroll = 0;
  ms_ctx *c = nullptr;
  const int rc = init_ctx(&c, nullptr, parent->d_key, &cfg);
  if (rc != MS_OK) return rc;
  {
    std::lock_guard<std::mutex> lk(parent->mu);
    c->tune = parent->tune;
    c->qtune = parent->qtune;
    c->shape_explicit = parent->shape_explicit;
  }
  *out = c;
  return MS_OK;
}

int ms_encrypt_pages(ms_ctx *ctx, const ms_page *pages, size_t n) { return submit_list_host(ctx, pages, n); }
int ms_decrypt_pages(ms_ctx *ctx, const ms_page *pages, size_t n) { return submit_list_host(ctx, pages, n); }
int ms_crypt_pages_dom(ms_ctx *ctx, const ms_page_dom *pages, size_t n) { return submit_list_host(ctx, pages, n); }

int ms_encrypt_pages_dev(ms_ctx *ctx, const ms_page *d_pages, size_t n) { return submit_list_dev(ctx, d_pages, n); }
int ms_decrypt_pages_dev(ms_ctx *ctx, const ms_page *d_pages, size_t n) { return submit_list_dev(ctx, d_pages, n); }
int ms_crypt_pages_dom_dev(ms_ctx *ctx, const ms_page_dom *d_pages, size_t n) {
  return submit_list_dev(ctx, d_pages, n);
}

int ms_crypt_range(ms_ctx *c, int op, void *d_base, uint64_t first_page_id, size_t n_pages) {
  if (!c || !c->alive) return MS_ENOTINIT;
  if (op != MS_ENCRYPT && op != MS_DECRYPT) return MS_EINVAL;
  if (n_pages == 0) return MS_OK;
  if (!d_base || ((uintptr_t)d_base & 15u)) return MS_EINVAL;
  // ids first_page_id .. first_page_id + n_pages - 1 must not wrap past 2^64 - 1
  // (a wrapped id would reuse the keystream of page 0, 1, ...)
  if (n_pages - 1 > ~first_page_id) return MS_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  PageArgs a = make_args(c);
  a.base = (uint8_t *)d_base;
  a.first_id = first_page_id;
  a.n_pages = n_pages;
  cudaError_t e = launch_pages(c, a, c->stream);
  return e == cudaSuccess ? MS_OK : cuda_fail(c, e);
}

namespace {
// The call status for status-word bits: a starved feed first, then a bad entry.
int status_code(unsigned st) {
  if (st & kStatusFeedTimeout) return MS_ESTARVED;
  return (st & kStatusBadEntry) ? MS_EINVAL : MS_OK;
}
}  // namespace

int ms_sync(ms_ctx *c) { return c ? ms_sync_for(c, c->cfg.timeout_ms) : MS_ENOTINIT; }

// ---------------------------------------------------------------- tickets
int ms_submit_host(ms_ctx *c, int op, const ms_page *pages, size_t n, uint64_t *ticket) {
  if (!c || !c->alive) return MS_ENOTINIT;
  if (!ticket || (op != MS_ENCRYPT && op != MS_DECRYPT)) return MS_EINVAL;
  if (n) {
    const int rc = check_list_host(c, pages, n);
    if (rc != MS_OK) return rc;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  const uint64_t t = c->tk_next.load();
  cudaEvent_t &ev = c->tk_ev[t % kTickets];
  if (!ev) {
    const cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(c, e);
  } else {
    // the slot's previous ticket (t - kTickets) must have finished before its event is reused
    const cudaError_t q = cudaEventQuery(ev);
    if (q == cudaErrorNotReady) return MS_EBUSY;
    if (q != cudaSuccess) return cuda_fail(c, q);
  }
  if (n) {
    const int rc = submit_list_host_locked(c, pages, n);
    if (rc != MS_OK) return rc;
  }
  const cudaError_t e = cudaEventRecord(ev, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  c->tk_next.store(t + 1, std::memory_order_release);  // the event exists and is recorded
  *ticket = t;
  return MS_OK;
}

int ms_host_device_address(const void *host_ptr, uint64_t *dev_addr) {
  if (!host_ptr || !dev_addr) return MS_EINVAL;
  void *dp = nullptr;
  if (cudaHostGetDevicePointer(&dp, const_cast<void *>(host_ptr), 0) != cudaSuccess || !dp) {
    cudaGetLastError();
    return MS_EINVAL;  // not pinned, mapped host memory
  }
  *dev_addr = (uint64_t)dp;
  return MS_OK;
}

// Lock-free, so that a client waiting on its ticket is not held up by
// another thread's ms_sync.  A newer ticket may re-record the slot's event
// after the distance check; that happens only once the old ticket has
// finished, and then reads as pending once, until the distance check says done.
int ms_poll(ms_ctx *c, uint64_t ticket) {
  if (!c || !c->alive) return MS_ENOTINIT;
  const uint64_t next = c->tk_next.load(std::memory_order_acquire);
  if (ticket >= next) return MS_EINVAL;
  if (next - ticket > kTickets) return 1;  // its slot was reused, which needs it finished
  DeviceGuard g(c->device);
  const cudaError_t q = cudaEventQuery(c->tk_ev[ticket % kTickets]);
  if (q == cudaSuccess) return 1;
  if (q == cudaErrorNotReady) return 0;
  return cuda_fail(c, q);
}

int ms_wait(ms_ctx *c, uint64_t ticket, uint32_t timeout_ms) {
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  for (int it = 0;; ++it) {
    const int p = ms_poll(c, ticket);
    if (p != 0) return p == 1 ? MS_OK : p;
    const auto el = clk::now() - t0;
    if (el > std::chrono::milliseconds(timeout_ms)) return MS_ETIMEDOUT;
    if (el > std::chrono::microseconds(50)) {
      struct timespec ts = {0, 5000};
      nanosleep(&ts, nullptr);
    }
  }
}

int ms_sync_for(ms_ctx *c, uint32_t timeout_ms) {
  if (!c || !c->alive) return MS_ENOTINIT;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  // A status read left unfinished by an earlier timed-out call is collected
  // first, so no bad-entry report is lost.
  if (c->status_pending) {
    int rc = wait_event(c, c->status_ev, timeout_ms);
    if (rc != MS_OK) return rc;
    c->status_pending = false;
    c->status_acc |= *(volatile unsigned int *)c->h_status;
  }
  if (!c->status_dirty) {
    // Nothing since the last read can have set a status bit: wait for the work.
    cudaError_t e = cudaEventRecord(c->sync_ev, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e);
    const int rc = wait_event(c, c->sync_ev, timeout_ms);
    if (rc != MS_OK) return rc;
    const unsigned st = c->status_acc;
    c->status_acc = 0;
    return status_code(st);
  }
  // Queue the read and clear of the device status word behind the submitted
  // work and wait once (one round trip).  On a timeout the read stays
  // pending and the next call collects it first (above).
  k_status_take<<<1, 1, 0, c->stream>>>(c->d_status, c->h_status_dev);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(c->status_ev, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  c->status_dirty = false;  // the queued read covers every launch before it
  c->status_pending = true;
  int rc = wait_event(c, c->status_ev, timeout_ms);
  if (rc != MS_OK) return rc;
  c->status_pending = false;
  const unsigned st = *(volatile unsigned int *)c->h_status | c->status_acc;
  c->status_acc = 0;
  return status_code(st);
}

int ms_shutdown(ms_ctx *c) {
  if (!c) return MS_OK;
  if (c->children.load() > 0) return MS_EBUSY;  // a batch, server or resident set still uses it
  DeviceGuard g(c->device);
  if (c->alive) {
    std::lock_guard<std::mutex> lk(c->mu);
    // Finish queued work (bounded).  If it does not finish, nothing is
    // touched: kernels still queued read the key and the buffers, so the
    // context stays as it is and the call can be repeated.
    cudaError_t e = cudaEventRecord(c->sync_ev, c->stream);
    int rc = e == cudaSuccess ? wait_event(c, c->sync_ev, c->cfg.timeout_ms) : cuda_fail(c, e);
    for (int i = 0; i < kMaxHostStreams && rc == MS_OK; ++i)
      if (c->hs[i]) {
        e = cudaEventRecord(c->hs_ev[i], c->hs[i]);
        rc = e == cudaSuccess ? wait_event(c, c->hs_ev[i], c->cfg.timeout_ms) : cuda_fail(c, e);
      }
    if (rc != MS_OK) return rc;
    // then overwrite the key on the device
    if (c->d_key) cudaMemsetAsync(c->d_key, 0, MS_KEY_BYTES, c->stream);
    e = cudaEventRecord(c->sync_ev, c->stream);
    rc = e == cudaSuccess ? wait_event(c, c->sync_ev, c->cfg.timeout_ms) : cuda_fail(c, e);
    if (rc != MS_OK) return rc;
    c->alive = false;
  }
  release(c);
  return MS_OK;
}

int ms_get_shape(const ms_ctx *c, ms_shape *out) {
  if (!c || !c->alive) return MS_ENOTINIT;
  if (!out) return MS_EINVAL;
  out->blocks_per_thread = (uint32_t)c->tune.bpt;
  out->threads_per_cta = (uint32_t)c->tune.tpc;
  out->dr_unroll = (uint32_t)c->tune.unr;
  out->rot_policy = (uint32_t)c->tune.pol;
  out->hoist = (uint32_t)c->tune.hoist;
  return MS_OK;
}

int ms_set_shape(ms_ctx *c, const ms_shape *sh) {
  if (!c || !c->alive) return MS_ENOTINIT;
  if (!sh) return MS_EINVAL;
  Tune t;
  t.bpt = (int)sh->blocks_per_thread;
  t.tpc = (int)sh->threads_per_cta;
  t.unr = (int)sh->dr_unroll;
  t.pol = (int)sh->rot_policy;
  t.hoist = (int)sh->hoist;
  if (!shape_available((int)c->cfg.rounds, t)) return MS_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  c->tune = t;
  c->shape_explicit = true;
  c->tune_gen.fetch_add(1);
  return MS_OK;
}

// ---------------------------------------------------------------- host pages
int ms_crypt_host(ms_ctx *c, int op, void *host_base, uint64_t first_page_id, size_t n_pages,
                  size_t chunk_bytes, int n_streams) {
  if (!c || !c->alive) return MS_ENOTINIT;
  if (op != MS_ENCRYPT && op != MS_DECRYPT) return MS_EINVAL;
  if (n_pages == 0) return MS_OK;
  if (!host_base) return MS_EINVAL;
  if (n_pages - 1 > ~first_page_id) return MS_EINVAL;  // ids must not wrap past 2^64 - 1
  if (chunk_bytes == 0) chunk_bytes = (size_t)16 << 20;
  if (chunk_bytes % MS_PAGE_BYTES) return MS_EINVAL;
  if (n_streams == 0) n_streams = 2;
  if (n_streams < 1 || n_streams > kMaxHostStreams) return MS_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaError_t e;
  if (c->hs_cap < chunk_bytes) {
    for (int i = 0; i < kMaxHostStreams; ++i) {
      if (c->hs_buf[i]) {
        if (c->hs[i]) cudaStreamSynchronize(c->hs[i]);
        cudaFree(c->hs_buf[i]);
        c->hs_buf[i] = nullptr;
      }
    }
    c->hs_cap = chunk_bytes;
  }
  // every per-stream buffer holds hs_cap >= chunk_bytes bytes
  for (int i = 0; i < n_streams; ++i) {
    if (!c->hs[i]) {
      e = cudaStreamCreateWithFlags(&c->hs[i], cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(c, e);
      e = cudaEventCreateWithFlags(&c->hs_ev[i], cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_fail(c, e);
    }
    if (!c->hs_buf[i]) {
      e = cudaMalloc(&c->hs_buf[i], c->hs_cap);
      if (e != cudaSuccess) return alloc_fail(c, e);
    }
  }
  // order after earlier work on the context stream
  e = cudaEventRecord(c->sync_ev, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  for (int i = 0; i < n_streams; ++i) cudaStreamWaitEvent(c->hs[i], c->sync_ev, 0);

  const size_t pages_per_chunk = chunk_bytes / MS_PAGE_BYTES;
  uint8_t *hb = (uint8_t *)host_base;
  size_t chunk = 0;
  int fail = MS_OK;  // the first error; chunks already issued are still drained
  for (size_t p0 = 0; p0 < n_pages; p0 += pages_per_chunk, ++chunk) {
    const int si = (int)(chunk % n_streams);
    const size_t np = std::min(pages_per_chunk, n_pages - p0);
    const size_t bytes = np * MS_PAGE_BYTES;
    cudaStream_t s = c->hs[si];
    e = injected(MS_FAULT_COPY);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->hs_buf[si], hb + p0 * MS_PAGE_BYTES, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      PageArgs a = make_args(c);
      a.base = (uint8_t *)c->hs_buf[si];
      a.first_id = first_page_id + p0;
      a.n_pages = np;
      e = launch_pages(c, a, s);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hb + p0 * MS_PAGE_BYTES, c->hs_buf[si], bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) {
      fail = cuda_fail(c, e);
      ++chunk;
      break;
    }
  }
  // Wait (bounded: timeout_ms per chunk) for everything issued, also after an
  // error, so no copy lands in the caller's buffer after this call returns.
  const uint64_t n_chunks = chunk;
  int rc = MS_OK;
  const int used = (int)std::min<uint64_t>((uint64_t)n_streams, n_chunks);
  const uint64_t limit = (uint64_t)c->cfg.timeout_ms * std::max<uint64_t>(1, n_chunks);
  for (int i = 0; i < used; ++i) {
    e = cudaEventRecord(c->hs_ev[i], c->hs[i]);
    int r = (e == cudaSuccess) ? wait_event(c, c->hs_ev[i], (uint32_t)std::min<uint64_t>(limit, 0xffffffffu))
                               : cuda_fail(c, e);
    if (r != MS_OK && rc == MS_OK) rc = r;
  }
  return fail != MS_OK ? fail : rc;
}

}  // extern "C"
