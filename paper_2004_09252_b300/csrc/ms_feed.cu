// Fed form: one persistent K2 launch drains a device work queue while the
// host is still filling it.  The batched form launches one graph per submit,
// and every launch pays a start, a tail where its last CTAs finish alone and,
// for the first one, the whole host fill before it; here the GPU starts after
// the first chunk and runs until the feed is closed.
//
// Publication: the host copies entries [published, filled) into the device
// queue on the feed's copy stream, then copies the new count (from a pinned
// slot written once) into the device count word on the same stream, so the
// count changes only after the entries it covers have landed.  Closing copies
// a 1 into the closed word after the last count.
//
// Kernel: each CTA claims entries with one atomicAdd on the head (guided
// sizes, as K2) and works through its claim as it is published, piece by
// piece.  Every wait is bounded: after wait_ms without a publication the
// kernel sets a timeout bit in the status word and leaves; after the close
// it leaves once nothing of its claim is left to publish.
// Paper counterpart (Sec. 4.4): the GPU module's workers consume queues that
// host threads keep filling.
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "ms_internal.h"

namespace {

constexpr uint32_t kMinChunk = 1024;  // entries per publication, at least
constexpr int kHeadWord = 32;         // the claimed head apart from the polled words
constexpr int kCtlWords = 64;
constexpr int kFeedThreads = 128;     // threads per CTA

struct FeedArgs {
  const ms_page *items;   // device queue
  const uint32_t *count;  // published entries (written by copies)
  const uint32_t *closed; // 1 after the last count
  uint32_t *head;         // next unclaimed entry
  uint32_t grab;          // largest claim
  uint64_t wait_ns;       // longest wait for a publication
  const uint4 *key;
  uint32_t domain;
  unsigned int *status;
  ms::MulConsts mc;
};

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0: wait until entry `pos` is published (returns the published
// count, > pos), or the feed is closed with nothing at `pos` (returns `pos`,
// *leave = 1), or wait_ns runs out (status bit, *leave = 1).  Polls back off
// from 0.25 to 8 us, so waiting CTAs leave the control words' L2 slice to
// the copies and the claims.
__device__ __forceinline__ uint32_t wait_published(const FeedArgs &q, uint32_t pos, int *leave) {
  const uint64_t t0 = gtime();
  uint32_t nap = 256;
  for (;;) {
    const uint32_t cl = ld_acquire_gpu(q.closed);  // read before the count: after a 1 the count is final
    const uint32_t c = ld_acquire_gpu(q.count);
    if (c > pos) return c;
    if (cl) {
      *leave = 1;
      return pos;
    }
    if (gtime() - t0 > q.wait_ns) {
      atomicOr(q.status, ms::kStatusFeedTimeout);
      *leave = 1;
      return pos;
    }
    __nanosleep(nap);
    nap = min(nap * 2u, 8192u);
  }
}

template <int ROUNDS, int BPT, int UNR, int POL, bool HOIST>
__global__ void __launch_bounds__(512) k_feed(const FeedArgs q) {
  constexpr uint32_t TPP = 64 / BPT;
  __shared__ uint32_t s_a, s_b;
  __shared__ int s_leave;
  const uint32_t pages_per_pass = blockDim.x / TPP;
  const uint32_t lp = threadIdx.x / TPP;
  const uint32_t t = threadIdx.x % TPP;
  const uint32_t cap = max(q.grab, pages_per_pass);
  ms::BlockSeed s;
  ms::load_key(q.key, s.k);
  s.n2 = q.domain;
  for (;;) {
    // claim: guided by what is published and not yet claimed
    if (threadIdx.x == 0) {
      const uint32_t seen = *reinterpret_cast<volatile const uint32_t *>(q.head);
      const uint32_t pub = ld_acquire_gpu(q.count);
      const uint32_t rem = seen < pub ? pub - seen : 0;
      uint32_t take = rem / (2u * gridDim.x);
      take = (take + pages_per_pass - 1) / pages_per_pass * pages_per_pass;
      take = min(max(take, pages_per_pass), cap);
      const uint32_t base = atomicAdd(q.head, take);
      s_a = base;
      s_b = base + take;
    }
    __syncthreads();
    uint32_t pos = s_a;
    const uint32_t claim_end = s_b;
    __syncthreads();
    // work through the claim as it is published
    int leave = 0;
    while (pos < claim_end) {
      if (threadIdx.x == 0) {
        int lv = 0;
        const uint32_t c = wait_published(q, pos, &lv);
        s_a = min(claim_end, c);
        s_leave = lv;
      }
      __syncthreads();
      const uint32_t hi = s_a;
      leave = s_leave;
      __syncthreads();
      for (uint32_t p = pos + lp; p < hi; p += pages_per_pass) {
        // the entry was written by a copy during this launch: read it from L2
        const ulonglong2 raw = __ldcg(reinterpret_cast<const ulonglong2 *>(q.items) + p);
        ms_page e;
        e.addr = raw.x;
        e.page_id = raw.y;
        if (!ms::entry_ok(e.addr)) {
          if (t == 0) atomicOr(q.status, ms::kStatusBadEntry);
          continue;
        }
        s.n0 = (uint32_t)e.page_id;
        s.n1 = (uint32_t)(e.page_id >> 32);
        ms::page_blocks<ROUNDS, BPT, UNR, POL, HOIST>(reinterpret_cast<uint4 *>(e.addr), s, t, TPP, q.mc);
      }
      if (leave) break;
      pos = hi;
    }
    if (leave) break;
  }
}

using FeedLaunch = cudaError_t (*)(const FeedArgs &, int grid, int tpc, cudaStream_t);

template <int R, int B, int U, int P, bool H>
cudaError_t launch_feed(const FeedArgs &a, int grid, int tpc, cudaStream_t s) {
  k_feed<R, B, U, P, H><<<grid, tpc, 0, s>>>(a);
  return cudaGetLastError();
}

struct FeedEntry {
  int rounds, bpt;
  const void *fn;
  FeedLaunch launch;
};

#define MS_FEED(R, B, H) {R, B, (const void *)&k_feed<R, B, R / 2, 1, H>, &launch_feed<R, B, R / 2, 1, H>}
const FeedEntry kFeed[] = {
    MS_FEED(20, 4, true), MS_FEED(20, 2, true), MS_FEED(20, 1, false),
    MS_FEED(12, 4, true), MS_FEED(12, 2, true), MS_FEED(12, 1, false),
    MS_FEED(8, 4, true),  MS_FEED(8, 2, true),  MS_FEED(8, 1, false),
};
#undef MS_FEED

// The instance with the context's blocks per thread (else 4), byte-permute
// rotations and, for 2 or 4 blocks per thread, the shared prelude.
const FeedEntry *feed_kernel(const ms_ctx *c) {
  const FeedEntry *fallback = nullptr;
  for (const FeedEntry &e : kFeed) {
    if (e.rounds != (int)c->cfg.rounds) continue;
    if (e.bpt == c->tune.bpt) return &e;
    if (e.bpt == 4) fallback = &e;
  }
  return fallback;
}

}  // namespace

struct ms_feed {
  ms_ctx *ctx = nullptr;
  ms_feed_config cfg{};
  ms_page *h_items = nullptr, *d_items = nullptr;
  uint32_t *d_ctl = nullptr;    // count @0, closed @1, head @32 (its own 128-byte line)
  uint32_t *h_counts = nullptr; // pinned: one slot per publication, written once
  uint32_t *h_one = nullptr;    // pinned 1, the closed value
  size_t n_slots = 0, n_pub = 0;
  uint32_t filled = 0, published = 0;
  bool closed = false;
  cudaStream_t cs = nullptr;
  cudaEvent_t started = nullptr, done = nullptr;
  const FeedEntry *kernel = nullptr;  // the instance chosen (and loaded) at creation
  int grid = 0;                       // persistent CTAs: all of it that fit
  std::mutex mu;
  ms_feed_stats stats{};
};

using namespace ms;

namespace {

void free_feed(ms_feed *f) {
  if (f->cs) cudaStreamDestroy(f->cs);
  if (f->started) cudaEventDestroy(f->started);
  if (f->done) cudaEventDestroy(f->done);
  if (f->h_items) cudaFreeHost(f->h_items);
  if (f->h_counts) cudaFreeHost(f->h_counts);
  if (f->h_one) cudaFreeHost(f->h_one);
  if (f->d_items) cudaFree(f->d_items);
  if (f->d_ctl) cudaFree(f->d_ctl);
  delete f;
}

// Copy [published, filled) and then the new count; the caller holds f->mu.
int publish(ms_feed *f) {
  if (f->filled == f->published) return MS_OK;
  if (f->n_pub >= f->n_slots) return MS_ERANGE;  // cannot happen: slots cover capacity / chunk + 1
  ms_ctx *c = f->ctx;
  DeviceGuard g(c->device);
  const size_t k = f->filled - f->published;
  f->h_counts[f->n_pub] = f->filled;
  cudaError_t e = injected(MS_FAULT_COPY);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(f->d_items + f->published, f->h_items + f->published, k * sizeof(ms_page),
                        cudaMemcpyHostToDevice, f->cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(f->d_ctl, f->h_counts + f->n_pub, sizeof(uint32_t), cudaMemcpyHostToDevice, f->cs);
  if (e != cudaSuccess) return cuda_fail(c, e);
  f->n_pub += 1;
  f->published = f->filled;
  f->stats.publications += 1;
  return MS_OK;
}

}  // namespace

extern "C" {

void ms_feed_config_default(ms_feed_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->capacity = 1u << 20;
  cfg->chunk = 16384;
  cfg->wait_ms = 2000;
}

int ms_feed_create(ms_ctx *c, const ms_feed_config *cfg_in, ms_feed **out) {
  if (!out) return MS_EINVAL;
  *out = nullptr;
  if (!c || !c->alive) return MS_ENOTINIT;
  ms_feed_config cfg;
  if (cfg_in) cfg = *cfg_in; else ms_feed_config_default(&cfg);
  if (cfg.capacity == 0) cfg.capacity = 1u << 20;
  if (cfg.chunk == 0) cfg.chunk = 16384;
  if (cfg.wait_ms == 0) cfg.wait_ms = 2000;
  if (cfg.capacity > MS_BATCH_MAX_CAPACITY) return MS_ERANGE;
  if (cfg.chunk < kMinChunk || cfg.wait_ms > 600000 || cfg.grab > 4096) return MS_EINVAL;
  if (!feed_kernel(c)) return MS_EINVAL;
  ms_feed *f = new (std::nothrow) ms_feed();
  if (!f) return MS_ENOMEM;
  f->ctx = c;
  f->cfg = cfg;
  f->n_slots = cfg.capacity / cfg.chunk + 2;
  f->closed = true;  // nothing running until ms_feed_open
  DeviceGuard g(c->device);
  cudaError_t e = cudaHostAlloc(&f->h_items, (size_t)cfg.capacity * sizeof(ms_page), cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaHostAlloc(&f->h_counts, f->n_slots * sizeof(uint32_t), cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaHostAlloc(&f->h_one, sizeof(uint32_t), cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaMalloc(&f->d_items, (size_t)cfg.capacity * sizeof(ms_page));
  if (e == cudaSuccess) e = cudaMalloc(&f->d_ctl, kCtlWords * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&f->cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->started, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_feed(f);
    return alloc_fail(c, e);
  }
  *f->h_one = 1;
  // Load the kernel and size its grid now (the occupancy query loads the
  // module), so that neither falls into a run.
  const FeedEntry *k = feed_kernel(c);
  f->kernel = k;
  int fit = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k->fn, kFeedThreads, 0);
  if (e != cudaSuccess) {
    free_feed(f);
    return cuda_fail(c, e);
  }
  f->grid = (fit < 1 ? 1 : fit) * c->sm_count;
  c->children.fetch_add(1);
  *out = f;
  return MS_OK;
}

int ms_feed_open(ms_feed *f) {
  if (!f) return MS_EINVAL;
  ms_ctx *c = f->ctx;
  if (!c || !c->alive) return MS_ENOTINIT;
  std::lock_guard<std::mutex> lk(f->mu);
  if (!f->closed) return MS_EBUSY;  // already open
  DeviceGuard g(c->device);
  // the previous run (if any) has left and its copies have landed before the
  // control words and the queue are reused
  int rc = wait_event(c, f->done, c->cfg.timeout_ms + f->cfg.wait_ms);
  if (rc == MS_OK) {
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return cuda_fail(c, cudaGetLastError());
    const cudaError_t e = cudaEventRecord(ev, f->cs);
    rc = e == cudaSuccess ? wait_event(c, ev, c->cfg.timeout_ms) : cuda_fail(c, e);
    cudaEventDestroy(ev);
  }
  if (rc != MS_OK) return rc;
  const FeedEntry *k = f->kernel;
  std::lock_guard<std::mutex> lk2(c->mu);
  // control words zeroed on the context stream, then the kernel; the copy
  // stream starts after the zeroing, so no publication is overwritten
  cudaError_t e = cudaMemsetAsync(f->d_ctl, 0, kCtlWords * sizeof(uint32_t), c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(f->started, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(f->cs, f->started, 0);
  FeedArgs a{};
  a.items = f->d_items;
  a.count = f->d_ctl;
  a.closed = f->d_ctl + 1;
  a.head = f->d_ctl + kHeadWord;
  a.grab = f->cfg.grab ? f->cfg.grab : (uint32_t)c->qtune.grab;
  a.wait_ns = (uint64_t)f->cfg.wait_ms * 1000000ull;
  a.key = c->d_key;
  a.domain = c->cfg.domain;
  a.status = c->d_status;
  a.mc.m12 = 1u << 12;
  a.mc.m7 = 1u << 7;
  if (e == cudaSuccess) e = injected(MS_FAULT_LAUNCH);
  if (e == cudaSuccess) e = k->launch(a, f->grid, kFeedThreads, c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(f->done, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);  // a kernel that did start leaves by its bounded wait
  c->status_dirty = true;  // the kernel may report a starved wait or a bad entry
  f->filled = f->published = 0;
  f->n_pub = 0;
  f->closed = false;
  f->stats.grid = (uint64_t)f->grid;
  f->stats.runs += 1;
  return MS_OK;
}

int ms_feed_add_requests(ms_feed *f, size_t n_requests, const int *ops, const uint64_t *offsets,
                         const ms_page *pages, size_t *added) {
  if (added) *added = 0;
  if (!f || (n_requests && (!ops || !offsets || !pages))) return MS_EINVAL;
  std::lock_guard<std::mutex> lk(f->mu);
  if (f->closed) return MS_EINVAL;  // not open
  for (size_t r = 0; r < n_requests; ++r) {
    if (offsets[r + 1] < offsets[r]) return MS_EINVAL;
    if (ops[r] != MS_ENCRYPT && ops[r] != MS_DECRYPT) return MS_EINVAL;
    const size_t n = (size_t)(offsets[r + 1] - offsets[r]);
    const ms_page *src = pages + offsets[r];
    uint64_t bad = 0;
    for (size_t i = 0; i < n; ++i) bad |= (uint64_t)(src[i].addr == 0) | (src[i].addr & 15u);
    if (bad) return MS_EINVAL;
    if (n > f->cfg.capacity - f->filled) return MS_ERANGE;  // the feed holds `capacity` entries in all
    std::memcpy(f->h_items + f->filled, src, n * sizeof(ms_page));
    f->filled += (uint32_t)n;
    f->stats.requests += 1;
    f->stats.pages += n;
    if (f->filled - f->published >= f->cfg.chunk) {
      const int rc = publish(f);
      if (rc != MS_OK) return rc;
    }
    if (added) *added = r + 1;
  }
  return MS_OK;
}

int ms_feed_close(ms_feed *f) {
  if (!f) return MS_EINVAL;
  std::lock_guard<std::mutex> lk(f->mu);
  if (f->closed) return MS_OK;
  int rc = publish(f);
  if (rc != MS_OK) return rc;
  DeviceGuard g(f->ctx->device);
  const cudaError_t e = cudaMemcpyAsync(f->d_ctl + 1, f->h_one, sizeof(uint32_t), cudaMemcpyHostToDevice, f->cs);
  f->stats.closes += 1;
  if (e != cudaSuccess) return cuda_fail(f->ctx, e);
  f->closed = true;
  return MS_OK;
}

int ms_feed_get_stats(const ms_feed *f, ms_feed_stats *out) {
  if (!f || !out) return MS_EINVAL;
  *out = f->stats;
  return MS_OK;
}

int ms_feed_destroy(ms_feed *f) {
  if (!f) return MS_OK;
  ms_ctx *c = f->ctx;
  int rc = ms_feed_close(f);  // if open: the kernel leaves once it has drained what was published
  DeviceGuard g(c->device);
  // the kernel ends by itself: after the close, or wait_ms after its last publication
  const uint64_t bound = (uint64_t)c->cfg.timeout_ms + f->cfg.wait_ms;
  int r = wait_event(c, f->done, (uint32_t)std::min<uint64_t>(bound, 0xffffffffu));
  if (r == MS_OK) {
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
      if (cudaEventRecord(ev, f->cs) == cudaSuccess) r = wait_event(c, ev, c->cfg.timeout_ms);
      cudaEventDestroy(ev);
    }
  }
  if (r != MS_OK) return r;  // still running: leave the buffers allocated
  free_feed(f);
  c->children.fetch_sub(1);
  return rc;
}

}  // extern "C"
