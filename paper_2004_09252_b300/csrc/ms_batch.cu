// Batched form: requests (uneven page lists, as faults and evictions produce
// them) are appended to a host-side queue buffer; a submit copies the buffer
// to the device work queue and launches the persistent kernel K2 through a
// captured CUDA graph (memset of the queue head, then K2).  Two queue buffers
// alternate, so the host fills one while the GPU drains the other, and the
// H2D copy of a submit runs on its own stream, beside the previous K2.
//
// Paper counterpart (Sec. 4.4): the GPU module's workers take pages from
// queues that many host threads fill; here one device queue per batch feeds
// every CTA of a persistent grid, and the grid ends when the queue is empty.
#include <cstring>
#include <mutex>
#include <new>

#include "ms_internal.h"

namespace {

constexpr size_t kHeader = 256;       // queue buffer: [count @0][head @128][items @256]
constexpr size_t kHeadOffset = 128;

struct QBuf {
  uint8_t *h = nullptr;  // pinned host copy (header + items)
  uint8_t *d = nullptr;  // device work queue
  size_t n = 0;          // items queued
  cudaEvent_t done = nullptr;    // K2 over this buffer finished (the device copy is free again)
  cudaEvent_t copied = nullptr;  // the H2D copy finished (the host copy is free again)
  bool inflight = false;  // submitted, host copy possibly still being read
  cudaGraphExec_t exec = nullptr;
  unsigned exec_key = ~0u;  // tune generation the graph was captured for
};

}  // namespace

struct ms_batch {
  ms_ctx *ctx = nullptr;
  ms_batch_config cfg{};
  QBuf buf[2];
  int cur = 0;
  cudaStream_t copy_stream = nullptr;  // queue H2D copies, overlapping the previous K2
  std::mutex mu;
  ms_batch_stats stats{};
};

using namespace ms;

namespace {

// Bounded wait for everything the batch issued.  An event never recorded
// counts as complete, so buffers never submitted need no care; a copy
// enqueued by a submit that failed later is waited for too.
int wait_batch(ms_batch *b) {
  for (QBuf &q : b->buf)
    for (cudaEvent_t ev : {q.copied, q.done})
      if (ev) {
        const int r = wait_event(b->ctx, ev, b->ctx->cfg.timeout_ms);
        if (r != MS_OK) return r;
      }
  return MS_OK;
}

// Frees a batch whose work has finished (or was never issued).
void free_batch(ms_batch *b) {
  for (QBuf &q : b->buf) {
    if (q.exec) cudaGraphExecDestroy(q.exec);
    if (q.done) cudaEventDestroy(q.done);
    if (q.copied) cudaEventDestroy(q.copied);
    if (q.h) cudaFreeHost(q.h);
    if (q.d) cudaFree(q.d);
  }
  if (b->copy_stream) cudaStreamDestroy(b->copy_stream);
  delete b;
}

// The K2 launch parameters of this batch (config overrides, else the context's tuning).
void batch_params(const ms_batch *b, QueueKernel *k, int *grid, int *grab) {
  const ms_ctx *c = b->ctx;
  queue_kernel((int)c->cfg.rounds, c->tune, k);
  const int cps = b->cfg.ctas_per_sm ? (int)b->cfg.ctas_per_sm : c->qtune.ctas_per_sm;
  *grid = queue_grid(c, *k, c->tune.tpc, cps);
  *grab = b->cfg.grab ? (int)b->cfg.grab : c->qtune.grab;
}

size_t item_bytes(const ms_batch *b) { return b->cfg.per_page_domain ? sizeof(ms_page_dom) : sizeof(ms_page); }

QueueArgs queue_args(const ms_batch *b, const QBuf &q, int grab) {
  const ms_ctx *c = b->ctx;
  QueueArgs a{};
  if (b->cfg.per_page_domain)
    a.ditems = reinterpret_cast<const ms_page_dom *>(q.d + kHeader);
  else
    a.items = reinterpret_cast<const ms_page *>(q.d + kHeader);
  a.count = reinterpret_cast<const uint32_t *>(q.d);
  a.head = reinterpret_cast<uint32_t *>(q.d + kHeadOffset);
  a.grab = (uint32_t)grab;
  a.key = c->d_key;
  a.domain = c->cfg.domain;
  a.status = c->d_status;
  a.mc.m12 = 1u << 12;
  a.mc.m7 = 1u << 7;
  return a;
}

// (Re)capture the graph of queue buffer q: head := 0, then K2 over the queue.
cudaError_t capture(ms_batch *b, QBuf &q) {
  QueueKernel k;
  int grid, grab;
  batch_params(b, &k, &grid, &grab);
  const QueueArgs a = queue_args(b, q, grab);
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaGraph_t g = nullptr;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = cudaMemsetAsync(q.d + kHeadOffset, 0, sizeof(uint32_t), cs);
    cudaError_t e2 = (e1 == cudaSuccess) ? k.launch(a, grid, b->ctx->tune.tpc, cs) : e1;
    e = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) {
    if (q.exec) {
      cudaGraphExecDestroy(q.exec);
      q.exec = nullptr;
    }
    e = cudaGraphInstantiate(&q.exec, g, 0);
  }
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e == cudaSuccess) q.exec_key = b->ctx->tune_gen.load();
  return e;
}

// The host copy of q may be rewritten once its last H2D copy has finished
// (the kernel reading the device copy may still run).
int host_buffer_ready(ms_ctx *c, QBuf &q) {
  if (!q.inflight) return MS_OK;
  DeviceGuard g(c->device);
  const int rc = wait_event(c, q.copied, c->cfg.timeout_ms);
  if (rc == MS_OK) q.inflight = false;
  return rc;
}

// Copy n entries into the queue buffer at dst while checking them (address
// non-null and 16-byte aligned).  ms_page into a per-page-domain queue takes
// the context's domain.  Returns false on a bad entry; dst is then partly
// written but not counted.
template <typename E>
bool copy_checked(const ms_batch *b, uint8_t *dst, const E *src, size_t n) {
  constexpr bool kDom = sizeof(E) == sizeof(ms_page_dom);
  uint64_t bad = 0;
  if (kDom || !b->cfg.per_page_domain) {
    E *d = reinterpret_cast<E *>(dst);
    for (size_t i = 0; i < n; ++i) {
      const uint64_t a = src[i].addr;
      bad |= (uint64_t)(a == 0) | (a & 15u);
      d[i] = src[i];
    }
  } else {
    ms_page_dom *d = reinterpret_cast<ms_page_dom *>(dst);
    const uint32_t dom = b->ctx->cfg.domain;
    for (size_t i = 0; i < n; ++i) {
      const uint64_t a = src[i].addr;
      bad |= (uint64_t)(a == 0) | (a & 15u);
      d[i] = ms_page_dom{};
      d[i].addr = a;
      d[i].page_id = src[i].page_id;
      d[i].domain = dom;
    }
  }
  return bad == 0;
}

// Append one request of n entries; the caller holds b->mu.
template <typename E>
int append_locked(ms_batch *b, int op, const E *pages, size_t n) {
  ms_ctx *c = b->ctx;
  if (op != MS_ENCRYPT && op != MS_DECRYPT) return MS_EINVAL;
  if (n == 0) return MS_OK;
  if (!pages) return MS_EINVAL;
  QBuf &q = b->buf[b->cur];
  if (n > b->cfg.capacity || q.n + n > b->cfg.capacity) {
    // the entries are still checked first: a bad entry is MS_EINVAL whatever the size
    for (size_t i = 0; i < n; ++i)
      if (pages[i].addr == 0 || (pages[i].addr & 15u)) return MS_EINVAL;
    return n > b->cfg.capacity ? MS_ERANGE : MS_EBUSY;  // ERANGE: can never fit; EBUSY: submit first
  }
  const int rc = host_buffer_ready(c, q);
  if (rc != MS_OK) return rc;
  if (!copy_checked(b, q.h + kHeader + item_bytes(b) * q.n, pages, n)) return MS_EINVAL;
  q.n += n;
  b->stats.requests += 1;
  b->stats.pages += n;
  return MS_OK;
}

template <typename E>
int batch_append(ms_batch *b, int op, const E *pages, size_t n) {
  if (!b) return MS_EINVAL;
  ms_ctx *c = b->ctx;
  if (!c || !c->alive) return MS_ENOTINIT;
  constexpr bool kDom = sizeof(E) == sizeof(ms_page_dom);
  if (kDom && !b->cfg.per_page_domain) return MS_EINVAL;
  std::lock_guard<std::mutex> lk(b->mu);
  return append_locked(b, op, pages, n);
}

}  // namespace

extern "C" {

void ms_batch_config_default(ms_batch_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->capacity = 1u << 20;
  cfg->use_graph = 1;
}

int ms_batch_create(ms_ctx *c, const ms_batch_config *cfg_in, ms_batch **out) {
  if (!out) return MS_EINVAL;
  *out = nullptr;
  if (!c || !c->alive) return MS_ENOTINIT;
  ms_batch_config cfg;
  if (cfg_in) cfg = *cfg_in; else ms_batch_config_default(&cfg);
  if (cfg.capacity == 0) cfg.capacity = 1u << 20;
  if (cfg.capacity > MS_BATCH_MAX_CAPACITY) return MS_ERANGE;
  if (cfg.grab > 4096) return MS_EINVAL;
  QueueKernel k;
  if (!queue_kernel((int)c->cfg.rounds, c->tune, &k)) return MS_EINVAL;
  ms_batch *b = new (std::nothrow) ms_batch();
  if (!b) return MS_ENOMEM;
  b->ctx = c;
  b->cfg = cfg;
  DeviceGuard g(c->device);
  if (cudaStreamCreateWithFlags(&b->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return MS_ECUDA;
  }
  const size_t bytes = kHeader + (cfg.per_page_domain ? sizeof(ms_page_dom) : sizeof(ms_page)) * (size_t)cfg.capacity;
  for (QBuf &q : b->buf) {
    cudaError_t e = cudaHostAlloc(&q.h, bytes, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&q.d, bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q.copied, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      free_batch(b);
      return alloc_fail(c, e);
    }
    std::memset(q.h, 0, kHeader);
  }
  if (cfg.use_graph) {
    // capture both buffers' graphs now, so that no submit pays for it
    std::lock_guard<std::mutex> lk(c->mu);
    for (QBuf &q : b->buf) {
      const cudaError_t e = capture(b, q);
      if (e != cudaSuccess) {
        free_batch(b);
        return cuda_fail(c, e);
      }
    }
  }
  c->children.fetch_add(1);
  *out = b;
  return MS_OK;
}

int ms_batch_add(ms_batch *b, int op, const ms_page *pages, size_t n) { return batch_append(b, op, pages, n); }
int ms_batch_add_dom(ms_batch *b, int op, const ms_page_dom *pages, size_t n) {
  return batch_append(b, op, pages, n);
}

int ms_batch_add_requests(ms_batch *b, size_t n_requests, const int *ops, const uint64_t *offsets,
                          const ms_page *pages, size_t *added) {
  if (added) *added = 0;
  if (!b || (n_requests && (!ops || !offsets || !pages))) return MS_EINVAL;
  ms_ctx *c = b->ctx;
  if (!c || !c->alive) return MS_ENOTINIT;
  std::lock_guard<std::mutex> lk(b->mu);
  for (size_t r = 0; r < n_requests; ++r) {
    if (offsets[r + 1] < offsets[r]) return MS_EINVAL;
    const int rc = append_locked(b, ops[r], pages + offsets[r], (size_t)(offsets[r + 1] - offsets[r]));
    if (rc != MS_OK) return rc;
    if (added) *added = r + 1;
  }
  return MS_OK;
}

int ms_batch_submit(ms_batch *b) {
  if (!b) return MS_EINVAL;
  ms_ctx *c = b->ctx;
  if (!c || !c->alive) return MS_ENOTINIT;
  std::lock_guard<std::mutex> lk(b->mu);
  QBuf &q = b->buf[b->cur];
  if (q.n == 0) return MS_OK;
  std::lock_guard<std::mutex> lk2(c->mu);
  DeviceGuard g(c->device);
  const uint32_t count = (uint32_t)q.n;
  std::memcpy(q.h, &count, sizeof(count));
  // The copy into q.d waits for the K2 that last read q.d (two submits back)
  // and overlaps the K2 of the previous submit; this submit's K2 waits for it.
  cudaError_t e = cudaStreamWaitEvent(b->copy_stream, q.done, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(q.d, q.h, kHeader + item_bytes(b) * q.n, cudaMemcpyHostToDevice, b->copy_stream);
  if (e == cudaSuccess) e = cudaEventRecord(q.copied, b->copy_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, q.copied, 0);
  if (e != cudaSuccess) return cuda_fail(c, e);
  if (b->cfg.use_graph) {
    if (!q.exec || q.exec_key != c->tune_gen.load()) {
      e = capture(b, q);
      if (e != cudaSuccess) return cuda_fail(c, e);
    }
    e = injected(MS_FAULT_GRAPH);
    if (e == cudaSuccess) e = cudaGraphLaunch(q.exec, c->stream);
    b->stats.graph_launches += 1;
  } else {
    QueueKernel k;
    int grid, grab;
    batch_params(b, &k, &grid, &grab);
    e = cudaMemsetAsync(q.d + kHeadOffset, 0, sizeof(uint32_t), c->stream);
    if (e == cudaSuccess) e = k.launch(queue_args(b, q, grab), grid, c->tune.tpc, c->stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(q.done, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  q.inflight = true;
  q.n = 0;
  b->stats.submits += 1;
  b->cur ^= 1;
  return MS_OK;
}

int ms_batch_get_stats(const ms_batch *b, ms_batch_stats *out) {
  if (!b || !out) return MS_EINVAL;
  *out = b->stats;
  return MS_OK;
}

int ms_batch_destroy(ms_batch *b) {
  if (!b) return MS_OK;
  ms_ctx *c = b->ctx;
  DeviceGuard g(c->device);
  const int rc = wait_batch(b);
  if (rc != MS_OK) return rc;  // still in use on the GPU: keep it allocated
  free_batch(b);
  c->children.fetch_sub(1);
  return MS_OK;
}

}  // extern "C"
