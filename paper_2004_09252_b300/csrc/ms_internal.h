// Host-side state shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <mutex>

#include "memshield.h"
#include "ms_cipher.cuh"

namespace ms {

// Status-word bits beyond kStatusBadEntry (1).
constexpr unsigned kStatusFeedTimeout = 2u;  // a fed kernel gave up waiting for entries

// Launch shape of the page kernels; picked by the autotuner or set in ms_config.
// The default is the fastest shape measured on B300 for the 1 GiB bulk
// configuration (1852 GB/s): 4 blocks per thread, 128 threads, full unroll,
// byte-permute rotations, shared prelude with the next block's bytes loaded
// while the current one is computed.
struct Tune {
  int bpt = 4;       // keystream blocks per thread
  int tpc = 128;     // threads per CTA
  int unr = 10;      // double rounds per loop trip
  int pol = kRotPerm;
  int hoist = 1;     // counter-free prelude once per page per thread (needs bpt >= 2)
};

// Launch parameters of the persistent queue kernel (K2).
struct QTune {
  int grab = 8;         // pages a CTA claims per atomic on the queue head
  int ctas_per_sm = 0;  // 0 = as many as fit (occupancy)
};

constexpr int kListSlots = 4;
constexpr int kTickets = MS_TICKETS;  // completion events of ms_submit_host, reused in a ring
constexpr int kMaxHostStreams = 4;

struct ListSlot {
  void *h = nullptr;  // pinned copy of a host entry list (room for list_capacity ms_page_dom)
  void *d = nullptr;  // device copy read by the kernel
  cudaEvent_t done = nullptr;
  bool used = false;
};

}  // namespace ms

struct ms_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  ms_config cfg{};
  int sm_count = 0;
  uint4 *d_key = nullptr;          // the 32-byte key, device memory only
  unsigned int *d_status = nullptr;
  unsigned int *h_status = nullptr;  // pinned, mapped landing word for ms_sync
  unsigned int *h_status_dev = nullptr;  // its device address
  cudaEvent_t sync_ev = nullptr;
  cudaEvent_t status_ev = nullptr;   // the status-word read of ms_sync
  bool status_pending = false;       // that read was queued but not yet collected
  unsigned status_acc = 0;           // status bits collected by a call that then timed out
  bool status_dirty = false;         // a device-list launch since the last status read: only
                                     // those can set a status bit (every other entry is checked
                                     // on the host or built by the library)
  ms::Tune tune;
  bool shape_explicit = false;  // set by the caller (config, ms_set_shape): never adapted
  ms::QTune qtune;
  std::atomic<unsigned> tune_gen{0};  // bumped whenever tune/qtune change
  ms::ListSlot slots[ms::kListSlots];
  int next_slot = 0;
  cudaEvent_t tk_ev[ms::kTickets] = {};  // created on first use
  std::atomic<uint64_t> tk_next{0};      // the next ticket (read without the lock by ms_poll)
  // host streaming (ms_crypt_host)
  cudaStream_t hs[ms::kMaxHostStreams] = {};
  cudaEvent_t hs_ev[ms::kMaxHostStreams] = {};
  void *hs_buf[ms::kMaxHostStreams] = {};
  size_t hs_cap = 0;
  std::mutex mu;
  std::atomic<int> last_cuda{0};
  std::atomic<int> children{0};  // live batches, servers and resident worker sets on this context
  bool alive = false;
};

namespace ms {

// Makes the context's device current for the scope, restoring the caller's.
class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev_);
    if (prev_ != dev) cudaSetDevice(dev);
    dev_ = dev;
  }
  ~DeviceGuard() {
    if (prev_ != dev_) cudaSetDevice(prev_);
  }

 private:
  int prev_ = 0, dev_ = 0;
};

// Records a CUDA error on the context (ms_last_cuda_error), clears the
// runtime's last-error state and returns MS_ECUDA.
int cuda_fail(ms_ctx *c, cudaError_t e);
// Allocation failure: MS_ENOMEM for out of memory (state cleared), else cuda_fail.
int alloc_fail(ms_ctx *c, cudaError_t e);

// Host-side fault injection (tests): returns the injected error when the
// armed countdown reaches zero at a site in the armed mask, else cudaSuccess.
cudaError_t injected(int site);
int wait_event(ms_ctx *c, cudaEvent_t ev, uint32_t timeout_ms);
PageArgs make_args(const ms_ctx *c);
// Launch K1 with the context's tuned shape (list mode when a.pages != nullptr).
cudaError_t launch_pages(const ms_ctx *c, const PageArgs &a, cudaStream_t s);
cudaError_t launch_pages_shape(const PageArgs &a, int rounds, const Tune &t, bool range,
                               cudaStream_t s);
bool shape_available(int rounds, const Tune &t);
// K1 with a short host entry list carried in the kernel parameters (no
// staging copy); n <= inline_max_pages<E>() (1024 ms_page, 512 ms_page_dom).
template <typename E>
size_t inline_max_pages();
template <typename E>
cudaError_t launch_pages_inline(const ms_ctx *c, const E *pages, size_t n, cudaStream_t s);
// K1 for pages in pinned, mapped host memory (every access crosses the host
// link): a bounded grid striding over the pages' blocks, the next block
// loaded while the current one is computed.  launch_pages_link carries the
// entries in the kernel parameters (n <= link_param_max_pages() = 512);
// launch_pages_link_dev reads them from device memory.
size_t link_param_max_pages();
cudaError_t launch_pages_link(const ms_ctx *c, const ms_page_dom *pages, size_t n, cudaStream_t s);
cudaError_t launch_pages_link_dev(const ms_ctx *c, const ms_page_dom *d_pages, size_t n, cudaStream_t s);
int k1_shape_count();
void k1_shape(int i, int *rounds, Tune *t);

// K2: the persistent queue kernel.  `t` picks the instance (the nearest
// compiled one when t itself is not compiled for K2).
struct QueueKernel {
  const void *fn = nullptr;  // kernel symbol, for occupancy queries and graph capture
  cudaError_t (*launch)(const QueueArgs &, int grid, int tpc, cudaStream_t) = nullptr;
  Tune shape;                // the instance actually used
};
bool queue_kernel(int rounds, const Tune &t, QueueKernel *out);
int queue_grid(const ms_ctx *c, const QueueKernel &k, int tpc, int ctas_per_sm);

}  // namespace ms
