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

// Launch shape of the page kernels; picked by the autotuner or set in ms_config.
struct Tune {
  int bpt = 1;       // keystream blocks per thread
  int tpc = 256;     // threads per CTA
  int unr = 10;      // double rounds per loop trip
  int pol = kRotPerm;
};

constexpr int kListSlots = 4;
constexpr int kMaxHostStreams = 4;

struct ListSlot {
  ms_page *h = nullptr;  // pinned copy of a host entry list
  ms_page *d = nullptr;  // device copy read by the kernel
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
  unsigned int *h_status = nullptr;  // pinned landing word for ms_sync
  cudaEvent_t sync_ev = nullptr;
  ms::Tune tune;
  ms::ListSlot slots[ms::kListSlots];
  int next_slot = 0;
  // host streaming (ms_crypt_host)
  cudaStream_t hs[ms::kMaxHostStreams] = {};
  cudaEvent_t hs_ev[ms::kMaxHostStreams] = {};
  void *hs_buf[ms::kMaxHostStreams] = {};
  size_t hs_cap = 0;
  std::mutex mu;
  std::atomic<int> last_cuda{0};
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

int cuda_fail(ms_ctx *c, cudaError_t e);
int wait_event(ms_ctx *c, cudaEvent_t ev, uint32_t timeout_ms);
PageArgs make_args(const ms_ctx *c);
// Launch K1 with the context's tuned shape (list mode when a.pages != nullptr).
cudaError_t launch_pages(const ms_ctx *c, const PageArgs &a, cudaStream_t s);
cudaError_t launch_pages_shape(const PageArgs &a, int rounds, const Tune &t, bool range,
                               cudaStream_t s);
bool shape_available(int rounds, const Tune &t);

}  // namespace ms
