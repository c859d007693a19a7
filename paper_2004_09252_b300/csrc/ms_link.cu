// K1 for pages that live in pinned, mapped host memory (the served forms'
// working set): every byte the kernel reads or writes crosses the host link.
// The page work is K1's (Sec. 4.4: 64 blocks per page, counter = block
// index); what differs is the launch shape.
//
// On B300 behind this host, SM-issued read-modify-write traffic to host
// memory depends first on how much of it is in flight (measured with 64
// threads per page, pages in random order):
//   - a grid of one thread per keystream block (tens of thousands of threads
//     in flight): about 7.5 GB/s each way, whatever the CTA size;
//   - 16 CTAs x 512 threads striding over the blocks, each thread loading its
//     next block while it computes the current one: about 32 GB/s each way;
//   - without that prefetch the same grid stays near 8 GB/s, and from about
//     48 CTAs x 512 threads up the rate falls back to 8 GB/s.
// And the access pattern matters once the concurrency is right: a thread
// reading its own 64-byte block as 4 x 16 bytes (a warp instruction touching
// 32 separate 16-byte pieces) fell to 8 GB/s on pages in random order over
// 1 GiB, where warp instructions of 512 contiguous bytes moved 42 GB/s at any
// grid of 8 to 32 CTAs x 512 threads.  So this kernel runs at most
// kLinkCtas CTAs, whatever the number of pages, moves whole 512-byte rows
// per warp instruction, and keeps the next step's bytes in flight.
#include <algorithm>

#include "ms_internal.h"
#include "ms_link.cuh"

namespace ms {
namespace {

constexpr int kLinkThreads = 512;   // threads per CTA (8 pages per CTA step)
constexpr unsigned kLinkCtas = 16;  // CTAs at most: the host link's best measured concurrency

struct LinkHead {
  const uint4 *key;
  unsigned int *status;
  MulConsts mc;
  uint32_t n_pages;
};

// Entries in device memory.
struct DevEntries {
  LinkHead h;
  const ms_page_dom *e;
  __device__ __forceinline__ ms_page_dom get(uint32_t i) const { return e[i]; }
};

// Pages back to back from `base` (device view), ids first_id + i.
struct RangeEntries {
  LinkHead h;
  uint64_t base, first_id;
  uint32_t domain;
  __device__ __forceinline__ ms_page_dom get(uint32_t i) const {
    ms_page_dom e{};
    e.addr = base + (uint64_t)i * MS_PAGE_BYTES;
    e.page_id = first_id + i;
    e.domain = domain;
    return e;
  }
};

// Entries in the kernel parameters (a short host list: no staging copy).
template <int CAP>
struct ParamEntries {
  LinkHead h;
  ms_page_dom e[CAP];
  __device__ __forceinline__ ms_page_dom get(uint32_t i) const { return e[i]; }
};

// Unit u = (page u / 64, block u % 64); thread g takes units g, g + stride,
// ...  Units per page (64) and the stride are multiples of 32, so the 32
// lanes of a warp always hold 32 consecutive blocks of one page and take
// every branch below together.  The next step's span is loaded while the
// current step's blocks are computed.
template <int ROUNDS, typename Src>
__global__ void __launch_bounds__(kLinkThreads) k_pages_link(const __grid_constant__ Src src) {
  __shared__ uint4 sbuf[kLinkThreads / 32][128];
  const uint64_t units = (uint64_t)src.h.n_pages * 64;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= units) return;
  const uint32_t lane = threadIdx.x & 31u;
  uint4 *sb = sbuf[threadIdx.x >> 5];
  BlockSeed s;
  load_key(src.h.key, s.k);
  ms_page_dom e = src.get((uint32_t)(u / 64));
  bool ok = entry_ok(e.addr);
  uint4 *span = ok ? span_of(e.addr, u) : nullptr;
  uint4 blk[4] = {};
  if (ok) {
    uint4 row[4];
    load_span(row, span, lane);
    rows_to_block(sb, row, blk, lane);
  }
  for (;;) {
    const uint64_t un = u + stride;
    ms_page_dom en{};
    bool okn = false;
    uint4 *spann = nullptr;
    uint4 nrow[4] = {};
    if (un < units) {  // the next span is in flight while this one is computed
      en = src.get((uint32_t)(un / 64));
      okn = entry_ok(en.addr);
      if (okn) {
        spann = span_of(en.addr, un);
        load_span(nrow, spann, lane);
      }
    }
    const uint32_t t = (uint32_t)(u % 64);
    if (ok) {
      s.n0 = (uint32_t)e.page_id;
      s.n1 = (uint32_t)(e.page_id >> 32);
      s.n2 = e.domain;
      xor_keystream<ROUNDS>(blk, s, t, src.h.mc);
      store_block(sb, blk, span, lane);
    } else if (t == 0) {
      atomicOr(src.h.status, kStatusBadEntry);
    }
    if (un >= units) break;
    u = un;
    e = en;
    ok = okn;
    span = spann;
    if (ok) rows_to_block(sb, nrow, blk, lane);
  }
}

LinkHead make_head(const ms_ctx *c, size_t n) {
  LinkHead h;
  h.key = c->d_key;
  h.status = c->d_status;
  h.mc.m12 = 1u << 12;
  h.mc.m7 = 1u << 7;
  h.n_pages = (uint32_t)n;
  return h;
}

unsigned link_grid(size_t n) {
  const uint64_t ctas = ((uint64_t)n * 64 + kLinkThreads - 1) / kLinkThreads;
  return (unsigned)std::min<uint64_t>(ctas, kLinkCtas);
}

template <typename Src>
cudaError_t launch_src(const ms_ctx *c, const Src &src, size_t n, cudaStream_t s) {
  const unsigned grid = link_grid(n);
  switch (c->cfg.rounds) {
    case 20: k_pages_link<20, Src><<<grid, kLinkThreads, 0, s>>>(src); break;
    case 12: k_pages_link<12, Src><<<grid, kLinkThreads, 0, s>>>(src); break;
    case 8: k_pages_link<8, Src><<<grid, kLinkThreads, 0, s>>>(src); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int CAP>
cudaError_t launch_params(const ms_ctx *c, const ms_page_dom *pages, size_t n, cudaStream_t s) {
  static_assert(sizeof(ParamEntries<CAP>) <= 16448, "parameter block above 16 KB");
  ParamEntries<CAP> p;
  p.h = make_head(c, n);
  std::copy(pages, pages + n, p.e);
  return launch_src(c, p, n, s);
}

}  // namespace

size_t link_param_max_pages() { return 512; }

cudaError_t launch_pages_link(const ms_ctx *c, const ms_page_dom *pages, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (n > link_param_max_pages()) return cudaErrorInvalidValue;
  const cudaError_t f = injected(MS_FAULT_LAUNCH);
  if (f != cudaSuccess) return f;
  if (n <= 16) return launch_params<16>(c, pages, n, s);
  if (n <= 128) return launch_params<128>(c, pages, n, s);
  return launch_params<512>(c, pages, n, s);
}

cudaError_t launch_pages_link_dev(const ms_ctx *c, const ms_page_dom *d_pages, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (n > UINT32_MAX) return cudaErrorInvalidValue;
  const cudaError_t f = injected(MS_FAULT_LAUNCH);
  if (f != cudaSuccess) return f;
  DevEntries d;
  d.h = make_head(c, n);
  d.e = d_pages;
  return launch_src(c, d, n, s);
}

}  // namespace ms

using namespace ms;

extern "C" int ms_crypt_host_inplace(ms_ctx *c, int op, void *host_base, uint64_t first_page_id,
                                     size_t n_pages) {
  if (!c || !c->alive) return MS_ENOTINIT;
  if (op != MS_ENCRYPT && op != MS_DECRYPT) return MS_EINVAL;
  if (n_pages == 0) return MS_OK;
  if (!host_base || ((uintptr_t)host_base & 15u)) return MS_EINVAL;
  if (n_pages - 1 > ~first_page_id) return MS_EINVAL;  // ids must not wrap past 2^64 - 1
  if (n_pages > UINT32_MAX) return MS_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  void *dev = nullptr;
  if (cudaHostGetDevicePointer(&dev, host_base, 0) != cudaSuccess || !dev) {
    cudaGetLastError();
    return MS_EINVAL;  // not pinned, mapped host memory
  }
  cudaError_t e = injected(MS_FAULT_LAUNCH);
  if (e == cudaSuccess) {
    RangeEntries r;
    r.h = make_head(c, n_pages);
    r.base = (uint64_t)dev;
    r.first_id = first_page_id;
    r.domain = c->cfg.domain;
    e = launch_src(c, r, n_pages, c->stream);
  }
  return e == cudaSuccess ? MS_OK : cuda_fail(c, e);
}
