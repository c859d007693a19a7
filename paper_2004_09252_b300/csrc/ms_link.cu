// K1 for pages that live in pinned, mapped host memory (the served forms'
// working set): every byte the kernel reads or writes crosses the host link.
// The page work is K1's (Sec. 4.4: 64 blocks per page, counter = block
// index); what differs is the launch shape.
//
// On B300 behind this host, SM-issued read-modify-write traffic to host
// memory depends on how much of it is in flight, not on the access pattern
// (measured with 64 threads per page, pages in random order):
//   - a grid of one thread per keystream block (tens of thousands of threads
//     in flight): about 7.5 GB/s each way, whatever the CTA size;
//   - 16 CTAs x 512 threads striding over the blocks, each thread loading its
//     next block while it computes the current one: about 32 GB/s each way;
//   - without that prefetch the same grid stays near 8 GB/s, and from about
//     48 CTAs x 512 threads up the rate falls back to 8 GB/s.
// So this kernel runs at most kLinkCtas CTAs, whatever the number of pages,
// and keeps two blocks per thread in flight.
#include <algorithm>

#include "ms_internal.h"

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

// Entries in the kernel parameters (a short host list: no staging copy).
template <int CAP>
struct ParamEntries {
  LinkHead h;
  ms_page_dom e[CAP];
  __device__ __forceinline__ ms_page_dom get(uint32_t i) const { return e[i]; }
};

// The keystream block `counter` XORed into the 64 bytes `d` already loaded
// from dst, then stored back.  The same block function as xor_block in the
// cipher header, minus the loads (they were issued one step earlier).
template <int ROUNDS>
__device__ __forceinline__ void xor_loaded(uint4 *__restrict__ dst, uint4 (&d)[4], const BlockSeed &s,
                                           uint32_t counter, const MulConsts &mc) {
  uint32_t x0 = kSigma0, x1 = kSigma1, x2 = kSigma2, x3 = kSigma3;
  uint32_t x4 = s.k[0], x5 = s.k[1], x6 = s.k[2], x7 = s.k[3];
  uint32_t x8 = s.k[4], x9 = s.k[5], x10 = s.k[6], x11 = s.k[7];
  uint32_t x12 = counter, x13 = s.n0, x14 = s.n1, x15 = s.n2;
#pragma unroll
  for (int r = 0; r < ROUNDS / 2; ++r) {
    quarter_round<kRotPerm, true>(x0, x4, x8, x12, mc);
    quarter_round<kRotPerm, true>(x1, x5, x9, x13, mc);
    quarter_round<kRotPerm, true>(x2, x6, x10, x14, mc);
    quarter_round<kRotPerm, true>(x3, x7, x11, x15, mc);
    quarter_round<kRotPerm, false>(x0, x5, x10, x15, mc);
    quarter_round<kRotPerm, false>(x1, x6, x11, x12, mc);
    quarter_round<kRotPerm, false>(x2, x7, x8, x13, mc);
    quarter_round<kRotPerm, false>(x3, x4, x9, x14, mc);
  }
  d[0].x ^= x0 + kSigma0;  d[0].y ^= x1 + kSigma1;  d[0].z ^= x2 + kSigma2;  d[0].w ^= x3 + kSigma3;
  d[1].x ^= x4 + s.k[0];   d[1].y ^= x5 + s.k[1];   d[1].z ^= x6 + s.k[2];   d[1].w ^= x7 + s.k[3];
  d[2].x ^= x8 + s.k[4];   d[2].y ^= x9 + s.k[5];   d[2].z ^= x10 + s.k[6];  d[2].w ^= x11 + s.k[7];
  d[3].x ^= x12 + counter; d[3].y ^= x13 + s.n0;    d[3].z ^= x14 + s.n1;    d[3].w ^= x15 + s.n2;
  __stcs(dst + 0, d[0]); __stcs(dst + 1, d[1]); __stcs(dst + 2, d[2]); __stcs(dst + 3, d[3]);
}

__device__ __forceinline__ void load_unit(uint4 (&d)[4], uint64_t addr, uint32_t t) {
  const uint4 *p = reinterpret_cast<const uint4 *>(addr) + 4 * t;
  d[0] = __ldcs(p); d[1] = __ldcs(p + 1); d[2] = __ldcs(p + 2); d[3] = __ldcs(p + 3);
}

// Unit u = (page u / 64, block u % 64); thread g takes units g, g + stride,
// ..., so at each step the 32 lanes of a warp work on 32 consecutive blocks
// (2 KiB) of one page.
template <int ROUNDS, typename Src>
__global__ void __launch_bounds__(kLinkThreads) k_pages_link(const __grid_constant__ Src src) {
  const uint64_t units = (uint64_t)src.h.n_pages * 64;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= units) return;
  BlockSeed s;
  load_key(src.h.key, s.k);
  ms_page_dom e = src.get((uint32_t)(u / 64));
  bool ok = entry_ok(e.addr);
  uint4 cur[4] = {};
  if (ok) load_unit(cur, e.addr, (uint32_t)(u % 64));
  for (;;) {
    const uint64_t un = u + stride;
    ms_page_dom en{};
    bool okn = false;
    uint4 nxt[4] = {};
    if (un < units) {  // the next unit's bytes are in flight while this one is computed
      en = src.get((uint32_t)(un / 64));
      okn = entry_ok(en.addr);
      if (okn) load_unit(nxt, en.addr, (uint32_t)(un % 64));
    }
    const uint32_t t = (uint32_t)(u % 64);
    if (ok) {
      s.n0 = (uint32_t)e.page_id;
      s.n1 = (uint32_t)(e.page_id >> 32);
      s.n2 = e.domain;
      xor_loaded<ROUNDS>(reinterpret_cast<uint4 *>(e.addr) + 4 * t, cur, s, t, src.h.mc);
    } else if (t == 0) {
      atomicOr(src.h.status, kStatusBadEntry);
    }
    if (un >= units) break;
    u = un;
    e = en;
    ok = okn;
    cur[0] = nxt[0]; cur[1] = nxt[1]; cur[2] = nxt[2]; cur[3] = nxt[3];
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
