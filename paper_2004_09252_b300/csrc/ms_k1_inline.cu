// K1 for short host entry lists: the entries travel in the kernel's
// parameter space (up to 32 KB of parameters per launch on this
// architecture), so a small request needs no pinned staging copy, no
// host-to-device copy and no event: one launch.  The page work is K1's
// (Sec. 4.4: 64 blocks per page, counter = block index), in the shape the
// one-launch form uses for launches too small to fill the GPU: one block per
// thread, 128 threads per CTA, byte-permute rotations.
#include <cstring>
#include <type_traits>

#include "ms_internal.h"

namespace ms {
namespace {

struct InlineHead {
  const uint4 *key;
  unsigned int *status;
  MulConsts mc;
  uint32_t domain;    // nonce word 15 for ms_page entries
  uint32_t n_pages;
};

template <typename E, int CAP>
struct InlineArgs {
  InlineHead h;
  E e[CAP];
};

template <int ROUNDS, typename E, int CAP>
__global__ void __launch_bounds__(128) k_pages_inline(const __grid_constant__ InlineArgs<E, CAP> p) {
  constexpr uint32_t TPP = 64;  // one keystream block per thread
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t page = g / TPP;
  if (page >= p.h.n_pages) return;
  const uint32_t t = g % TPP;
  const uint64_t addr = p.e[page].addr, pid = p.e[page].page_id;
  uint32_t domain = p.h.domain;
  if constexpr (std::is_same<E, ms_page_dom>::value) domain = p.e[page].domain;
  if (!entry_ok(addr)) {
    if (t == 0) atomicOr(p.h.status, kStatusBadEntry);
    return;
  }
  BlockSeed s;
  load_key(p.h.key, s.k);
  s.n0 = (uint32_t)pid;
  s.n1 = (uint32_t)(pid >> 32);
  s.n2 = domain;
  page_blocks<ROUNDS, 1, ROUNDS / 2, kRotPerm, false>(reinterpret_cast<uint4 *>(addr), s, t, TPP, p.h.mc);
}

// The smallest parameter block that holds n entries; 16 KB at most.
template <int ROUNDS, typename E, int CAP>
cudaError_t launch_cap(const ms_ctx *c, const E *pages, size_t n, cudaStream_t s) {
  static_assert(sizeof(InlineArgs<E, CAP>) <= 16448, "parameter block above 16 KB");
  InlineArgs<E, CAP> p;
  p.h.key = c->d_key;
  p.h.status = c->d_status;
  p.h.mc.m12 = 1u << 12;
  p.h.mc.m7 = 1u << 7;
  p.h.domain = c->cfg.domain;
  p.h.n_pages = (uint32_t)n;
  std::memcpy(p.e, pages, n * sizeof(E));
  const unsigned grid = (unsigned)((n * 64 + 127) / 128);
  k_pages_inline<ROUNDS, E, CAP><<<grid, 128, 0, s>>>(p);
  return cudaGetLastError();
}

template <int ROUNDS, typename E>
cudaError_t launch_rounds(const ms_ctx *c, const E *pages, size_t n, cudaStream_t s) {
  constexpr int kMax = (int)(16384 / sizeof(E));  // 1024 ms_page or 512 ms_page_dom
  if (n <= 16) return launch_cap<ROUNDS, E, 16>(c, pages, n, s);
  if (n <= 128) return launch_cap<ROUNDS, E, 128>(c, pages, n, s);
  return launch_cap<ROUNDS, E, kMax>(c, pages, n, s);
}

}  // namespace

template <typename E>
size_t inline_max_pages() {
  return 16384 / sizeof(E);
}
template size_t inline_max_pages<ms_page>();
template size_t inline_max_pages<ms_page_dom>();

template <typename E>
cudaError_t launch_pages_inline(const ms_ctx *c, const E *pages, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (n > inline_max_pages<E>()) return cudaErrorInvalidValue;
  const cudaError_t f = injected(MS_FAULT_LAUNCH);
  if (f != cudaSuccess) return f;
  switch (c->cfg.rounds) {
    case 20: return launch_rounds<20>(c, pages, n, s);
    case 12: return launch_rounds<12>(c, pages, n, s);
    case 8: return launch_rounds<8>(c, pages, n, s);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_pages_inline<ms_page>(const ms_ctx *, const ms_page *, size_t, cudaStream_t);
template cudaError_t launch_pages_inline<ms_page_dom>(const ms_ctx *, const ms_page_dom *, size_t, cudaStream_t);

}  // namespace ms
