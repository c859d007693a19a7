// Device side of the page cipher: the ChaCha20 block held in registers and the
// page kernels built on it.
//
// Method (MemShield Sec. 4.4): a 4096-byte page is XORed in place with the 64
// keystream blocks whose 128-bit seed value is (block index j = 0..63, page
// id, domain); the 256-bit key sits in device memory.  Each thread makes one
// 64-byte keystream block at a time and XORs it into the same 64 bytes of the
// page, so a block never leaves the thread's registers.  ChaCha20 block: the
// 16-word state (four constant words, eight key words, the counter, three
// nonce words) goes through 10 double rounds, each four column
// quarter-rounds and four diagonal quarter-rounds, and the input state is
// then added back word by word.
#pragma once

#include <cstdint>

#include "memshield.h"

namespace ms {

// ASCII "expand 32-byte k" as four little-endian 32-bit words.
constexpr uint32_t kSigma0 = 0x61707865u;  // "expa"
constexpr uint32_t kSigma1 = 0x3320646eu;  // "nd 3"
constexpr uint32_t kSigma2 = 0x79622d32u;  // "2-by"
constexpr uint32_t kSigma3 = 0x6b206574u;  // "te k"

constexpr unsigned kStatusBadEntry = 1u;   // a device-side entry check failed

// Rotation policies.  All compute the same left rotation; they differ in the
// execution pipe each rotation lands on.  LOP3 (xor), funnel shifts and byte
// permutes share the integer ALU pipe, which bounds this kernel; adds already
// go to the multiply-add pipe, so the policies move some rotations there.
//   kRotFunnel  every rotation is a funnel shift
//   kRotPerm    rotations by 16 and 8 are byte permutes, 12 and 7 funnel shifts
//   kRotMul     as kRotPerm, 12 and 7 as (x * 2^k).hi + (x * 2^k).lo
//   kRotMul7    as kRotPerm, only the rotations by 7 through the multiplier
//   kRotMul12   as kRotPerm, only the rotations by 12 through the multiplier
//   kRotMul7Col as kRotPerm, rotations by 7 of the column rounds only
//   kRotWide7   as kRotMul7, with one 32x32->64 multiply and an add
//   kRotMulCol  as kRotPerm, rotations by 12 and 7 of the column rounds only
// The multipliers 2^k come from a kernel argument, so the compiler keeps them
// as real multiplies instead of folding them back into shifts.
enum RotPolicy {
  kRotFunnel = 0, kRotPerm = 1, kRotMul = 2, kRotMul7 = 3, kRotMul12 = 4,
  kRotMul7Col = 5, kRotWide7 = 6, kRotMulCol = 7
};

struct MulConsts {
  uint32_t m12;  // 1 << 12
  uint32_t m7;   // 1 << 7
};

template <int N>
__device__ __forceinline__ uint32_t rotl_funnel(uint32_t x) {
  return __funnelshift_l(x, x, N);
}

template <int POL>
__device__ __forceinline__ uint32_t rotl16(uint32_t x) {
  if (POL == kRotFunnel) return rotl_funnel<16>(x);
  return __byte_perm(x, 0u, 0x1032u);
}

template <int POL>
__device__ __forceinline__ uint32_t rotl8(uint32_t x) {
  if (POL == kRotFunnel) return rotl_funnel<8>(x);
  return __byte_perm(x, 0u, 0x2103u);
}

// x * 2^k as a 64-bit product: low word = x << k, high word = x >> (32 - k);
// the two never overlap, so their sum is the rotation.
__device__ __forceinline__ uint32_t rotl_mul(uint32_t x, uint32_t m) {
  uint32_t hi = __umulhi(x, m);
  uint32_t r;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(m), "r"(hi));
  return r;
}

__device__ __forceinline__ uint32_t rotl_wide(uint32_t x, uint32_t m) {
  uint64_t p;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(x), "r"(m));
  return (uint32_t)p + (uint32_t)(p >> 32);
}

template <int POL, bool COL>
__device__ __forceinline__ uint32_t rotl12(uint32_t x, const MulConsts &mc) {
  if (POL == kRotMul || POL == kRotMul12 || (POL == kRotMulCol && COL)) return rotl_mul(x, mc.m12);
  return rotl_funnel<12>(x);
}

template <int POL, bool COL>
__device__ __forceinline__ uint32_t rotl7(uint32_t x, const MulConsts &mc) {
  if (POL == kRotMul || POL == kRotMul7 || ((POL == kRotMul7Col || POL == kRotMulCol) && COL))
    return rotl_mul(x, mc.m7);
  if (POL == kRotWide7) return rotl_wide(x, mc.m7);
  return rotl_funnel<7>(x);
}

// COL: the quarter round belongs to a column round (else a diagonal round).
template <int POL, bool COL>
__device__ __forceinline__ void quarter_round(uint32_t &a, uint32_t &b, uint32_t &c, uint32_t &d,
                                              const MulConsts &mc) {
  a += b; d = rotl16<POL>(d ^ a);
  c += d; b = rotl12<POL, COL>(b ^ c, mc);
  a += b; d = rotl8<POL>(d ^ a);
  c += d; b = rotl7<POL, COL>(b ^ c, mc);
}

// Key words 0..7 and the per-page nonce words (13, 14, 15).
struct BlockSeed {
  uint32_t k[8];
  uint32_t n0, n1, n2;
};

__device__ __forceinline__ void load_key(const uint4 *__restrict__ key, uint32_t (&k)[8]) {
  const uint4 a = __ldg(key), b = __ldg(key + 1);
  k[0] = a.x; k[1] = a.y; k[2] = a.z; k[3] = a.w;
  k[4] = b.x; k[5] = b.y; k[6] = b.z; k[7] = b.w;
}

// Keystream block `counter` for `seed`, XORed into the 64 bytes at dst.
// ROUNDS is 8, 12 or 20; UNR is how many double rounds one loop trip holds.
template <int ROUNDS, int UNR, int POL>
__device__ __forceinline__ void xor_block(uint4 *__restrict__ dst, const BlockSeed &s,
                                          uint32_t counter, const MulConsts &mc) {
  // Issue the page loads first so their latency hides behind the rounds.
  uint4 d0 = __ldcs(dst + 0), d1 = __ldcs(dst + 1), d2 = __ldcs(dst + 2), d3 = __ldcs(dst + 3);

  uint32_t x0 = kSigma0, x1 = kSigma1, x2 = kSigma2, x3 = kSigma3;
  uint32_t x4 = s.k[0], x5 = s.k[1], x6 = s.k[2], x7 = s.k[3];
  uint32_t x8 = s.k[4], x9 = s.k[5], x10 = s.k[6], x11 = s.k[7];
  uint32_t x12 = counter, x13 = s.n0, x14 = s.n1, x15 = s.n2;

  static_assert((ROUNDS / 2) % UNR == 0, "unroll must divide the double-round count");
#pragma unroll 1
  for (int r = 0; r < ROUNDS / 2; r += UNR) {
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      // column round
      quarter_round<POL, true>(x0, x4, x8, x12, mc);
      quarter_round<POL, true>(x1, x5, x9, x13, mc);
      quarter_round<POL, true>(x2, x6, x10, x14, mc);
      quarter_round<POL, true>(x3, x7, x11, x15, mc);
      // diagonal round
      quarter_round<POL, false>(x0, x5, x10, x15, mc);
      quarter_round<POL, false>(x1, x6, x11, x12, mc);
      quarter_round<POL, false>(x2, x7, x8, x13, mc);
      quarter_round<POL, false>(x3, x4, x9, x14, mc);
    }
  }

  // Feed-forward (add the input state), then XOR; words are little-endian in
  // memory, which is the byte order of the uint4 lanes on the GPU.
  d0.x ^= x0 + kSigma0;  d0.y ^= x1 + kSigma1;  d0.z ^= x2 + kSigma2;  d0.w ^= x3 + kSigma3;
  d1.x ^= x4 + s.k[0];   d1.y ^= x5 + s.k[1];   d1.z ^= x6 + s.k[2];   d1.w ^= x7 + s.k[3];
  d2.x ^= x8 + s.k[4];   d2.y ^= x9 + s.k[5];   d2.z ^= x10 + s.k[6];  d2.w ^= x11 + s.k[7];
  d3.x ^= x12 + counter; d3.y ^= x13 + s.n0;    d3.z ^= x14 + s.n1;    d3.w ^= x15 + s.n2;
  __stcs(dst + 0, d0); __stcs(dst + 1, d1); __stcs(dst + 2, d2); __stcs(dst + 3, d3);
}

// The part of the first double round that is the same for all 64 blocks of a
// page.  Only word 12 (the block counter) differs between them, and in the
// first column round it enters only the quarter round on words (0, 4, 8, 12);
// the other three column quarter rounds, the first add of that one, and the
// counter-free steps of two diagonal quarter rounds depend on key and nonce
// alone (41 of the 992 operations of a block).
struct Prelude {
  uint32_t a0;                                  // x0 + x4 (first step of column QR 0)
  uint32_t x1, x2, x3, x5, x6, x7, x9, x10, x11, x13, x14, x15;  // after column QRs 1..3
  uint32_t da1;                                 // diagonal QR (1,6,11,12): a = x1 + x6
  uint32_t da2, dd2;                            // diagonal QR (2,7,8,13): a = x2 + x7, d = (x13 ^ a) <<< 16
};

template <int POL>
__device__ __forceinline__ Prelude make_prelude(const BlockSeed &s, const MulConsts &mc) {
  Prelude p;
  uint32_t x1 = kSigma1, x2 = kSigma2, x3 = kSigma3;
  uint32_t x5 = s.k[1], x6 = s.k[2], x7 = s.k[3];
  uint32_t x9 = s.k[5], x10 = s.k[6], x11 = s.k[7];
  uint32_t x13 = s.n0, x14 = s.n1, x15 = s.n2;
  quarter_round<POL, true>(x1, x5, x9, x13, mc);
  quarter_round<POL, true>(x2, x6, x10, x14, mc);
  quarter_round<POL, true>(x3, x7, x11, x15, mc);
  p.a0 = kSigma0 + s.k[0];
  p.x1 = x1; p.x2 = x2; p.x3 = x3; p.x5 = x5; p.x6 = x6; p.x7 = x7;
  p.x9 = x9; p.x10 = x10; p.x11 = x11; p.x13 = x13; p.x14 = x14; p.x15 = x15;
  p.da1 = x1 + x6;
  p.da2 = x2 + x7;
  p.dd2 = rotl16<POL>(x13 ^ p.da2);
  return p;
}

// Keystream block `counter` XORed into the 64 bytes `d` already loaded (and
// stored to dst), with the first double round started from a Prelude.  The
// remaining double rounds are fully unrolled.
template <int ROUNDS, int POL>
__device__ __forceinline__ void xor_loaded_hoisted(uint4 *__restrict__ dst, uint4 (&d)[4], const BlockSeed &s,
                                                   const Prelude &p, uint32_t counter, const MulConsts &mc) {
  uint32_t x0, x4, x8, x12;
  uint32_t x1, x2, x3, x5 = p.x5, x6, x7, x9 = p.x9, x10 = p.x10, x11, x13, x14 = p.x14, x15 = p.x15;
  {  // column QR (0, 4, 8, 12), the only one that sees the counter
    uint32_t a = p.a0, b = s.k[0], c = s.k[4], dd = counter;
    dd = rotl16<POL>(dd ^ a);
    c += dd; b = rotl12<POL, true>(b ^ c, mc);
    a += b; dd = rotl8<POL>(dd ^ a);
    c += dd; b = rotl7<POL, true>(b ^ c, mc);
    x0 = a; x4 = b; x8 = c; x12 = dd;
  }
  // diagonal round
  quarter_round<POL, false>(x0, x5, x10, x15, mc);
  {  // (1, 6, 11, 12): a = x1 + x6 precomputed
    uint32_t a = p.da1, b = p.x6, c = p.x11, dd = x12;
    dd = rotl16<POL>(dd ^ a);
    c += dd; b = rotl12<POL, false>(b ^ c, mc);
    a += b; dd = rotl8<POL>(dd ^ a);
    c += dd; b = rotl7<POL, false>(b ^ c, mc);
    x1 = a; x6 = b; x11 = c; x12 = dd;
  }
  {  // (2, 7, 8, 13): a = x2 + x7 and d = (x13 ^ a) <<< 16 precomputed
    uint32_t a = p.da2, b = p.x7, c = x8, dd = p.dd2;
    c += dd; b = rotl12<POL, false>(b ^ c, mc);
    a += b; dd = rotl8<POL>(dd ^ a);
    c += dd; b = rotl7<POL, false>(b ^ c, mc);
    x2 = a; x7 = b; x8 = c; x13 = dd;
  }
  x3 = p.x3;
  quarter_round<POL, false>(x3, x4, x9, x14, mc);
#pragma unroll
  for (int r = 1; r < ROUNDS / 2; ++r) {
    quarter_round<POL, true>(x0, x4, x8, x12, mc);
    quarter_round<POL, true>(x1, x5, x9, x13, mc);
    quarter_round<POL, true>(x2, x6, x10, x14, mc);
    quarter_round<POL, true>(x3, x7, x11, x15, mc);
    quarter_round<POL, false>(x0, x5, x10, x15, mc);
    quarter_round<POL, false>(x1, x6, x11, x12, mc);
    quarter_round<POL, false>(x2, x7, x8, x13, mc);
    quarter_round<POL, false>(x3, x4, x9, x14, mc);
  }
  d[0].x ^= x0 + kSigma0;  d[0].y ^= x1 + kSigma1;  d[0].z ^= x2 + kSigma2;  d[0].w ^= x3 + kSigma3;
  d[1].x ^= x4 + s.k[0];   d[1].y ^= x5 + s.k[1];   d[1].z ^= x6 + s.k[2];   d[1].w ^= x7 + s.k[3];
  d[2].x ^= x8 + s.k[4];   d[2].y ^= x9 + s.k[5];   d[2].z ^= x10 + s.k[6];  d[2].w ^= x11 + s.k[7];
  d[3].x ^= x12 + counter; d[3].y ^= x13 + s.n0;    d[3].z ^= x14 + s.n1;    d[3].w ^= x15 + s.n2;
  __stcs(dst + 0, d[0]); __stcs(dst + 1, d[1]); __stcs(dst + 2, d[2]); __stcs(dst + 3, d[3]);
}

// All blocks `t + b * TPP` (b < BPT) of one page for one thread; with HOIST the
// counter-free prelude is computed once for them.
template <int ROUNDS, int BPT, int UNR, int POL, bool HOIST>
__device__ __forceinline__ void page_blocks(uint4 *__restrict__ pg, const BlockSeed &s, uint32_t t, uint32_t tpp,
                                            const MulConsts &mc) {
  if (HOIST) {
    // Software pipeline: the next block's 64 bytes are loaded while the
    // current block's keystream is computed, so the loads are in flight
    // however the compiler schedules the rounds.
    uint4 cur[4], nxt[4];
    const uint4 *src = pg + 4 * t;
    cur[0] = __ldcs(src + 0); cur[1] = __ldcs(src + 1); cur[2] = __ldcs(src + 2); cur[3] = __ldcs(src + 3);
    const Prelude p = make_prelude<POL>(s, mc);
#pragma unroll 1
    for (int b = 0; b < BPT; ++b) {
      const uint32_t j = t + b * tpp;
      if (b + 1 < BPT) {
        const uint4 *nsrc = pg + 4 * (j + tpp);
        nxt[0] = __ldcs(nsrc + 0); nxt[1] = __ldcs(nsrc + 1); nxt[2] = __ldcs(nsrc + 2); nxt[3] = __ldcs(nsrc + 3);
      }
      xor_loaded_hoisted<ROUNDS, POL>(pg + 4 * j, cur, s, p, j, mc);
      cur[0] = nxt[0]; cur[1] = nxt[1]; cur[2] = nxt[2]; cur[3] = nxt[3];
    }
  } else {
#pragma unroll 1
    for (int b = 0; b < BPT; ++b) {
      const uint32_t j = t + b * tpp;
      xor_block<ROUNDS, UNR, POL>(pg + 4 * j, s, j, mc);
    }
  }
}

// How K1 finds its pages.
enum PageMode {
  kModeList = 0,     // ms_page entries; domain from the context
  kModeRange = 1,    // contiguous pages from `base`, ids first_id + k
  kModeListDom = 2,  // ms_page_dom entries, each with its own domain word
};

// Arguments shared by the page kernels.
struct PageArgs {
  const ms_page *pages;   // entry list (list mode)
  const ms_page_dom *dpages;  // entry list with domains (list-domain mode)
  uint8_t *base;          // first page (range mode)
  uint64_t first_id;      // id of the first page (range mode)
  uint64_t n_pages;
  const uint4 *key;       // 32-byte key in device memory
  uint32_t domain;        // nonce word 15
  unsigned int *status;   // device status word (kStatus* bits)
  MulConsts mc;           // multipliers for kRotMul
};

__device__ __forceinline__ bool entry_ok(uint64_t addr) { return addr != 0 && (addr & 15u) == 0; }

// K1, the one-launch bulk kernel.  Thread g works on page g / (64 / BPT) and,
// inside it, on blocks t, t + 64/BPT, ... (t = g mod 64/BPT), so at each step
// the threads of a warp touch consecutive 64-byte blocks of one page.
template <int ROUNDS, int BPT, int UNR, int POL, int MODE, bool HOIST = false>
__global__ void __launch_bounds__(512) k_pages(const PageArgs a) {
  constexpr uint32_t TPP = 64 / BPT;  // threads per page
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t page = g / TPP;
  if (page >= a.n_pages) return;
  const uint32_t t = (uint32_t)(g % TPP);

  uint64_t addr, pid;
  uint32_t domain = a.domain;
  if (MODE == kModeRange) {
    addr = (uint64_t)a.base + page * (uint64_t)MS_PAGE_BYTES;
    pid = a.first_id + page;
  } else {
    if (MODE == kModeListDom) {
      const ms_page_dom e = a.dpages[page];
      addr = e.addr;
      pid = e.page_id;
      domain = e.domain;
    } else {
      const ms_page e = a.pages[page];
      addr = e.addr;
      pid = e.page_id;
    }
    if (!entry_ok(addr)) {
      if (t == 0) atomicOr(a.status, kStatusBadEntry);
      return;
    }
  }
  BlockSeed s;
  load_key(a.key, s.k);
  s.n0 = (uint32_t)pid;
  s.n1 = (uint32_t)(pid >> 32);
  s.n2 = domain;
  page_blocks<ROUNDS, BPT, UNR, POL, HOIST>(reinterpret_cast<uint4 *>(addr), s, t, TPP, a.mc);
}

// Arguments of the persistent queue kernel.
struct QueueArgs {
  const ms_page *items;   // the device work queue: one entry per page
  const ms_page_dom *ditems;  // the same with a domain per entry (DOM instances)
  const uint32_t *count;  // number of valid entries (device word written with the items)
  uint32_t *head;         // next unclaimed entry; 0 at launch
  uint32_t grab;          // pages a CTA claims per atomic on head
  const uint4 *key;
  uint32_t domain;
  unsigned int *status;
  MulConsts mc;
};

// K2, the persistent batched kernel.  A grid sized to the resident capacity
// of the GPU drains the work queue: each CTA claims consecutive entries with
// one atomic on the queue head and processes them blockDim / TPP pages at a
// time (TPP = 64 / BPT threads per page), until the head passes the count.
// Claims are guided: `grab` entries while the queue is long, then about
// remaining / (2 * CTAs), never less than one pass, so that the CTAs run out
// of work at nearly the same time.  The head only grows, so every CTA leaves
// after at most count / pass + 1 claims; nothing waits.
template <int ROUNDS, int BPT, int UNR, int POL, bool HOIST = false, bool DOM = false>
__global__ void __launch_bounds__(512) k_queue(const QueueArgs q) {
  constexpr uint32_t TPP = 64 / BPT;
  __shared__ uint32_t s_base;
  const uint32_t n = *q.count;
  const uint32_t pages_per_pass = blockDim.x / TPP;
  const uint32_t lp = threadIdx.x / TPP;  // page slot of this thread within a pass
  const uint32_t t = threadIdx.x % TPP;
  BlockSeed s;
  load_key(q.key, s.k);
  s.n2 = q.domain;
  __shared__ uint32_t s_take;
  const uint32_t cap = max(q.grab, pages_per_pass);
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t seen = *reinterpret_cast<volatile const uint32_t *>(q.head);
      const uint32_t rem = seen < n ? n - seen : 0;
      uint32_t take = rem / (2u * gridDim.x);
      take = (take + pages_per_pass - 1) / pages_per_pass * pages_per_pass;
      take = min(max(take, pages_per_pass), cap);
      s_base = atomicAdd(q.head, take);
      s_take = take;
    }
    __syncthreads();
    const uint32_t base = s_base, take = s_take;
    __syncthreads();
    if (base >= n) break;
    const uint32_t end = base + min(take, n - base);
    for (uint32_t p = base + lp; p < end; p += pages_per_pass) {
      ms_page e;
      if (DOM) {
        const ms_page_dom ed = q.ditems[p];
        e.addr = ed.addr;
        e.page_id = ed.page_id;
        s.n2 = ed.domain;
      } else {
        e = q.items[p];
      }
      if (!entry_ok(e.addr)) {
        if (t == 0) atomicOr(q.status, kStatusBadEntry);
        continue;
      }
      s.n0 = (uint32_t)e.page_id;
      s.n1 = (uint32_t)(e.page_id >> 32);
      page_blocks<ROUNDS, BPT, UNR, POL, HOIST>(reinterpret_cast<uint4 *>(e.addr), s, t, TPP, q.mc);
    }
  }
}

}  // namespace ms
