// Device helpers for page work over the host link (pinned, mapped host
// memory): a warp moves 32 consecutive keystream blocks (2 KiB) of a page
// as whole 512-byte rows and swaps them through shared memory so that each
// lane computes one block.  Used by the bounded-grid page kernel and by the
// resident workers.
#pragma once

#include "ms_cipher.cuh"

namespace ms {

// The keystream block `counter` XORed into the 64 bytes `d` (in registers).
// The same block function as xor_block in the cipher header, without its
// loads and stores: here those go through the warp's transpose below.
template <int ROUNDS>
__device__ __forceinline__ void xor_keystream(uint4 (&d)[4], const BlockSeed &s, uint32_t counter,
                                              const MulConsts &mc) {
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
}

// A warp works on 32 consecutive keystream blocks (2 KiB) of one page per
// step.  It moves them over the host link as 4 loads (and 4 stores) of 512
// contiguous bytes -- lane l takes 16-byte slot 32 k + l of the span -- and
// swaps them through 2 KiB of shared memory so that lane l holds block l
// (slots 4 l .. 4 l + 3).  Slot i is kept at i ^ ((i >> 3) & 3), which makes
// both the row pattern (32 k + l) and the block pattern (4 l + j) free of
// bank conflicts (each quarter-warp phase touches 8 distinct 16-byte banks).
__device__ __forceinline__ uint32_t swz(uint32_t i) { return i ^ ((i >> 3) & 3u); }

__device__ __forceinline__ uint4 *span_of(uint64_t addr, uint64_t u) {
  return reinterpret_cast<uint4 *>(addr) + ((u % 64) & ~31ull) * 4;
}

__device__ __forceinline__ void load_span(uint4 (&row)[4], const uint4 *span, uint32_t lane) {
#pragma unroll
  for (int k = 0; k < 4; ++k) row[k] = __ldcs(span + 32 * k + lane);
}

__device__ __forceinline__ void rows_to_block(uint4 *sb, const uint4 (&row)[4], uint4 (&blk)[4], uint32_t lane) {
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 4; ++k) sb[swz(32 * k + lane)] = row[k];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 4; ++j) blk[j] = sb[swz(4 * lane + j)];
}

__device__ __forceinline__ void store_block(uint4 *sb, const uint4 (&blk)[4], uint4 *span, uint32_t lane) {
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 4; ++j) sb[swz(4 * lane + j)] = blk[j];
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 4; ++k) __stcs(span + 32 * k + lane, sb[swz(32 * k + lane)]);
}

}  // namespace ms
