// K2 variant table: compiled instances of the persistent queue kernel.
#include "ms_internal.h"

namespace ms {
namespace {

template <int R, int B, int U, int P, bool H>
cudaError_t launch_k2(const QueueArgs &q, int grid, int tpc, cudaStream_t s) {
  if (q.ditems)
    k_queue<R, B, U, P, H, true><<<grid, tpc, 0, s>>>(q);
  else
    k_queue<R, B, U, P, H, false><<<grid, tpc, 0, s>>>(q);
  return cudaGetLastError();
}

struct Entry {
  int rounds, bpt, unr, pol, hoist;
  const void *fn;
  cudaError_t (*launch)(const QueueArgs &, int, int, cudaStream_t);
};

#define MS_K2(R, B, U, P) {R, B, U, P, 0, (const void *)&k_queue<R, B, U, P, false>, &launch_k2<R, B, U, P, false>}
#define MS_K2H(R, B, P) {R, B, R / 2, P, 1, (const void *)&k_queue<R, B, R / 2, P, true>, \
                         &launch_k2<R, B, R / 2, P, true>}

const Entry kTable[] = {
    MS_K2(20, 1, 10, 1), MS_K2(20, 2, 10, 1), MS_K2(20, 4, 10, 1),
    MS_K2(20, 1, 2, 1),  MS_K2(20, 2, 2, 1),  MS_K2(20, 4, 2, 1),
    MS_K2(20, 1, 10, 0), MS_K2(20, 2, 10, 0), MS_K2(20, 4, 10, 0),
    MS_K2(12, 1, 6, 1),  MS_K2(12, 2, 6, 1),  MS_K2(12, 4, 6, 1),
    MS_K2(8, 1, 4, 1),   MS_K2(8, 2, 4, 1),   MS_K2(8, 4, 4, 1),
    MS_K2H(20, 2, 1), MS_K2H(20, 4, 1), MS_K2H(12, 2, 1), MS_K2H(12, 4, 1), MS_K2H(8, 2, 1), MS_K2H(8, 4, 1),
};

#undef MS_K2

}  // namespace

bool queue_kernel(int rounds, const Tune &t, QueueKernel *out) {
  const Entry *best = nullptr;
  int best_score = -1;
  for (const Entry &e : kTable) {
    if (e.rounds != rounds) continue;
    // prefer the exact shape, then the same blocks-per-thread, then the same unroll
    int score = (e.bpt == t.bpt) * 8 + (e.hoist == t.hoist) * 4 + (e.unr == t.unr) * 2 + (e.pol == t.pol);
    if (score > best_score) {
      best_score = score;
      best = &e;
    }
  }
  if (!best) return false;
  out->fn = best->fn;
  out->launch = best->launch;
  out->shape.bpt = best->bpt;
  out->shape.unr = best->unr;
  out->shape.pol = best->pol;
  out->shape.hoist = best->hoist;
  out->shape.tpc = t.tpc;
  return true;
}

int queue_grid(const ms_ctx *c, const QueueKernel &k, int tpc, int ctas_per_sm) {
  int fit = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k.fn, tpc, 0) != cudaSuccess || fit < 1) fit = 1;
  const int per_sm = (ctas_per_sm > 0 && ctas_per_sm < fit) ? ctas_per_sm : fit;
  return per_sm * c->sm_count;
}

}  // namespace ms
