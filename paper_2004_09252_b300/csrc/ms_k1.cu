// K1 variant table: every compiled (rounds, blocks/thread, unroll, rotation
// policy, prelude) instance of the bulk page kernel, each in its three entry
// modes (list, range, list with per-entry domain), and its launcher.
#include "ms_internal.h"

namespace ms {
namespace {

using LaunchFn = cudaError_t (*)(const PageArgs &, int, cudaStream_t);

template <int R, int B, int U, int P, int M, bool H>
cudaError_t launch_k1(const PageArgs &a, int tpc, cudaStream_t s) {
  constexpr uint64_t TPP = 64 / B;
  const uint64_t threads = a.n_pages * TPP;
  const uint64_t grid = (threads + tpc - 1) / tpc;
  if (grid > 0x7fffffffull) return cudaErrorInvalidConfiguration;
  k_pages<R, B, U, P, M, H><<<(unsigned)grid, tpc, 0, s>>>(a);
  return cudaGetLastError();
}

struct Entry {
  int rounds, bpt, unr, pol, hoist;
  LaunchFn fn[3];  // indexed by PageMode
};

#define MS_K1(R, B, U, P)                                                                          \
  {R, B, U, P, 0,                                                                                  \
   {&launch_k1<R, B, U, P, kModeList, false>, &launch_k1<R, B, U, P, kModeRange, false>,           \
    &launch_k1<R, B, U, P, kModeListDom, false>}}
// hoisted prelude; the remaining double rounds are always fully unrolled (unr = rounds / 2)
#define MS_K1H(R, B, P)                                                                            \
  {R, B, R / 2, P, 1,                                                                              \
   {&launch_k1<R, B, R / 2, P, kModeList, true>, &launch_k1<R, B, R / 2, P, kModeRange, true>,     \
    &launch_k1<R, B, R / 2, P, kModeListDom, true>}}

const Entry kTable[] = {
    // ChaCha20, the paper's cipher: the tuned search space.
    MS_K1(20, 1, 1, 0), MS_K1(20, 1, 2, 0), MS_K1(20, 1, 10, 0),
    MS_K1(20, 1, 1, 1), MS_K1(20, 1, 2, 1), MS_K1(20, 1, 10, 1),
    MS_K1(20, 1, 1, 2), MS_K1(20, 1, 2, 2), MS_K1(20, 1, 10, 2),
    MS_K1(20, 2, 2, 0), MS_K1(20, 2, 10, 0),
    MS_K1(20, 2, 2, 1), MS_K1(20, 2, 10, 1),
    MS_K1(20, 2, 2, 2), MS_K1(20, 2, 10, 2),
    MS_K1(20, 4, 2, 1), MS_K1(20, 4, 10, 1),
    MS_K1(20, 4, 2, 2), MS_K1(20, 4, 10, 2),
    // finer moves of rotations onto the multiply pipe
    MS_K1(20, 1, 10, 3), MS_K1(20, 2, 10, 3), MS_K1(20, 4, 10, 3), MS_K1(20, 1, 2, 3),
    MS_K1(20, 1, 10, 4), MS_K1(20, 2, 10, 4), MS_K1(20, 4, 10, 4),
    MS_K1(20, 1, 10, 5), MS_K1(20, 2, 10, 5), MS_K1(20, 4, 10, 5),
    MS_K1(20, 1, 10, 6), MS_K1(20, 2, 10, 6), MS_K1(20, 4, 10, 6),
    MS_K1(20, 1, 10, 7), MS_K1(20, 2, 10, 7), MS_K1(20, 4, 10, 7),
    // counter-free part of the first double round computed once per page per thread
    MS_K1H(20, 2, 1), MS_K1H(20, 4, 1), MS_K1H(20, 2, 0), MS_K1H(20, 4, 0),
    MS_K1H(12, 2, 1), MS_K1H(12, 4, 1), MS_K1H(8, 2, 1), MS_K1H(8, 4, 1),
    // Reduced-round variants.
    MS_K1(12, 1, 6, 1), MS_K1(12, 2, 6, 1), MS_K1(12, 1, 2, 1),
    MS_K1(8, 1, 4, 1), MS_K1(8, 2, 4, 1), MS_K1(8, 1, 2, 1),
};

#undef MS_K1

const Entry *find(int rounds, const Tune &t) {
  for (const Entry &e : kTable)
    if (e.rounds == rounds && e.bpt == t.bpt && e.unr == t.unr && e.pol == t.pol && e.hoist == t.hoist) return &e;
  return nullptr;
}

}  // namespace

bool shape_available(int rounds, const Tune &t) {
  return find(rounds, t) != nullptr && (t.tpc == 128 || t.tpc == 256 || t.tpc == 512);
}

cudaError_t launch_pages_shape(const PageArgs &a, int rounds, const Tune &t, bool range,
                               cudaStream_t s) {
  const Entry *e = find(rounds, t);
  if (!e) return cudaErrorInvalidValue;
  if (a.n_pages == 0) return cudaSuccess;
  const int mode = range ? kModeRange : (a.dpages ? kModeListDom : kModeList);
  const cudaError_t f = injected(MS_FAULT_LAUNCH);
  if (f != cudaSuccess) return f;
  return e->fn[mode](a, t.tpc, s);
}

cudaError_t launch_pages(const ms_ctx *c, const PageArgs &a, cudaStream_t s) {
  Tune t = c->tune;
  // A launch too small to fill the GPU with the default shape gets one block
  // per thread instead: 4x the threads, a quarter of the serial work per
  // thread, so small requests finish sooner.  Shapes the caller chose are
  // used as they are.
  if (!c->shape_explicit && t.bpt > 1 && a.n_pages * (uint64_t)(64 / t.bpt) < (uint64_t)c->sm_count * 1024) {
    Tune small;
    small.bpt = 1;
    small.tpc = 128;
    small.unr = (int)c->cfg.rounds / 2;
    small.pol = kRotPerm;
    small.hoist = 0;
    if (shape_available((int)c->cfg.rounds, small)) t = small;
  }
  return launch_pages_shape(a, (int)c->cfg.rounds, t, a.pages == nullptr && a.dpages == nullptr, s);
}

// Every compiled shape, for the autotuner.
int k1_shape_count() { return (int)(sizeof(kTable) / sizeof(kTable[0])); }
void k1_shape(int i, int *rounds, Tune *t) {
  *rounds = kTable[i].rounds;
  t->bpt = kTable[i].bpt;
  t->unr = kTable[i].unr;
  t->pol = kTable[i].pol;
  t->hoist = kTable[i].hoist;
}

}  // namespace ms
