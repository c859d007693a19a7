// Autotuner: times every compiled launch shape of the page kernels on this
// GPU and keeps the fastest.  K1 (one launch) is tuned over blocks per
// thread, threads per CTA, double-round unroll and rotation policy on a
// contiguous sample; K2 (persistent queue) is then tuned over pages claimed
// per atomic and CTAs per SM on a scattered sample list.  The result can be
// saved to / loaded from a one-line text table keyed by GPU name, SM count
// and round count.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ms_internal.h"

using namespace ms;

namespace {

constexpr int kReps = 5;

struct Scratch {
  uint8_t *pages = nullptr;
  ms_page *list = nullptr;
  uint32_t *hdr = nullptr;  // [count, head]
  cudaEvent_t a = nullptr, b = nullptr;
  ~Scratch() {
    if (pages) cudaFree(pages);
    if (list) cudaFree(list);
    if (hdr) cudaFree(hdr);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// Median of kReps timed runs of `fn` (each enqueued on s), in milliseconds.
template <typename F>
cudaError_t time_median(cudaStream_t s, Scratch &x, F fn, float *ms_out) {
  cudaError_t e = fn();  // warm-up
  if (e != cudaSuccess) return e;
  std::vector<float> t;
  for (int r = 0; r < kReps; ++r) {
    cudaEventRecord(x.a, s);
    e = fn();
    if (e != cudaSuccess) return e;
    cudaEventRecord(x.b, s);
    e = cudaEventSynchronize(x.b);
    if (e != cudaSuccess) return e;
    float ms = 0;
    cudaEventElapsedTime(&ms, x.a, x.b);
    t.push_back(ms);
  }
  std::sort(t.begin(), t.end());
  *ms_out = t[t.size() / 2];
  return cudaSuccess;
}

std::string device_tag(int dev, int sms) {
  cudaDeviceProp p;
  std::string name = "unknown";
  if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) name = p.name;
  for (char &ch : name)
    if (ch == ' ') ch = '_';
  return name + " " + std::to_string(sms);
}

}  // namespace

extern "C" {

int ms_autotune(ms_ctx *c, size_t sample_pages, ms_tune_result *out) {
  if (!c || !c->alive) return MS_ENOTINIT;
  if (sample_pages == 0) sample_pages = 65536;
  if (sample_pages > (1u << 24)) return MS_ERANGE;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  Scratch x;
  cudaError_t e = cudaMalloc(&x.pages, sample_pages * MS_PAGE_BYTES);
  if (e == cudaSuccess) e = cudaMalloc(&x.list, sample_pages * sizeof(ms_page));
  if (e == cudaSuccess) e = cudaMalloc(&x.hdr, 2 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaEventCreate(&x.a);
  if (e == cudaSuccess) e = cudaEventCreate(&x.b);
  if (e != cudaSuccess) return alloc_fail(c, e);
  cudaStream_t s = c->stream;
  e = cudaMemsetAsync(x.pages, 0, sample_pages * MS_PAGE_BYTES, s);
  // scattered list: a fixed pseudo-random permutation of the sample's slots
  std::vector<ms_page> h(sample_pages);
  std::vector<uint32_t> perm(sample_pages);
  for (size_t i = 0; i < sample_pages; ++i) perm[i] = (uint32_t)i;
  uint64_t st = 0x243F6A8885A308D3ull;
  for (size_t i = sample_pages - 1; i > 0; --i) {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    std::swap(perm[i], perm[(st >> 33) % (i + 1)]);
  }
  for (size_t i = 0; i < sample_pages; ++i) {
    h[i].addr = (uint64_t)(x.pages + (size_t)perm[i] * MS_PAGE_BYTES);
    h[i].page_id = i;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(x.list, h.data(), sample_pages * sizeof(ms_page), cudaMemcpyHostToDevice, s);
  const uint32_t hdr[2] = {(uint32_t)sample_pages, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(x.hdr, hdr, sizeof(hdr), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e);

  const int rounds = (int)c->cfg.rounds;
  const double bytes = (double)sample_pages * MS_PAGE_BYTES;
  ms_tune_result r{};
  // ---- K1 over every compiled shape
  Tune best = c->tune;
  float best_ms = 1e30f;
  const int tpcs[3] = {128, 256, 512};
  for (int i = 0; i < k1_shape_count(); ++i) {
    int rr;
    Tune t;
    k1_shape(i, &rr, &t);
    if (rr != rounds) continue;
    for (int tpc : tpcs) {
      t.tpc = tpc;
      PageArgs a = make_args(c);
      a.base = x.pages;
      a.n_pages = sample_pages;
      float ms = 0.0f;
      e = time_median(s, x, [&] { return launch_pages_shape(a, rounds, t, true, s); }, &ms);
      if (e != cudaSuccess) return cuda_fail(c, e);
      r.tried += 1;
      if (ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
  }
  c->tune = best;
  r.shape.blocks_per_thread = (uint32_t)best.bpt;
  r.shape.threads_per_cta = (uint32_t)best.tpc;
  r.shape.dr_unroll = (uint32_t)best.unr;
  r.shape.rot_policy = (uint32_t)best.pol;
  r.shape.hoist = (uint32_t)best.hoist;
  r.k1_gbs = bytes / (best_ms * 1e-3) / 1e9;

  // ---- K2 over pages-per-claim and CTAs per SM, with the chosen shape
  QueueKernel k;
  if (!queue_kernel(rounds, best, &k)) return MS_EINVAL;
  int fit = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k.fn, best.tpc, 0);
  if (fit < 1) fit = 1;
  const int grabs[7] = {1, 2, 4, 8, 16, 32, 64};
  const int cps_opts[2] = {fit, std::max(1, fit / 2)};
  QTune qbest = c->qtune;
  float qbest_ms = 1e30f;
  for (int grab : grabs) {
    for (int ci = 0; ci < (fit > 1 ? 2 : 1); ++ci) {
      const int cps = cps_opts[ci];
      QueueArgs q{};
      q.items = x.list;
      q.count = x.hdr;
      q.head = x.hdr + 1;
      q.grab = (uint32_t)grab;
      q.key = c->d_key;
      q.domain = c->cfg.domain;
      q.status = c->d_status;
      q.mc.m12 = 1u << 12;
      q.mc.m7 = 1u << 7;
      const int grid = queue_grid(c, k, best.tpc, cps);
      float ms = 0.0f;
      e = time_median(s, x, [&] {
        cudaError_t e1 = cudaMemsetAsync(x.hdr + 1, 0, sizeof(uint32_t), s);
        return e1 == cudaSuccess ? k.launch(q, grid, best.tpc, s) : e1;
      }, &ms);
      if (e != cudaSuccess) return cuda_fail(c, e);
      r.tried += 1;
      if (ms < qbest_ms) {
        qbest_ms = ms;
        qbest.grab = grab;
        qbest.ctas_per_sm = (cps == fit) ? 0 : cps;
      }
    }
  }
  c->qtune = qbest;
  c->tune_gen.fetch_add(1);
  r.grab = (uint32_t)qbest.grab;
  r.ctas_per_sm = (uint32_t)(qbest.ctas_per_sm ? qbest.ctas_per_sm : fit);
  r.queue_gbs = bytes / (qbest_ms * 1e-3) / 1e9;
  if (out) *out = r;
  return MS_OK;
}

int ms_tune_save(const ms_ctx *c, const char *path) {
  if (!c || !c->alive) return MS_ENOTINIT;
  if (!path) return MS_EINVAL;
  FILE *f = std::fopen(path, "w");
  if (!f) return MS_EINVAL;
  const std::string tag = device_tag(c->device, c->sm_count);
  std::fprintf(f, "memshield-tune-v2 %s %u %d %d %d %d %d %d %d\n", tag.c_str(), c->cfg.rounds, c->tune.bpt,
               c->tune.tpc, c->tune.unr, c->tune.pol, c->tune.hoist, c->qtune.grab, c->qtune.ctas_per_sm);
  std::fclose(f);
  return MS_OK;
}

int ms_tune_load(ms_ctx *c, const char *path) {
  if (!c || !c->alive) return MS_ENOTINIT;
  if (!path) return MS_EINVAL;
  FILE *f = std::fopen(path, "r");
  if (!f) return MS_EINVAL;
  char magic[32], name[256];
  int sms, rounds;
  Tune t;
  QTune q;
  const int got = std::fscanf(f, "%31s %255s %d %d %d %d %d %d %d %d %d", magic, name, &sms, &rounds, &t.bpt,
                              &t.tpc, &t.unr, &t.pol, &t.hoist, &q.grab, &q.ctas_per_sm);
  std::fclose(f);
  if (got != 11 || std::strcmp(magic, "memshield-tune-v2") != 0) return MS_EINVAL;
  const std::string tag = std::string(name) + " " + std::to_string(sms);
  if (tag != device_tag(c->device, c->sm_count) || rounds != (int)c->cfg.rounds) return MS_EINVAL;
  if (!shape_available(rounds, t) || q.grab < 1 || q.grab > 4096 || q.ctas_per_sm < 0) return MS_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  c->tune = t;  // like a tuning run's result: small launches may still adapt it
  c->qtune = q;
  c->tune_gen.fetch_add(1);
  return MS_OK;
}

}  // extern "C"
