// Host-only simulation of the served form's admission policy (ms_admission.h):
// random requests, waves formed while the pipeline has room, waves released
// in issue order at random times.  Checks on every step:
//   - a wave's slots lie inside the ring and do not overlap an in-flight wave's
//     slots, and the ring's use never exceeds its size;
//   - a page is never in two in-flight waves, nor twice in one wave;
//   - requests that share a page are admitted in arrival order;
//   - every request is admitted in the end (no starvation).
// With inplace_max > 0, in-place waves (form_inplace: no staging slots, at
// most inplace_max pages, formed only while the whole queue fits) are mixed
// in and complete in random order; the same checks cover them.
// Usage: admission_sim seed slots max_wave one_per_launch n_pages n_req max_req_pages depth inplace_max
#include <cstdio>
#include <cstdlib>
#include <deque>
#include <map>
#include <set>
#include <vector>

#include "ms_admission.h"

static uint64_t s_state;
static uint64_t rnd() {  // splitmix64 step
  uint64_t z = (s_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

#define FAIL(...)                 \
  do {                            \
    std::printf("FAIL ");         \
    std::printf(__VA_ARGS__);     \
    std::printf("\n");           \
    return 1;                     \
  } while (0)

int main(int argc, char **argv) {
  if (argc != 10) return 2;
  s_state = std::strtoull(argv[1], nullptr, 10);
  const uint32_t S = (uint32_t)std::atoi(argv[2]), max_wave = (uint32_t)std::atoi(argv[3]);
  const bool one = std::atoi(argv[4]) != 0;
  const uint64_t n_pages = std::strtoull(argv[5], nullptr, 10);
  const size_t n_req = std::strtoull(argv[6], nullptr, 10);
  const uint32_t max_req = (uint32_t)std::atoi(argv[7]), depth = (uint32_t)std::atoi(argv[8]);
  const uint32_t inplace_max = (uint32_t)std::atoi(argv[9]);

  std::vector<std::vector<uint64_t>> pages(n_req);
  for (size_t r = 0; r < n_req; ++r) {
    const uint32_t n = 1 + (uint32_t)(rnd() % max_req);
    std::set<uint64_t> s;
    while (s.size() < n) s.insert(rnd() % n_pages);
    pages[r].assign(s.begin(), s.end());
  }
  ms::Admission adm(S, max_wave, one, n_pages, 64);
  auto pages_of = [&](uint64_t t) -> const std::vector<uint64_t> & { return pages[t]; };
  std::deque<uint64_t> queue;
  std::deque<ms::AdmittedWave> inflight, inplace;
  std::vector<long> admitted_at(n_req, -1);
  std::map<uint64_t, std::vector<uint64_t>> page_order;  // page -> tickets in admission order
  size_t next = 0, done = 0, n_inplace = 0;
  long step = 0;
  while (done < n_req) {
    if (++step > 50000000) FAIL("no progress");
    const uint64_t x = rnd() % 8;
    if (x < 3 && next < n_req) {  // arrivals
      const size_t k = 1 + rnd() % 8;
      for (size_t i = 0; i < k && next < n_req; ++i) queue.push_back(next++);
    } else if (x < 6 && (inflight.size() < depth || inplace.size() < depth)) {
      ms::AdmittedWave w;
      bool ip = false, ok = false;
      if (inplace_max && inplace.size() < depth) ok = ip = adm.form_inplace(queue, pages_of, w, inplace_max);
      if (!ok && inflight.size() < depth) ok = adm.form(queue, pages_of, w);
      if (ok) {
        if (ip && (w.span != 0 || w.len > inplace_max)) FAIL("in-place wave: span %u len %u", w.span, w.len);
        if (!ip && (w.pos + w.len > S || w.span < w.len)) FAIL("wave outside the ring: pos %u len %u", w.pos, w.len);
        if (adm.used() > S) FAIL("ring over-used: %u > %u", adm.used(), S);
        if (!ip && one && w.tickets.size() != 1) FAIL("one-per-launch wave with %zu requests", w.tickets.size());
        if (!ip && w.len > max_wave && w.tickets.size() > 1) FAIL("wave of %u pages", w.len);
        uint32_t len = 0;
        std::set<uint64_t> in_wave;
        for (uint64_t t : w.tickets) {
          len += (uint32_t)pages[t].size();
          admitted_at[t] = step;
          for (uint64_t pg : pages[t]) {
            if (!in_wave.insert(pg).second) FAIL("page %llu twice in one wave", (unsigned long long)pg);
            page_order[pg].push_back(t);
          }
        }
        if (len != w.len) FAIL("wave length %u, requests hold %u pages", w.len, len);
        for (const auto *set : {&inflight, &inplace})
          for (const auto &o : *set) {
            const bool overlap = !ip && o.span && !(w.pos + w.len <= o.pos || o.pos + o.len <= w.pos);
            if (overlap) FAIL("slots [%u,%u) overlap in-flight [%u,%u)", w.pos, w.pos + w.len, o.pos, o.pos + o.len);
            for (uint64_t t : o.tickets)
              for (uint64_t pg : pages[t])
                if (in_wave.count(pg)) FAIL("page %llu in two in-flight waves", (unsigned long long)pg);
          }
        (ip ? inplace : inflight).push_back(w);
        n_inplace += ip;
      }
    } else if (!inplace.empty() && (inflight.empty() || rnd() % 2)) {  // any in-place wave completes
      const size_t i = rnd() % inplace.size();
      adm.release(inplace[i], pages_of);
      done += inplace[i].tickets.size();
      inplace.erase(inplace.begin() + (long)i);
    } else if (!inflight.empty()) {  // the oldest staged wave completes
      adm.release(inflight.front(), pages_of);
      done += inflight.front().tickets.size();
      inflight.pop_front();
    }
  }
  for (size_t r = 0; r < n_req; ++r)
    if (admitted_at[r] < 0) FAIL("request %zu never admitted", r);
  for (const auto &kv : page_order)
    for (size_t i = 1; i < kv.second.size(); ++i)
      if (kv.second[i] < kv.second[i - 1])
        FAIL("page %llu: request %llu admitted before earlier request %llu", (unsigned long long)kv.first,
             (unsigned long long)kv.second[i], (unsigned long long)kv.second[i - 1]);
  if (adm.used() != 0) FAIL("ring not empty at the end: %u", adm.used());
  if (inplace_max && n_inplace == 0) FAIL("no in-place wave was formed");
  std::printf("OK requests %zu conflict_waits %llu budget_waits %llu in_place_waves %zu\n", n_req,
              (unsigned long long)adm.conflict_waits, (unsigned long long)adm.budget_waits, n_inplace);
  return 0;
}
