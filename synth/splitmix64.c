/* Threaded SplitMix64 fill for large synthetic host buffers.
 *
 * Writes outputs first..first+count-1 of the SplitMix64 stream with the
 * given seed (Steele, Lea and Flood, OOPSLA 2014, counter form: output i is
 * mix64(seed + (i + 1) * 0x9E3779B97F4A7C15)) as little-endian u64 words.
 * It produces exactly the bytes of synth.page_bytes() and holds no cipher
 * arithmetic.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

typedef struct {
  uint8_t *dst;
  uint64_t seed, first, count;
} job_t;

static void *run(void *arg) {
  job_t *j = (job_t *)arg;
  for (uint64_t i = 0; i < j->count; i++) {
    uint64_t v = mix64(j->seed + (j->first + i + 1) * 0x9E3779B97F4A7C15ULL);
    uint8_t *p = j->dst + 8 * i;
    for (int b = 0; b < 8; b++) p[b] = (uint8_t)(v >> (8 * b));
  }
  return NULL;
}

void synth_fill_u64(void *dst, uint64_t seed, uint64_t first, uint64_t count, int threads) {
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  if (count < (1u << 16)) threads = 1;
  pthread_t tid[256];
  job_t jobs[256];
  uint64_t per = (count + threads - 1) / threads;
  int started = 0;
  for (int t = 0; t < threads; t++) {
    uint64_t a = per * t;
    if (a >= count) break;
    uint64_t n = (a + per > count) ? count - a : per;
    jobs[t].dst = (uint8_t *)dst + 8 * a;
    jobs[t].seed = seed;
    jobs[t].first = first + a;
    jobs[t].count = n;
    if (pthread_create(&tid[t], NULL, run, &jobs[t]) != 0) {
      run(&jobs[t]);
      tid[t] = 0;
    }
    started = t + 1;
  }
  for (int t = 0; t < started; t++)
    if (tid[t]) pthread_join(tid[t], NULL);
}
