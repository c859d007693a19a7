/* Uses the library from plain C: encrypts 4 host pages (ids 100..103, domain
 * 9, key bytes 0..31, page bytes (i * 7 + page) mod 256) through
 * ms_crypt_host, prints the ciphertext as hex, decrypts and checks the round
 * trip.  Exit 0: printed and restored; 77: no usable CUDA device; 1: error. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "memshield.h"

int main(void) {
  uint8_t key[MS_KEY_BYTES];
  for (unsigned i = 0; i < MS_KEY_BYTES; ++i) key[i] = (uint8_t)i;
  enum { N = 4 };
  static uint8_t buf[N * MS_PAGE_BYTES], plain[N * MS_PAGE_BYTES];
  for (unsigned p = 0; p < N; ++p)
    for (unsigned i = 0; i < MS_PAGE_BYTES; ++i) plain[p * MS_PAGE_BYTES + i] = (uint8_t)(i * 7u + p);
  memcpy(buf, plain, sizeof(buf));
  ms_config cfg;
  ms_config_default(&cfg);
  cfg.domain = 9;
  ms_ctx *ctx = NULL;
  int rc = ms_init(&ctx, key, &cfg);
  if (rc == MS_ECUDA) {
    fprintf(stderr, "no usable CUDA device: %s\n", ms_strerror(rc));
    return 77;
  }
  if (rc != MS_OK) {
    fprintf(stderr, "ms_init: %s\n", ms_strerror(rc));
    return 1;
  }
  rc = ms_crypt_host(ctx, MS_ENCRYPT, buf, 100, N, 0, 0);
  if (rc != MS_OK) {
    fprintf(stderr, "encrypt: %s\n", ms_strerror(rc));
    return 1;
  }
  for (unsigned i = 0; i < sizeof(buf); ++i) printf("%02x", buf[i]);
  printf("\n");
  rc = ms_crypt_host(ctx, MS_DECRYPT, buf, 100, N, 0, 0);
  if (rc != MS_OK || memcmp(buf, plain, sizeof(buf)) != 0) {
    fprintf(stderr, "round trip failed\n");
    return 1;
  }
  return ms_shutdown(ctx) == MS_OK ? 0 : 1;
}
