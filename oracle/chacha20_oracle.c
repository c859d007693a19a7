/*
 * MemShield page-cipher oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, scalar C statement of what the GPU page cipher computes.  It
 * exists to check the CUDA library; only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes (MemShield, Sec. 4.4 "GPU encryption"):
 *   - every cryptographic operation acts on one 4096-byte page;
 *   - the page is XORed with 64 ChaCha20 keystream blocks of 64 bytes;
 *   - each block comes from a 384-bit seed: the 256-bit master key plus a
 *     128-bit value built from the page's address, the client's PID and a
 *     block counter 0..63 (the index of the 64-byte block in the page);
 *   - encryption and decryption are the same operation.
 * ChaCha20 itself is Bernstein's ChaCha with 20 rounds (the paper's cited
 * "strongest variant"), in the RFC 8439 state layout:
 *   words 0..3  the ASCII constant "expand 32-byte k" read as LE words,
 *   words 4..11 the key as 8 little-endian words,
 *   word  12    the 32-bit block counter,
 *   words 13..15 the 96-bit nonce as 3 little-endian words;
 *   10 double rounds (4 column quarter-rounds, then 4 diagonal ones), then
 *   the input state is added word-wise and the words are written LE.
 *
 * Readings where the paper is silent (Sec. 4.4 gives no field order):
 *   - counter word = block index j in 0..63, starting at 0 (not RFC AEAD's 1);
 *   - nonce = LE32(lo32(page_id)) || LE32(hi32(page_id)) || LE32(domain),
 *     where page_id stands for the paper's page address and domain for the
 *     client PID (0 unless a caller sets it);
 *   - the round count is a parameter so the reduced-round variants (8, 12)
 *     use the same code; the paper's configuration is 20.
 */
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#define ORACLE_PAGE_BYTES 4096
#define ORACLE_BLOCK_BYTES 64

static uint32_t rotl32(uint32_t v, int c) { return (uint32_t)((v << c) | (v >> (32 - c))); }

static uint32_t load_le32(const uint8_t *p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

static void store_le32(uint8_t *p, uint32_t v) {
  p[0] = (uint8_t)(v);
  p[1] = (uint8_t)(v >> 8);
  p[2] = (uint8_t)(v >> 16);
  p[3] = (uint8_t)(v >> 24);
}

/* The ChaCha quarter round on four words of the state (Bernstein's ChaCha,
 * the cipher Sec. 4.4 names; RFC 8439 Sec. 2.1): add, xor, rotate by 16, 12,
 * 8 and 7. */
void oracle_quarter_round(uint32_t *a, uint32_t *b, uint32_t *c, uint32_t *d) {
  *a += *b; *d ^= *a; *d = rotl32(*d, 16);
  *c += *d; *b ^= *c; *b = rotl32(*b, 12);
  *a += *b; *d ^= *a; *d = rotl32(*d, 8);
  *c += *d; *b ^= *c; *b = rotl32(*b, 7);
}

/* The ChaCha permutation: rounds/2 double rounds, each four column quarter
 * rounds then four diagonal ones (RFC 8439 Sec. 2.3); no feed-forward. */
void oracle_permute(uint32_t x[16], int rounds) {
  for (int r = 0; r < rounds; r += 2) {
    /* column round */
    oracle_quarter_round(&x[0], &x[4], &x[8], &x[12]);
    oracle_quarter_round(&x[1], &x[5], &x[9], &x[13]);
    oracle_quarter_round(&x[2], &x[6], &x[10], &x[14]);
    oracle_quarter_round(&x[3], &x[7], &x[11], &x[15]);
    /* diagonal round */
    oracle_quarter_round(&x[0], &x[5], &x[10], &x[15]);
    oracle_quarter_round(&x[1], &x[6], &x[11], &x[12]);
    oracle_quarter_round(&x[2], &x[7], &x[8], &x[13]);
    oracle_quarter_round(&x[3], &x[4], &x[9], &x[14]);
  }
}

/* One 64-byte keystream block (Sec. 4.4: 512 bits from the 256-bit key and a
 * 128-bit value; RFC 8439 Sec. 2.3 layout): permute the input state, add it
 * back, serialise little-endian. */
void oracle_block(const uint8_t key[32], uint32_t counter, const uint8_t nonce[12], int rounds,
                  uint8_t out[64]) {
  static const char sigma[17] = "expand 32-byte k";
  uint32_t in[16], x[16];
  for (int i = 0; i < 4; i++) in[i] = load_le32((const uint8_t *)sigma + 4 * i);
  for (int i = 0; i < 8; i++) in[4 + i] = load_le32(key + 4 * i);
  in[12] = counter;
  for (int i = 0; i < 3; i++) in[13 + i] = load_le32(nonce + 4 * i);
  memcpy(x, in, sizeof x);
  oracle_permute(x, rounds);
  for (int i = 0; i < 16; i++) store_le32(out + 4 * i, x[i] + in[i]);
}

/* The per-page 96-bit nonce (Sec. 4.4: page address + client PID; the field
 * order is this library's reading): page id (64 bits, LE) then the domain
 * word (PID slot). */
void oracle_page_nonce(uint64_t page_id, uint32_t domain, uint8_t nonce[12]) {
  store_le32(nonce + 0, (uint32_t)(page_id & 0xffffffffu));
  store_le32(nonce + 4, (uint32_t)(page_id >> 32));
  store_le32(nonce + 8, domain);
}

/* XOR one 4096-byte page with its 64 keystream blocks, counters 0..63
 * (Sec. 4.4: the counter is the index of the 512-bit block in the page, and
 * the same XOR encrypts and decrypts). */
void oracle_page_xor(const uint8_t key[32], uint64_t page_id, uint32_t domain, int rounds,
                     uint8_t *page) {
  uint8_t nonce[12], ks[ORACLE_BLOCK_BYTES];
  oracle_page_nonce(page_id, domain, nonce);
  for (uint32_t j = 0; j < ORACLE_PAGE_BYTES / ORACLE_BLOCK_BYTES; j++) {
    oracle_block(key, j, nonce, rounds, ks);
    for (int k = 0; k < ORACLE_BLOCK_BYTES; k++) page[ORACLE_BLOCK_BYTES * j + k] ^= ks[k];
  }
}

/* Encrypt (equivalently decrypt) n pages: page k lives at base + 4096 * slot[k]
 * and uses id ids[k].  Pages are processed one after another, in list order. */
void oracle_crypt_pages(const uint8_t key[32], uint32_t domain, int rounds, uint8_t *base,
                        const uint64_t *slot, const uint64_t *ids, size_t n) {
  for (size_t k = 0; k < n; k++)
    oracle_page_xor(key, ids[k], domain, rounds, base + (size_t)ORACLE_PAGE_BYTES * slot[k]);
}
