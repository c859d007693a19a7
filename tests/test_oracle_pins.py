"""Pins for the CPU oracle: checks against things other than the oracle itself.

* The ChaCha20 block and the whole-page keystream are compared with the
  OpenSSL ChaCha20 of the ``cryptography`` package, whose 16-byte IV is
  LE32(block counter) || 96-bit nonce.  A 4096-byte stream from counter 0 is
  exactly one page's 64 keystream blocks (MemShield Sec. 4.4: 64 blocks, the
  counter being the block index 0..63).
* Reduced-round variants (8, 12) have no library counterpart; they are pinned
  through the composition law of the permutation, anchored on the library-
  pinned 20-round case.
* Invariants from Sec. 4.4: encryption and decryption are the same XOR
  (involution), blocks are independent, one plaintext bit flips one
  ciphertext bit, and distinct (counter, page, domain) seeds give distinct
  keystream blocks (brute force on tiny inputs).
"""
import struct

import numpy as np
import pytest

import synth

try:
    from cryptography.hazmat.primitives import ciphers as crypto
except ImportError:  # only the library comparisons need it; the invariants still run
    crypto = None


def lib_stream(key: bytes, counter: int, nonce12: bytes, nbytes: int) -> bytes:
    """OpenSSL ChaCha20 keystream starting at ``counter``."""
    if crypto is None:
        pytest.skip("cryptography (OpenSSL ChaCha20) not installed")
    c = crypto.Cipher(crypto.algorithms.ChaCha20(key, struct.pack("<I", counter) + nonce12), mode=None)
    return c.encryptor().update(bytes(nbytes))


def reading_nonce(page_id: int, domain: int) -> bytes:
    # the stated reading of Sec. 4.4: 64-bit page id (LE) then 32-bit domain (LE)
    return struct.pack("<QI", page_id, domain)


def rand_cases(n, seed=11):
    w = synth.splitmix64(seed, 0, 6 * n)
    out = []
    for i in range(n):
        key = w[6 * i:6 * i + 4].astype("<u8").tobytes()
        pid = int(w[6 * i + 4])
        dom = int(w[6 * i + 5] & np.uint64(0xFFFFFFFF)) if i % 3 == 0 else 0
        out.append((key, pid, dom))
    return out


# ------------------------------------------------------------------ library pins
@pytest.mark.parametrize("counter", [0, 1, 2, 7, 63, 64, 0x7FFFFFFF, 0xFFFFFFFF])
def test_block_matches_openssl_counters(oracle_mod, counter):
    key = bytes(range(32))
    for nonce in (bytes(12), bytes.fromhex("000000090000004a00000000"),
                  bytes.fromhex("000000000000004a00000000"), bytes(range(12))):
        assert oracle_mod.block(key, counter, nonce) == lib_stream(key, counter, nonce, 64)


def test_block_matches_openssl_random_keys(oracle_mod):
    for key, pid, dom in rand_cases(64):
        nonce = reading_nonce(pid, dom)
        for ctr in (0, 31, 63):
            assert oracle_mod.block(key, ctr, nonce) == lib_stream(key, ctr, nonce, 64)


def test_page_nonce_layout(oracle_mod):
    for _, pid, dom in rand_cases(32, seed=12):
        assert oracle_mod.page_nonce(pid, dom) == reading_nonce(pid, dom)


def test_page_keystream_is_one_library_stream(oracle_mod):
    """Sec. 4.4: a page's 64 blocks, counters 0..63, equal one continuous 4096-byte stream."""
    for key, pid, dom in rand_cases(100, seed=13):
        assert oracle_mod.page_keystream(key, pid, dom) == lib_stream(key, 0, reading_nonce(pid, dom), 4096)


def test_page_keystream_config_key(oracle_mod, key1):
    for pid in (0, 1, 255, 262143, 2**32, 2**63, 2**64 - 1):
        assert oracle_mod.page_keystream(key1, pid) == lib_stream(key1, 0, reading_nonce(pid, 0), 4096)


def test_crypt_pages_uses_id_not_slot(oracle_mod, key1):
    n = 16
    data = synth.page_bytes(0, 0, n)
    buf = data.copy()
    slots = np.arange(n)[::-1].copy()
    ids = (np.arange(n) * 977 + 5).astype(np.uint64)
    oracle_mod.crypt_pages(key1, buf, slots, ids)
    for k in range(n):
        s, pid = int(slots[k]), int(ids[k])
        want = np.bitwise_xor(data[4096 * s:4096 * s + 4096],
                              np.frombuffer(lib_stream(key1, 0, reading_nonce(pid, 0), 4096), np.uint8))
        assert (buf[4096 * s:4096 * s + 4096] == want).all()


# ----------------------------------------------------------- reduced-round pins
def _state(key, counter, nonce):
    w = list(struct.unpack("<4I", b"expand 32-byte k")) + list(struct.unpack("<8I", key))
    return w + [counter] + list(struct.unpack("<3I", nonce))


def test_permute20_is_block_minus_input(oracle_mod):
    """The 20-round permutation is what the library-pinned block adds the input to."""
    for key, pid, dom in rand_cases(16, seed=14):
        nonce = reading_nonce(pid, dom)
        st = _state(key, 5, nonce)
        out = struct.unpack("<16I", lib_stream(key, 5, nonce, 64))
        assert oracle_mod.permute(st, 20) == [(o - s) & 0xFFFFFFFF for o, s in zip(out, st)]


def test_reduced_rounds_compose(oracle_mod):
    """P_a(P_b(x)) = P_(a+b)(x); with P_20 pinned, this pins the double round and P_8, P_12."""
    for key, pid, dom in rand_cases(8, seed=15):
        st = _state(key, 9, reading_nonce(pid, dom))
        d = st
        for _ in range(10):
            d = oracle_mod.permute(d, 2)
        assert d == oracle_mod.permute(st, 20)
        assert oracle_mod.permute(oracle_mod.permute(st, 8), 12) == oracle_mod.permute(st, 20)
        p8 = st
        for _ in range(4):
            p8 = oracle_mod.permute(p8, 2)
        assert p8 == oracle_mod.permute(st, 8)
        assert oracle_mod.permute(oracle_mod.permute(st, 12), 8) == oracle_mod.permute(st, 20)
        assert oracle_mod.permute(st, 0) == st


def test_reduced_round_block_is_permute_plus_input(oracle_mod):
    key, pid, dom = rand_cases(1, seed=16)[0]
    nonce = reading_nonce(pid, dom)
    for rounds in (8, 12, 20):
        st = _state(key, 3, nonce)
        want = struct.pack("<16I", *[(a + b) & 0xFFFFFFFF for a, b in zip(oracle_mod.permute(st, rounds), st)])
        assert oracle_mod.block(key, 3, nonce, rounds) == want
    assert oracle_mod.block(key, 3, nonce, 8) != oracle_mod.block(key, 3, nonce, 12)


def test_quarter_round_inverts(oracle_mod):
    """The quarter round is a bijection: undoing its 12 steps in reverse restores the input."""
    def rotr(v, c):
        return ((v >> c) | (v << (32 - c))) & 0xFFFFFFFF
    w = synth.splitmix64(17, 0, 200).astype(np.uint64)
    for i in range(50):
        x = [int(w[4 * i + k] & np.uint64(0xFFFFFFFF)) for k in range(4)]
        a, b, c, d = oracle_mod.quarter_round(*x)
        b = rotr(b, 7) ^ c; c = (c - d) & 0xFFFFFFFF
        d = rotr(d, 8) ^ a; a = (a - b) & 0xFFFFFFFF
        b = rotr(b, 12) ^ c; c = (c - d) & 0xFFFFFFFF
        d = rotr(d, 16) ^ a; a = (a - b) & 0xFFFFFFFF
        assert [a, b, c, d] == x


# ------------------------------------------------------------------- invariants
def test_round_trip_and_zero_page(oracle_mod, key1):
    p = synth.page_bytes(0, 3, 1)
    q = p.copy()
    oracle_mod.page_xor(key1, 3, q)
    assert not (q == p).all()
    oracle_mod.page_xor(key1, 3, q)          # decrypt = encrypt (Sec. 4.4)
    assert (q == p).all()
    z = np.zeros(4096, np.uint8)
    oracle_mod.page_xor(key1, 3, z)
    assert z.tobytes() == oracle_mod.page_keystream(key1, 3)


def test_bit_flip_is_local(oracle_mod, key1):
    p = synth.page_bytes(0, 0, 1)
    c0 = p.copy()
    oracle_mod.page_xor(key1, 0, c0)
    for bit in (0, 7, 511, 4095 * 8 + 3, 2048 * 8):
        q = p.copy()
        q[bit // 8] ^= np.uint8(1 << (bit % 8))
        oracle_mod.page_xor(key1, 0, q)
        diff = np.unpackbits(np.bitwise_xor(q, c0))
        assert diff.sum() == 1 and diff[(bit // 8) * 8 + 7 - bit % 8] == 1


def test_blocks_depend_only_on_key_page_counter(oracle_mod, key1):
    """Block j of page X equals the block computed in isolation (independence, Sec. 4.4)."""
    ks = oracle_mod.page_keystream(key1, 77)
    for j in (0, 1, 31, 62, 63):
        assert ks[64 * j:64 * j + 64] == oracle_mod.block(key1, j, reading_nonce(77, 0))


def test_blocks_distinct_brute_force(oracle_mod, key1):
    """No two 64-byte blocks repeat across counters, nearby ids, bit-63 ids and domains."""
    seen = set()
    for pid in (0, 1, 2, 2**63, 2**63 + 1, 2**32):
        for dom in (0, 1):
            ks = oracle_mod.page_keystream(key1, pid, dom)
            for j in range(64):
                blk = ks[64 * j:64 * j + 64]
                assert blk not in seen
                seen.add(blk)
    assert len(seen) == 6 * 2 * 64


def test_duplicate_entries_closed_form(oracle_mod, key1):
    """An odd number of applications gives p ^ K, an even number gives p, in any order."""
    n = 4
    data = synth.page_bytes(6, 0, n)
    counts = [1, 2, 3, 4]
    slots = np.concatenate([[s] * c for s, c in enumerate(counts)]).astype(np.uint64)
    order = synth.splitmix64(18, 0, slots.size).argsort()
    slots = slots[order]
    buf = data.copy()
    oracle_mod.crypt_pages(key1, buf, slots, slots)
    for s, c in enumerate(counts):
        page = data[4096 * s:4096 * s + 4096].copy()
        if c % 2:
            page ^= np.frombuffer(oracle_mod.page_keystream(key1, s), np.uint8)
        assert (buf[4096 * s:4096 * s + 4096] == page).all()


def test_threaded_split_equals_serial(oracle_mod, key1):
    n = 64
    data = synth.page_bytes(2, 0, n)
    a, b = data.copy(), data.copy()
    ids = np.arange(n, dtype=np.uint64)
    oracle_mod.crypt_pages(key1, a, ids, ids, threads=1)
    oracle_mod.crypt_pages(key1, b, ids, ids, threads=4)
    assert (a == b).all()


def test_argument_checks(oracle_mod, key1):
    with pytest.raises(ValueError):
        oracle_mod.block(b"short", 0, bytes(12))
    with pytest.raises(ValueError):
        oracle_mod.crypt_pages(key1, np.zeros(4096, np.uint8), [1], [1])
