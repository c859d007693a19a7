"""Stored oracle vectors: the oracle still reproduces them, and OpenSSL agrees with them."""
import hashlib
import os
import struct

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_vectors.txt")


def load():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            rows.setdefault(parts[0], []).append(parts[1:])
    return rows


def test_oracle_reproduces_golden(oracle_mod):
    g = load()
    key = bytes.fromhex(g["key"][0][0])
    assert key == synth.key_bytes(1)
    buf = synth.page_bytes(0, 0, 256)
    assert hashlib.sha256(buf.tobytes()).hexdigest() == g["small_plain_sha256"][0][0]
    ids = np.arange(256, dtype=np.uint64)
    oracle_mod.crypt_pages(key, buf, ids, ids)
    assert hashlib.sha256(buf.tobytes()).hexdigest() == g["small_cipher_sha256"][0][0]
    for pid, dom, h in g["page_keystream_sha256"]:
        assert hashlib.sha256(oracle_mod.page_keystream(key, int(pid), int(dom))).hexdigest() == h
    for pid, dom, j, hx in g["block"]:
        j = int(j)
        assert oracle_mod.page_keystream(key, int(pid), int(dom))[64 * j:64 * j + 64].hex() == hx


def test_golden_agrees_with_openssl():
    crypto = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    g = load()
    key = bytes.fromhex(g["key"][0][0])

    def stream(pid, dom):
        iv = struct.pack("<I", 0) + struct.pack("<QI", pid, dom)
        return crypto.Cipher(crypto.algorithms.ChaCha20(key, iv), mode=None).encryptor().update(bytes(4096))

    for pid, dom, h in g["page_keystream_sha256"]:
        assert hashlib.sha256(stream(int(pid), int(dom))).hexdigest() == h
    buf = synth.page_bytes(0, 0, 256).reshape(256, 4096)
    for p in range(256):
        buf[p] ^= np.frombuffer(stream(p, 0), np.uint8)
    assert hashlib.sha256(buf.tobytes()).hexdigest() == g["small_cipher_sha256"][0][0]
