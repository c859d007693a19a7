"""CPU oracle for the MemShield page cipher -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, the smoke check and the benchmark's CPU-baseline / reference
leg may import this package.  The product library never does, and this
package never imports the product library: the two share no code.

``chacha20_oracle.c`` is a plain scalar C statement of the page cipher of
MemShield Sec. 4.4 ("GPU encryption"): each 4096-byte page is XORed with the
64 ChaCha20 keystream blocks whose counter is the block index 0..63 and whose
96-bit nonce is (page id, domain), encryption and decryption being the same
operation.  This module compiles it with gcc and wraps it with ctypes
(argument marshalling only).

Pins (tests/test_oracle_pins.py): the block and whole-page keystreams against
the OpenSSL ChaCha20 of the ``cryptography`` package, composition of the
permutation for the reduced-round variants, the round-trip, zero-page and
bit-flip invariants, and brute-force distinctness on tiny inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

PAGE_BYTES = 4096
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chacha20_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build() -> str:
    """Compile the oracle (plain -O2, no vector intrinsics) into oracle/liboracle.so."""
    if (not os.path.exists(_SO)) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", _SO + ".tmp", _SRC])
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.oracle_quarter_round.argtypes = [u32p, u32p, u32p, u32p]
            lib.oracle_permute.argtypes = [u32p, ctypes.c_int]
            lib.oracle_block.argtypes = [ctypes.c_char_p, ctypes.c_uint32, ctypes.c_char_p,
                                         ctypes.c_int, ctypes.c_void_p]
            lib.oracle_page_nonce.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p]
            lib.oracle_page_xor.argtypes = [ctypes.c_char_p, ctypes.c_uint64, ctypes.c_uint32,
                                            ctypes.c_int, ctypes.c_void_p]
            lib.oracle_crypt_pages.argtypes = [ctypes.c_char_p, ctypes.c_uint32, ctypes.c_int,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_size_t]
            for f in ("oracle_quarter_round", "oracle_permute", "oracle_block",
                      "oracle_page_nonce", "oracle_page_xor", "oracle_crypt_pages"):
                getattr(lib, f).restype = None
            _lib = lib
    return _lib


def _key(key: bytes) -> bytes:
    key = bytes(key)
    if len(key) != 32:
        raise ValueError("key must be 32 bytes")
    return key


def quarter_round(a: int, b: int, c: int, d: int):
    w = [ctypes.c_uint32(v & 0xFFFFFFFF) for v in (a, b, c, d)]
    _load().oracle_quarter_round(*[ctypes.byref(x) for x in w])
    return tuple(x.value for x in w)


def permute(words, rounds: int = 20):
    arr = (ctypes.c_uint32 * 16)(*[int(v) & 0xFFFFFFFF for v in words])
    _load().oracle_permute(arr, rounds)
    return list(arr)


def block(key: bytes, counter: int, nonce: bytes, rounds: int = 20) -> bytes:
    nonce = bytes(nonce)
    if len(nonce) != 12:
        raise ValueError("nonce must be 12 bytes")
    out = ctypes.create_string_buffer(64)
    _load().oracle_block(_key(key), counter & 0xFFFFFFFF, nonce, rounds, out)
    return out.raw


def page_nonce(page_id: int, domain: int = 0) -> bytes:
    out = ctypes.create_string_buffer(12)
    _load().oracle_page_nonce(page_id & 0xFFFFFFFFFFFFFFFF, domain & 0xFFFFFFFF, out)
    return out.raw


def page_keystream(key: bytes, page_id: int, domain: int = 0, rounds: int = 20) -> bytes:
    buf = np.zeros(PAGE_BYTES, dtype=np.uint8)
    _load().oracle_page_xor(_key(key), page_id & 0xFFFFFFFFFFFFFFFF, domain & 0xFFFFFFFF, rounds,
                            buf.ctypes.data)
    return buf.tobytes()


def page_xor(key: bytes, page_id: int, page: np.ndarray, domain: int = 0, rounds: int = 20) -> None:
    """XOR one page (uint8 array of 4096 bytes, C-contiguous) in place."""
    if page.dtype != np.uint8 or page.size != PAGE_BYTES or not page.flags.c_contiguous:
        raise ValueError("page must be a contiguous uint8[4096]")
    _load().oracle_page_xor(_key(key), page_id & 0xFFFFFFFFFFFFFFFF, domain & 0xFFFFFFFF, rounds,
                            page.ctypes.data)


def crypt_pages(key: bytes, buf: np.ndarray, slots, ids, domain: int = 0, rounds: int = 20,
                threads: int = 1) -> None:
    """Encrypt/decrypt in place the pages ``buf[4096*slot : 4096*slot+4096]`` with ids ``ids``.

    ``threads`` > 1 splits the list into contiguous parts run on a thread pool
    (the ctypes call releases the GIL); each part is the same scalar routine.
    """
    if buf.dtype != np.uint8 or not buf.flags.c_contiguous:
        raise ValueError("buf must be contiguous uint8")
    slots = np.ascontiguousarray(slots, dtype=np.uint64)
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    if slots.shape != ids.shape:
        raise ValueError("slots and ids differ in length")
    n = slots.size
    if n and int(slots.max()) * PAGE_BYTES + PAGE_BYTES > buf.size:
        raise ValueError("slot outside buffer")
    lib, k = _load(), _key(key)

    def run(a, b):
        if b > a:
            lib.oracle_crypt_pages(k, domain & 0xFFFFFFFF, rounds, buf.ctypes.data,
                                   slots.ctypes.data + 8 * a, ids.ctypes.data + 8 * a, b - a)

    if threads <= 1 or n < 2:
        run(0, n)
        return
    parts = np.linspace(0, n, threads + 1).astype(np.int64)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda i: run(int(parts[i]), int(parts[i + 1])), range(threads)))
