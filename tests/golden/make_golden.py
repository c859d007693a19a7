"""Write tests/golden/oracle_vectors.txt from the CPU oracle alone.

Stored values: for the small configuration (256 pages of SplitMix64 seed 0,
key = first 32 bytes of SplitMix64 seed 1, page ids 0..255, domain 0) the
SHA-256 of the encrypted buffer, plus the SHA-256 of single page keystreams
and a few raw 64-byte blocks.  test_golden.py checks that the oracle still
gives these values and that the OpenSSL ChaCha20 of the ``cryptography``
package gives them too.

Run: python tests/golden/make_golden.py
"""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_vectors.txt")
PAGE_IDS = [0, 1, 255, 262143, 2**32 + 7, 2**63 + 1]


def main():
    key = synth.key_bytes(1)
    lines = ["# MemShield page cipher, written by make_golden.py from the CPU oracle.",
             "# key = SplitMix64(seed 1)[0:32]; nonce = LE64(page_id) || LE32(domain); counter = block 0..63",
             f"key {key.hex()}"]
    buf = synth.page_bytes(0, 0, 256)
    lines.append(f"small_plain_sha256 {hashlib.sha256(buf.tobytes()).hexdigest()}")
    ids = np.arange(256, dtype=np.uint64)
    oracle.crypt_pages(key, buf, ids, ids)
    lines.append(f"small_cipher_sha256 {hashlib.sha256(buf.tobytes()).hexdigest()}")
    for pid in PAGE_IDS:
        ks = oracle.page_keystream(key, pid)
        lines.append(f"page_keystream_sha256 {pid} 0 {hashlib.sha256(ks).hexdigest()}")
    ks = oracle.page_keystream(key, 9, 3)
    lines.append(f"page_keystream_sha256 9 3 {hashlib.sha256(ks).hexdigest()}")
    for pid, j in ((0, 0), (0, 63), (255, 17)):
        blk = oracle.page_keystream(key, pid)[64 * j:64 * j + 64]
        lines.append(f"block {pid} 0 {j} {blk.hex()}")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"wrote {OUT}")


if __name__ == "__main__":
    main()
