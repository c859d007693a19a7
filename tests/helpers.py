"""Shared helpers for the GPU parity tests (oracle on the host, library on the device)."""
import numpy as np

import oracle
import synth

PAGE = 4096


def oracle_expected(key, plain: np.ndarray, slots, ids, domain=0, rounds=20, threads=8):
    """Oracle result for pages ``slots`` (ids ``ids``) of a host copy of ``plain``."""
    out = plain.copy()
    oracle.crypt_pages(key, out, slots, ids, domain=domain, rounds=rounds, threads=threads)
    return out


def oracle_pages(key, seed, page_indices, ids, domain=0, rounds=20):
    """Oracle output for single pages of the SplitMix64 buffer ``seed`` (any buffer size)."""
    page_indices = np.asarray(page_indices, dtype=np.int64)
    out = np.empty((len(page_indices), PAGE), dtype=np.uint8)
    for k, p in enumerate(page_indices):
        pg = synth.page_bytes(seed, int(p), 1)
        oracle.page_xor(key, int(ids[k]), pg, domain=domain, rounds=rounds)
        out[k] = pg
    return out


def sample_pages(seed, n_pages, count):
    """A seeded sample of page indices that always includes the first and last page."""
    idx = (synth.splitmix64(seed, 0, count) % np.uint64(n_pages)).astype(np.int64)
    return np.unique(np.concatenate([[0, n_pages - 1], idx]))


def check_whole_buffer(key, seed, n_pages, odd, got_chunk, threads=None, chunk_pages=262144):
    """Whole-buffer parity against the closed form: page p of SplitMix64(seed)
    ends XORed with its keystream (page id p) iff odd[p] (an odd number of
    applications), else unchanged.  The expected buffer is built chunk by chunk
    on the host (the oracle over all host cores on the chunk's odd pages) and
    compared with got_chunk(first_page, n) byte for byte; both sides are also
    hashed.  Returns (SHA-256 of the result, SHA-256 of the expectation)."""
    import hashlib
    import os
    threads = threads or max(1, os.cpu_count() or 1)
    hg, hw = hashlib.sha256(), hashlib.sha256()
    for p0 in range(0, n_pages, chunk_pages):
        m = min(chunk_pages, n_pages - p0)
        want = np.empty(m * PAGE, dtype=np.uint8)
        synth.fill_pages(want.ctypes.data, seed, p0, m)
        sel = np.nonzero(odd[p0:p0 + m])[0].astype(np.uint64)
        oracle.crypt_pages(key, want, sel, sel + np.uint64(p0), threads=threads)
        got = np.ascontiguousarray(got_chunk(p0, m))
        hg.update(got)
        hw.update(want)
        if not np.array_equal(got, want):
            bad = np.nonzero((got.reshape(m, PAGE) != want.reshape(m, PAGE)).any(axis=1))[0]
            raise AssertionError(f"{len(bad)} pages differ in chunk at page {p0}, first {p0 + int(bad[0])}")
    return hg.hexdigest(), hw.hexdigest()


def check_sampled_pages(key, seed, touched, odd, got_pages, sample_seed, fraction=16):
    """A seeded 1/fraction sample of the touched pages, each recomputed on its
    own from the input generator and the oracle's single-page routine, against
    got_pages(page indices) -> uint8[k, PAGE]."""
    k = max(1, len(touched) // fraction)
    pick = np.unique(touched[(synth.splitmix64(sample_seed, 0, k) % np.uint64(len(touched))).astype(np.int64)])
    got = got_pages(pick)
    for i, p in enumerate(pick):
        pg = synth.page_bytes(seed, int(p), 1)
        if odd[p]:
            oracle.page_xor(key, int(p), pg)
        assert np.array_equal(got[i], pg), f"page {p}"
    return len(pick)


def fill_device(d, seed, n_pages, chunk_pages=262144):
    """Write pages 0..n_pages-1 of SplitMix64(seed) into the device tensor d."""
    import torch
    h = torch.empty(min(chunk_pages, n_pages) * PAGE, dtype=torch.uint8).pin_memory()
    for p0 in range(0, n_pages, chunk_pages):
        m = min(chunk_pages, n_pages - p0)
        synth.fill_pages(h.data_ptr(), seed, p0, m)
        d[p0 * PAGE:(p0 + m) * PAGE].copy_(h[:m * PAGE])
    torch.cuda.synchronize()
