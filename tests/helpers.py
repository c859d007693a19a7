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
