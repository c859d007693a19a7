"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds no cipher arithmetic: it only produces page bytes, keys,
page-id lists, request sizes and arrival times.  Every random draw comes from
SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used in its counter form: output i (0-based) of the
stream with seed s is mix64(s + (i + 1) * 0x9E3779B97F4A7C15), where mix64 is
the published finaliser (xor-shift 30, multiply 0xBF58476D1CE4E5B9, xor-shift
27, multiply 0x94D049BB133111EB, xor-shift 31).  Because output i depends on
i alone, any slice of a stream can be produced independently (for example one
page of a 16 GiB working set), and the C fill in ``splitmix64.c`` produces the
same bytes as the numpy code here.

Recipes (one stream per purpose, each with its own seed):

* page bytes: u64 outputs written little-endian; page p of a buffer holds
  outputs [512 p, 512 p + 512) of the buffer's stream;
* key: the first 32 bytes of the stream with seed 1;
* Zipf(s) request sizes truncated to 1..K by inverse CDF on u = top 53 bits;
* scattered page slots: partial Fisher-Yates without replacement;
* Poisson arrivals: exponential gaps -ln(1 - u) / rate.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
PAGE_BYTES = 4096
U64_PER_PAGE = PAGE_BYTES // 8

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lib = None
_lib_lock = threading.Lock()


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * M1
    z = (z ^ (z >> np.uint64(27))) * M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, first: int, count: int) -> np.ndarray:
    """Outputs first..first+count-1 of the SplitMix64 stream with ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(first + 1, first + 1 + count, dtype=np.uint64)
        return _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GAMMA)


def uniform01(seed: int, first: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each output."""
    return (splitmix64(seed, first, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def key_bytes(seed: int = 1) -> bytes:
    """256-bit key: the first 32 bytes (4 outputs, little-endian) of stream ``seed``."""
    return splitmix64(seed, 0, 4).astype("<u8").tobytes()


# ---------------------------------------------------------------- page bytes
def build() -> str:
    """Compile the multi-threaded C fill (same bytes as ``page_bytes``)."""
    src = os.path.join(_HERE, "splitmix64.c")
    if (not os.path.exists(_SO)) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-pthread", "-o", _SO + ".tmp", src])
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    with _lib_lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.synth_fill_u64.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.c_uint64, ctypes.c_int]
            lib.synth_fill_u64.restype = None
            _lib = lib
    return _lib


def fill_pages(ptr: int, seed: int, first_page: int, n_pages: int, threads: int = 0) -> None:
    """Write pages first_page..first_page+n_pages-1 of stream ``seed`` to host address ``ptr``."""
    threads = threads or (os.cpu_count() or 1)
    _load().synth_fill_u64(ctypes.c_void_p(ptr), seed, first_page * U64_PER_PAGE,
                           n_pages * U64_PER_PAGE, threads)


def page_bytes(seed: int, first_page: int, n_pages: int) -> np.ndarray:
    """Pages [first_page, first_page + n_pages) of stream ``seed`` as a uint8 array (numpy path)."""
    words = splitmix64(seed, first_page * U64_PER_PAGE, n_pages * U64_PER_PAGE)
    return words.astype("<u8").view(np.uint8).copy()


def page_bytes_fast(seed: int, first_page: int, n_pages: int) -> np.ndarray:
    """Same bytes as ``page_bytes``, filled by the threaded C routine (for GiB-sized buffers)."""
    out = np.empty(n_pages * PAGE_BYTES, dtype=np.uint8)
    if n_pages:
        fill_pages(out.ctypes.data, seed, first_page, n_pages)
    return out


# ------------------------------------------------------------ workload recipes
def zipf_sizes(seed: int, n: int, s: float = 1.2, kmax: int = 512) -> np.ndarray:
    """``n`` request sizes from Zipf(s) truncated to 1..kmax (inverse CDF)."""
    k = np.arange(1, kmax + 1, dtype=np.float64)
    cdf = np.cumsum(k ** -s)
    cdf /= cdf[-1]
    u = uniform01(seed, 0, n)
    return (np.searchsorted(cdf, u, side="right") + 1).clip(1, kmax).astype(np.int64)


def zipf_mean(s: float = 1.2, kmax: int = 512) -> float:
    k = np.arange(1, kmax + 1, dtype=np.float64)
    w = k ** -s
    return float((k * w).sum() / w.sum())


def scattered_slots(seed: int, n_slots: int, count: int, first: int = 0) -> np.ndarray:
    """``count`` distinct slots of 0..n_slots-1 by partial Fisher-Yates (no replacement).

    Step i swaps position i with i + (x_i mod (n_slots - i)), x_i = output
    ``first + i`` of stream ``seed``; the modulo bias is below 2^-40 here.
    """
    if count > n_slots:
        raise ValueError("count > n_slots")
    perm = np.arange(n_slots, dtype=np.int64)
    x = splitmix64(seed, first, count)
    span = (n_slots - np.arange(count, dtype=np.int64)).astype(np.uint64)
    off = (x % span).astype(np.int64)
    for i in range(count):
        j = i + off[i]
        perm[i], perm[j] = perm[j], perm[i]
    return perm[:count].copy()


def poisson_arrivals(seed: int, n: int, rate_per_s: float) -> np.ndarray:
    """Arrival times in seconds of a Poisson process with ``rate_per_s`` events/s."""
    u = uniform01(seed, 0, n)
    return np.cumsum(-np.log1p(-u) / rate_per_s)


def batching_workload(seed: int = 3, n_requests: int = 20000, n_slots: int = 2097152,
                      s: float = 1.2, kmax: int = 512):
    """Batching workload: Zipf request sizes, pages scattered without replacement.

    Returns (sizes, slots, ops): ``slots`` is the concatenation of every
    request's page slots (page_id = slot), ``ops`` is 0 (encrypt) or 1
    (decrypt) per request, drawn with p = 1/2.  Independent sub-streams are
    taken from ``seed`` by offsetting the SplitMix64 counter.
    """
    sizes = zipf_sizes(seed, n_requests, s, kmax)
    total = int(sizes.sum())
    slots = scattered_slots(seed ^ 0x5A5A5A5A, n_slots, total)
    ops = (splitmix64(seed ^ 0xA5A5A5A5, 0, n_requests) >> np.uint64(63)).astype(np.int32)
    return sizes, slots, ops


def serving_workload(seed: int, n_requests: int, page_rate: float, n_pages_ws: int,
                     p_fault: float = 0.8, evict_lo: int = 8, evict_hi: int = 64):
    """Serving workload: Poisson arrivals, 80 % 1-page decrypts, 20 % U{8..64}-page encrypts.

    Returns (arrival_s, ops, offsets, pages): request r touches
    ``pages[offsets[r]:offsets[r + 1]]`` (page indices into the working set,
    uniform, distinct within a request).  Mean pages per request is
    p_fault * 1 + (1 - p_fault) * (evict_lo + evict_hi) / 2 = 8.0, so the
    request rate is page_rate / 8.
    """
    mean_pages = p_fault + (1 - p_fault) * (evict_lo + evict_hi) / 2
    arrival = poisson_arrivals(seed, n_requests, page_rate / mean_pages)
    u = uniform01(seed ^ 0x1111, 0, n_requests)
    is_fault = u < p_fault
    span = evict_hi - evict_lo + 1
    ev = evict_lo + (splitmix64(seed ^ 0x2222, 0, n_requests) % np.uint64(span)).astype(np.int64)
    sizes = np.where(is_fault, 1, ev).astype(np.int64)
    ops = np.where(is_fault, 1, 0).astype(np.int32)  # 1 = decrypt (fault), 0 = encrypt (evict)
    offsets = np.zeros(n_requests + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    raw = splitmix64(seed ^ 0x3333, 0, int(offsets[-1])) % np.uint64(n_pages_ws)
    pages = raw.astype(np.int64)
    # distinct within a request: re-draw duplicates deterministically (rare at 4 Mi pages)
    for r in np.nonzero(sizes > 1)[0]:
        a, b = offsets[r], offsets[r + 1]
        seg = pages[a:b]
        if len(np.unique(seg)) != len(seg):
            seen = set()
            for i in range(len(seg)):
                v = int(seg[i])
                while v in seen:
                    v = (v + 1) % n_pages_ws
                seen.add(v)
                seg[i] = v
    return arrival, ops, offsets, pages


def window_trace(seed: int, n_pages: int, length: int, hot_frac: float = 0.6, zipf_s: float = 1.1) -> np.ndarray:
    """Page-access trace of one synthetic client, for the sliding-window driver.

    Each access is, with probability ``hot_frac``, a Zipf(zipf_s)-ranked page
    of a seeded permutation of the client's pages (a hot set) and otherwise
    the next page of a sequential scan that wraps around (streaming access).
    Page numbers are relative to the client's first page.
    """
    u = uniform01(seed, 0, length)
    k = np.arange(1, n_pages + 1, dtype=np.float64)
    cdf = np.cumsum(k ** -zipf_s)
    cdf /= cdf[-1]
    rank = np.searchsorted(cdf, uniform01(seed ^ 0x7777, 0, length), side="right").clip(0, n_pages - 1)
    perm = (splitmix64(seed ^ 0x9999, 0, n_pages)).argsort()
    hot = u < hot_frac
    start = int(splitmix64(seed ^ 0x5555, 0, 1)[0] % np.uint64(n_pages))
    scan = (start + np.cumsum(~hot) - 1) % n_pages
    return np.where(hot, perm[rank], scan).astype(np.uint64)
