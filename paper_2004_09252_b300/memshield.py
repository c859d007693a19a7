"""Thin ctypes binding of libmemshield.so (the C ABI in include/memshield.h).

Argument marshalling only: every step of the page cipher runs in the CUDA
library.  Functions keep the C names; pointers are passed as Python ints
(``tensor.data_ptr()``, ``ndarray.ctypes.data``) and errors become
``MemShieldError``.  Importing this module loads the library and fails loudly
if it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MS_PAGE_BYTES = 4096
MS_BLOCKS_PER_PAGE = 64
MS_KEY_BYTES = 32
MS_OK, MS_EINVAL, MS_ENOTINIT, MS_ENOMEM, MS_ECUDA, MS_ETIMEDOUT, MS_EBUSY, MS_ERANGE = 0, -1, -2, -3, -4, -5, -6, -7
MS_ESTARVED = -8
MS_ENCRYPT, MS_DECRYPT = 0, 1
MS_NOALLOC_MAX_PAGES = 16384
MS_TICKETS = 4096
MS_BATCH_MAX_CAPACITY = 1 << 26
MS_FAULT_LAUNCH, MS_FAULT_COPY, MS_FAULT_GRAPH, MS_FAULT_SERVER = 1, 2, 4, 8

PAGE_DTYPE = np.dtype([("addr", "<u8"), ("page_id", "<u8")])
PAGE_DOM_DTYPE = np.dtype([("addr", "<u8"), ("page_id", "<u8"), ("domain", "<u4"), ("reserved0", "<u4"),
                           ("reserved1", "<u8")])


class MemShieldError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class ms_config(ctypes.Structure):
    _fields_ = [
        ("device", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("domain", ctypes.c_uint32),
        ("rounds", ctypes.c_uint32),
        ("list_capacity", ctypes.c_uint32),
        ("timeout_ms", ctypes.c_uint32),
        ("blocks_per_thread", ctypes.c_uint32),
        ("threads_per_cta", ctypes.c_uint32),
        ("dr_unroll", ctypes.c_uint32),
        ("check_duplicates", ctypes.c_uint32),
        ("use_stream", ctypes.c_uint32),
    ]


class ms_shape(ctypes.Structure):
    _fields_ = [
        ("blocks_per_thread", ctypes.c_uint32),
        ("threads_per_cta", ctypes.c_uint32),
        ("dr_unroll", ctypes.c_uint32),
        ("rot_policy", ctypes.c_uint32),
        ("hoist", ctypes.c_uint32),
    ]


class ms_batch_config(ctypes.Structure):
    _fields_ = [
        ("capacity", ctypes.c_uint32),
        ("use_graph", ctypes.c_uint32),
        ("grab", ctypes.c_uint32),
        ("ctas_per_sm", ctypes.c_uint32),
        ("per_page_domain", ctypes.c_uint32),
    ]


class ms_batch_stats(ctypes.Structure):
    _fields_ = [
        ("requests", ctypes.c_uint64),
        ("pages", ctypes.c_uint64),
        ("submits", ctypes.c_uint64),
        ("graph_launches", ctypes.c_uint64),
    ]


class ms_tune_result(ctypes.Structure):
    _fields_ = [
        ("shape", ms_shape),
        ("k1_gbs", ctypes.c_double),
        ("grab", ctypes.c_uint32),
        ("ctas_per_sm", ctypes.c_uint32),
        ("queue_gbs", ctypes.c_double),
        ("tried", ctypes.c_uint32),
    ]


class ms_server_config(ctypes.Structure):
    _fields_ = [
        ("staging_bytes", ctypes.c_uint64),
        ("max_wave_pages", ctypes.c_uint32),
        ("waves_in_flight", ctypes.c_uint32),
        ("copy_threads", ctypes.c_uint32),
        ("max_pending", ctypes.c_uint32),
        ("mode", ctypes.c_uint32),
        ("zero_staging", ctypes.c_uint32),
        ("max_request_pages", ctypes.c_uint32),
        ("idle_spin_us", ctypes.c_uint32),
        ("zero_copy_max_pages", ctypes.c_uint32),
    ]


class ms_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("requests_done", "pages_done", "waves", "max_wave_requests",
                                               "max_wave_pages", "conflict_waits", "budget_waits",
                                               "max_staged_pages", "gather_ns", "scatter_ns", "inplace_waves",
                                               "staged_waves", "max_pass_ns", "replay_max_lag_ns",
                                               "replay_late")]


MS_SERVE_CONTINUOUS, MS_SERVE_ONE_PER_LAUNCH, MS_SERVE_ZERO_COPY = 0, 1, 2


class ms_window_config(ctypes.Structure):
    _fields_ = [("window_pages", ctypes.c_uint32), ("evict_batch", ctypes.c_uint32),
                ("background_free", ctypes.c_uint32), ("sync_evict", ctypes.c_uint32)]


class ms_window_client(ctypes.Structure):
    _fields_ = [("domain", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("first_page", ctypes.c_uint64),
                ("n_pages", ctypes.c_uint64), ("trace", ctypes.c_void_p), ("trace_len", ctypes.c_uint64)]


class ms_window_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("accesses", "hits", "faults", "evictions", "evict_requests",
                                               "final_window_pages")] + \
               [(n, ctypes.c_double) for n in ("fault_p50_us", "fault_p99_us", "fault_max_us", "elapsed_s")] + \
               [(n, ctypes.c_uint64) for n in ("background_evictions", "background_requests")]


class ms_feed_config(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_uint32), ("chunk", ctypes.c_uint32), ("wait_ms", ctypes.c_uint32),
                ("grab", ctypes.c_uint32)]


class ms_feed_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("requests", "pages", "publications", "grid", "runs", "closes")]


class ms_pipe_rate(ctypes.Structure):
    _fields_ = [("op_class", ctypes.c_int32), ("reserved", ctypes.c_int32), ("lanes_per_sm_clk", ctypes.c_double),
                ("sm_mhz", ctypes.c_double), ("tops", ctypes.c_double)]


PIPE_CLASSES = ("add", "xor", "shf", "prmt", "mad", "mulhi", "xor+mad", "shf+mad", "xor+add", "xor+shf")


class ms_resident_config(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_uint32), ("ring_entries", ctypes.c_uint32), ("idle_exit_us", ctypes.c_uint32),
                ("max_run_ms", ctypes.c_uint32)]


class ms_resident_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("requests", "launches", "max_run_exits", "workers_running",
                                                "replay_max_lag_ns")]


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        if os.environ.get("MEMSHIELD_NO_BUILD"):
            raise ImportError(f"libmemshield.so not built at {path}")
        _build.build()
    elif _build.needs_build() and not os.environ.get("MEMSHIELD_NO_BUILD"):
        _build.build()
    lib = ctypes.CDLL(path)
    P, S, I, U64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint64
    sig = {
        "ms_config_default": (None, [ctypes.POINTER(ms_config)]),
        "ms_init": (I, [ctypes.POINTER(P), P, ctypes.POINTER(ms_config)]),
        "ms_encrypt_pages": (I, [P, P, S]),
        "ms_decrypt_pages": (I, [P, P, S]),
        "ms_encrypt_pages_dev": (I, [P, P, S]),
        "ms_decrypt_pages_dev": (I, [P, P, S]),
        "ms_crypt_range": (I, [P, I, P, U64, S]),
        "ms_sync": (I, [P]),
        "ms_sync_for": (I, [P, ctypes.c_uint32]),
        "ms_shutdown": (I, [P]),
        "ms_strerror": (ctypes.c_char_p, [I]),
        "ms_last_cuda_error": (I, [P]),
        "ms_debug_inject_fault": (I, [I, I, I]),
        "ms_crypt_host": (I, [P, I, P, U64, S, S, I]),
        "ms_crypt_host_inplace": (I, [P, I, P, U64, S]),
        "ms_get_shape": (I, [P, ctypes.POINTER(ms_shape)]),
        "ms_set_shape": (I, [P, ctypes.POINTER(ms_shape)]),
        "ms_crypt_pages_noalloc": (I, [P, I, P, S]),
        "ms_batch_config_default": (None, [ctypes.POINTER(ms_batch_config)]),
        "ms_batch_create": (I, [P, ctypes.POINTER(ms_batch_config), ctypes.POINTER(P)]),
        "ms_batch_add": (I, [P, I, P, S]),
        "ms_batch_add_dom": (I, [P, I, P, S]),
        "ms_batch_submit": (I, [P]),
        "ms_batch_add_requests": (I, [P, S, P, P, P, ctypes.POINTER(ctypes.c_size_t)]),
        "ms_batch_get_stats": (I, [P, ctypes.POINTER(ms_batch_stats)]),
        "ms_batch_destroy": (I, [P]),
        "ms_autotune": (I, [P, S, ctypes.POINTER(ms_tune_result)]),
        "ms_server_config_default": (None, [ctypes.POINTER(ms_server_config)]),
        "ms_server_create": (I, [P, P, U64, ctypes.POINTER(ms_server_config), ctypes.POINTER(P)]),
        "ms_server_submit": (I, [P, I, P, ctypes.c_uint32, ctypes.POINTER(U64)]),
        "ms_server_poll": (I, [P, U64]),
        "ms_server_wait": (I, [P, U64, ctypes.c_uint32]),
        "ms_server_replay": (I, [P, S, P, P, P, P, P, P, ctypes.POINTER(ctypes.c_double), ctypes.c_uint32]),
        "ms_server_submit_dom": (I, [P, I, ctypes.c_uint32, P, ctypes.c_uint32, ctypes.POINTER(U64)]),
        "ms_crypt_pages_dom": (I, [P, P, S]),
        "ms_resident_config_default": (None, [ctypes.POINTER(ms_resident_config)]),
        "ms_resident_create": (I, [P, ctypes.POINTER(ms_resident_config), ctypes.POINTER(P)]),
        "ms_resident_submit": (I, [P, P, ctypes.POINTER(U64)]),
        "ms_resident_poll": (I, [P, U64]),
        "ms_resident_wait": (I, [P, U64, ctypes.c_uint32]),
        "ms_resident_get_stats": (I, [P, ctypes.POINTER(ms_resident_stats)]),
        "ms_resident_destroy": (I, [P]),
        "ms_resident_replay": (I, [P, P, U64, S, P, P, P, P, P, ctypes.POINTER(ctypes.c_double), ctypes.c_uint32]),
        "ms_window_run": (I, [P, ctypes.POINTER(ms_window_config), ctypes.POINTER(ms_window_client), S,
                              ctypes.POINTER(ms_window_stats), P, ctypes.c_uint32]),
        "ms_probe_int_pipes": (I, [I, ctypes.POINTER(ms_pipe_rate), S]),
        "ms_submit_host": (I, [P, I, P, S, ctypes.POINTER(U64)]),
        "ms_clone": (I, [P, ctypes.c_uint32, ctypes.POINTER(P)]),
        "ms_poll": (I, [P, U64]),
        "ms_wait": (I, [P, U64, ctypes.c_uint32]),
        "ms_host_device_address": (I, [P, ctypes.POINTER(U64)]),
        "ms_feed_config_default": (None, [ctypes.POINTER(ms_feed_config)]),
        "ms_feed_create": (I, [P, ctypes.POINTER(ms_feed_config), ctypes.POINTER(P)]),
        "ms_feed_open": (I, [P]),
        "ms_feed_add_requests": (I, [P, S, P, P, P, ctypes.POINTER(ctypes.c_size_t)]),
        "ms_feed_close": (I, [P]),
        "ms_feed_get_stats": (I, [P, ctypes.POINTER(ms_feed_stats)]),
        "ms_feed_destroy": (I, [P]),
        "ms_window_run_ticketed": (I, [P, P, U64, ctypes.POINTER(ms_window_config), ctypes.POINTER(ms_window_client),
                                       S, ctypes.POINTER(ms_window_stats), P, ctypes.c_uint32]),
        "ms_window_run_resident": (I, [P, P, U64, ctypes.POINTER(ms_window_config), ctypes.POINTER(ms_window_client),
                                       S, ctypes.POINTER(ms_window_stats), P, ctypes.c_uint32]),
        "ms_crypt_pages_dom_dev": (I, [P, P, S]),
        "ms_server_get_stats": (I, [P, ctypes.POINTER(ms_server_stats)]),
        "ms_server_destroy": (I, [P]),
        "ms_tune_save": (I, [P, ctypes.c_char_p]),
        "ms_tune_load": (I, [P, ctypes.c_char_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
lib = _lib


def strerror(code: int) -> str:
    return _lib.ms_strerror(code).decode()


def _check(code: int, where: str) -> int:
    if code != MS_OK:
        raise MemShieldError(code, where)
    return code


def inject_fault(site_mask: int, countdown: int = 0, cuda_error: int = 719) -> None:
    """Arm a one-shot host-side failure (719 = cudaErrorLaunchFailure by default)."""
    _check(_lib.ms_debug_inject_fault(site_mask, countdown, cuda_error), "ms_debug_inject_fault")


def config_default() -> ms_config:
    cfg = ms_config()
    _lib.ms_config_default(ctypes.byref(cfg))
    return cfg


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def host_device_address(host_base) -> int:
    """Device address of pinned, mapped host memory (ms_host_device_address)."""
    a = ctypes.c_uint64()
    _check(_lib.ms_host_device_address(_ptr(host_base), ctypes.byref(a)), "ms_host_device_address")
    return a.value


def probe_int_pipes(device: int = 0) -> list[dict]:
    """Sustained lane operations per SM per clock of the cipher's integer op
    classes on `device` (ms_probe_int_pipes)."""
    arr = (ms_pipe_rate * len(PIPE_CLASSES))()
    _check(_lib.ms_probe_int_pipes(device, arr, len(PIPE_CLASSES)), "ms_probe_int_pipes")
    return [{"class": PIPE_CLASSES[r.op_class], "lanes_per_sm_clk": round(r.lanes_per_sm_clk, 2),
             "sm_mhz": round(r.sm_mhz, 1), "tops": round(r.tops, 3)} for r in arr]


def pages_dom_array(addrs, page_ids, domains) -> np.ndarray:
    """Pack (addr, page_id, domain) triples into the 32-byte ms_page_dom layout."""
    a = np.zeros(len(addrs), dtype=PAGE_DOM_DTYPE)
    a["addr"] = np.asarray(addrs, dtype=np.uint64)
    a["page_id"] = np.asarray(page_ids, dtype=np.uint64)
    a["domain"] = np.asarray(domains, dtype=np.uint32)
    return a


def pages_array(addrs, page_ids) -> np.ndarray:
    """Pack (addr, page_id) pairs into the 16-byte ms_page layout."""
    a = np.empty(len(addrs), dtype=PAGE_DTYPE)
    a["addr"] = np.asarray(addrs, dtype=np.uint64)
    a["page_id"] = np.asarray(page_ids, dtype=np.uint64)
    return a


class Context:
    """An ms_ctx: the key on one device plus the stream the work runs on."""

    def __init__(self, key: bytes | None = None, *, device: int = -1, stream=None, domain: int = 0,
                 rounds: int = 20, list_capacity: int = 0, timeout_ms: int = 0,
                 blocks_per_thread: int = 0, threads_per_cta: int = 0, dr_unroll: int = 0,
                 check_duplicates: bool = False):
        cfg = config_default()
        cfg.device = device
        if stream is not None:
            # an explicit stream, including handle 0 (the legacy default stream)
            cfg.stream = stream if isinstance(stream, int) else stream.cuda_stream
            cfg.use_stream = 1
        cfg.domain = domain
        cfg.rounds = rounds
        if list_capacity:
            cfg.list_capacity = list_capacity
        if timeout_ms:
            cfg.timeout_ms = timeout_ms
        cfg.blocks_per_thread = blocks_per_thread
        cfg.threads_per_cta = threads_per_cta
        cfg.dr_unroll = dr_unroll
        cfg.check_duplicates = 1 if check_duplicates else 0
        h = ctypes.c_void_p()
        kb = None
        if key is not None:
            if len(key) != MS_KEY_BYTES:
                raise ValueError("key must be 32 bytes")
            kb = ctypes.create_string_buffer(bytes(key), MS_KEY_BYTES)
        _check(_lib.ms_init(ctypes.byref(h), kb, ctypes.byref(cfg)), "ms_init")
        if kb is not None:
            ctypes.memset(kb, 0, MS_KEY_BYTES)
        self.handle = h.value
        self.cfg = cfg

    def clone(self, domain: int) -> "Context":
        """ms_clone: the same key (device to device), another domain, its own stream."""
        h = ctypes.c_void_p()
        _check(_lib.ms_clone(self.handle, domain, ctypes.byref(h)), "ms_clone")
        c = Context.__new__(Context)
        c.handle = h.value
        c.cfg = None
        return c

    # -- one-launch forms
    def encrypt_pages(self, pages: np.ndarray) -> None:
        pages = np.ascontiguousarray(pages, dtype=PAGE_DTYPE)
        _check(_lib.ms_encrypt_pages(self.handle, pages.ctypes.data, pages.size), "ms_encrypt_pages")

    def decrypt_pages(self, pages: np.ndarray) -> None:
        pages = np.ascontiguousarray(pages, dtype=PAGE_DTYPE)
        _check(_lib.ms_decrypt_pages(self.handle, pages.ctypes.data, pages.size), "ms_decrypt_pages")

    def encrypt_pages_dev(self, d_pages, n: int) -> None:
        _check(_lib.ms_encrypt_pages_dev(self.handle, _ptr(d_pages), n), "ms_encrypt_pages_dev")

    def decrypt_pages_dev(self, d_pages, n: int) -> None:
        _check(_lib.ms_decrypt_pages_dev(self.handle, _ptr(d_pages), n), "ms_decrypt_pages_dev")

    def crypt_pages_dom(self, pages: np.ndarray) -> None:
        pages = np.ascontiguousarray(pages, dtype=PAGE_DOM_DTYPE)
        _check(_lib.ms_crypt_pages_dom(self.handle, pages.ctypes.data, pages.size), "ms_crypt_pages_dom")

    def crypt_pages_dom_dev(self, d_pages, n: int) -> None:
        _check(_lib.ms_crypt_pages_dom_dev(self.handle, _ptr(d_pages), n), "ms_crypt_pages_dom_dev")

    def crypt_range(self, op: int, d_base, first_page_id: int, n_pages: int) -> None:
        _check(_lib.ms_crypt_range(self.handle, op, _ptr(d_base), first_page_id, n_pages), "ms_crypt_range")

    def crypt_host(self, op: int, host_base, first_page_id: int, n_pages: int, chunk_bytes: int = 0,
                   n_streams: int = 0) -> None:
        _check(_lib.ms_crypt_host(self.handle, op, _ptr(host_base), first_page_id, n_pages, chunk_bytes,
                                  n_streams), "ms_crypt_host")

    def crypt_host_inplace(self, op: int, host_base, first_page_id: int, n_pages: int) -> None:
        """In place on pinned, mapped host pages over the host link (asynchronous; sync waits)."""
        _check(_lib.ms_crypt_host_inplace(self.handle, op, _ptr(host_base), first_page_id, n_pages),
               "ms_crypt_host_inplace")

    def crypt_pages_noalloc(self, op: int, pages: np.ndarray) -> None:
        """Same transform as encrypt_pages, with no allocation in the call (waits for completion)."""
        pages = np.ascontiguousarray(pages, dtype=PAGE_DTYPE)
        _check(_lib.ms_crypt_pages_noalloc(self.handle, op, pages.ctypes.data, pages.size),
               "ms_crypt_pages_noalloc")

    def autotune(self, sample_pages: int = 0) -> dict:
        r = ms_tune_result()
        _check(_lib.ms_autotune(self.handle, sample_pages, ctypes.byref(r)), "ms_autotune")
        return {"shape": {f: getattr(r.shape, f) for f, _ in ms_shape._fields_}, "k1_gbs": r.k1_gbs,
                "grab": r.grab, "ctas_per_sm": r.ctas_per_sm, "queue_gbs": r.queue_gbs, "tried": r.tried}

    def tune_save(self, path: str) -> None:
        _check(_lib.ms_tune_save(self.handle, path.encode()), "ms_tune_save")

    def tune_load(self, path: str) -> int:
        return _lib.ms_tune_load(self.handle, path.encode())

    def batch(self, capacity: int = 0, use_graph: bool = True, grab: int = 0, ctas_per_sm: int = 0,
              per_page_domain: bool = False) -> "Batch":
        return Batch(self, capacity, use_graph, grab, ctas_per_sm, per_page_domain)

    def submit_host(self, op: int, pages: np.ndarray) -> int:
        """Queue one host list; returns its ticket (ms_submit_host)."""
        pages = np.ascontiguousarray(pages, dtype=PAGE_DTYPE)
        t = ctypes.c_uint64()
        _check(_lib.ms_submit_host(self.handle, op, pages.ctypes.data, pages.size, ctypes.byref(t)), "ms_submit_host")
        return t.value

    def poll(self, ticket: int) -> int:
        """1 done, 0 pending, < 0 an error code."""
        return _lib.ms_poll(self.handle, ticket)

    def wait(self, ticket: int, timeout_ms: int = 10000) -> None:
        _check(_lib.ms_wait(self.handle, ticket, timeout_ms), "ms_wait")

    def run_window_clients(self, host_base, n_pages: int, window_pages: int, evict_batch: int, clients,
                           timeout_ms: int = 60000, background_free: int = 0, sync_evict: bool = False):
        """Sliding-window clients served by ticketed launches, one clone of this
        context per client (its domain, its stream), in place on a pinned, mapped
        working set."""
        base = _ptr(host_base)
        return _run_window(lambda cfg, arr, n, st, fw: _lib.ms_window_run_ticketed(
            self.handle, base, n_pages, cfg, arr, n, st, fw, timeout_ms),
            "ms_window_run_ticketed", window_pages, evict_batch, clients, background_free, sync_evict)

    def feed(self, capacity: int = 0, chunk: int = 0, wait_ms: int = 0, grab: int = 0) -> "Feed":
        return Feed(self, capacity, chunk, wait_ms, grab)

    def get_shape(self) -> dict:
        sh = ms_shape()
        _check(_lib.ms_get_shape(self.handle, ctypes.byref(sh)), "ms_get_shape")
        return {f: getattr(sh, f) for f, _ in ms_shape._fields_}

    def set_shape(self, blocks_per_thread: int, threads_per_cta: int, dr_unroll: int, rot_policy: int,
                  hoist: int = 0) -> None:
        sh = ms_shape(blocks_per_thread, threads_per_cta, dr_unroll, rot_policy, hoist)
        _check(_lib.ms_set_shape(self.handle, ctypes.byref(sh)), "ms_set_shape")

    def sync(self) -> int:
        return _lib.ms_sync(self.handle)

    def sync_for(self, timeout_ms: int) -> int:
        return _lib.ms_sync_for(self.handle, timeout_ms)

    def sync_checked(self) -> None:
        _check(self.sync(), "ms_sync")

    def last_cuda_error(self) -> int:
        return _lib.ms_last_cuda_error(self.handle)

    def shutdown(self) -> int:
        """ms_shutdown; the handle stays valid when it returns MS_EBUSY (children
        alive) or MS_ETIMEDOUT (queued work still running)."""
        if self.handle:
            rc = _lib.ms_shutdown(self.handle)
            if rc not in (MS_EBUSY, MS_ETIMEDOUT):
                self.handle = None
            return rc
        return MS_OK

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.shutdown()

    def __del__(self):
        try:
            self.shutdown()
        except Exception:
            pass


class Feed:
    """An ms_feed: one persistent kernel drains a device queue the host is still
    filling.  Created closed; open() starts a run, close() ends it."""

    def __init__(self, ctx: Context, capacity: int = 0, chunk: int = 0, wait_ms: int = 0, grab: int = 0):
        cfg = ms_feed_config()
        _lib.ms_feed_config_default(ctypes.byref(cfg))
        if capacity:
            cfg.capacity = capacity
        if chunk:
            cfg.chunk = chunk
        if wait_ms:
            cfg.wait_ms = wait_ms
        cfg.grab = grab
        h = ctypes.c_void_p()
        _check(_lib.ms_feed_create(ctx.handle, ctypes.byref(cfg), ctypes.byref(h)), "ms_feed_create")
        self.handle = h.value
        self.ctx = ctx

    def open(self) -> "Feed":
        _check(_lib.ms_feed_open(self.handle), "ms_feed_open")
        return self

    def add_requests(self, ops: np.ndarray, offsets: np.ndarray, pages: np.ndarray, first: int = 0,
                     count: int | None = None) -> int:
        """Append requests first..first+count-1 of a request table; returns how many were appended."""
        ops = np.ascontiguousarray(ops, dtype=np.int32)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        pages = np.ascontiguousarray(pages, dtype=PAGE_DTYPE)
        n = (len(ops) - first) if count is None else count
        added = ctypes.c_size_t(0)
        _check(_lib.ms_feed_add_requests(self.handle, n, ops.ctypes.data + 4 * first, offsets.ctypes.data + 8 * first,
                                         pages.ctypes.data, ctypes.byref(added)), "ms_feed_add_requests")
        return added.value

    def close(self) -> None:
        _check(_lib.ms_feed_close(self.handle), "ms_feed_close")

    def stats(self) -> dict:
        st = ms_feed_stats()
        _check(_lib.ms_feed_get_stats(self.handle, ctypes.byref(st)), "ms_feed_get_stats")
        return {f: getattr(st, f) for f, _ in ms_feed_stats._fields_}

    def destroy(self) -> int:
        if self.handle:
            rc = _lib.ms_feed_destroy(self.handle)
            if rc != MS_ETIMEDOUT:  # still in use on the GPU: the handle stays valid, call again
                self.handle = None
            return rc
        return MS_OK

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()


class Batch:
    """An ms_batch: requests queued on the host, drained on the GPU by the persistent kernel."""

    def __init__(self, ctx: Context, capacity: int = 0, use_graph: bool = True, grab: int = 0,
                 ctas_per_sm: int = 0, per_page_domain: bool = False):
        cfg = ms_batch_config()
        _lib.ms_batch_config_default(ctypes.byref(cfg))
        if capacity:
            cfg.capacity = capacity
        cfg.use_graph = 1 if use_graph else 0
        cfg.grab = grab
        cfg.ctas_per_sm = ctas_per_sm
        cfg.per_page_domain = 1 if per_page_domain else 0
        h = ctypes.c_void_p()
        _check(_lib.ms_batch_create(ctx.handle, ctypes.byref(cfg), ctypes.byref(h)), "ms_batch_create")
        self.handle = h.value
        self.ctx = ctx

    def add(self, op: int, pages: np.ndarray) -> int:
        """Queue one request; returns the status code (MS_EBUSY when full) without raising for it."""
        pages = np.ascontiguousarray(pages, dtype=PAGE_DTYPE)
        rc = _lib.ms_batch_add(self.handle, op, pages.ctypes.data, pages.size)
        if rc not in (MS_OK, MS_EBUSY):
            raise MemShieldError(rc, "ms_batch_add")
        return rc

    def add_dom(self, op: int, pages: np.ndarray) -> int:
        """Queue one request with a domain per page; returns the status (MS_EBUSY when full)."""
        pages = np.ascontiguousarray(pages, dtype=PAGE_DOM_DTYPE)
        rc = _lib.ms_batch_add_dom(self.handle, op, pages.ctypes.data, pages.size)
        if rc not in (MS_OK, MS_EBUSY):
            raise MemShieldError(rc, "ms_batch_add_dom")
        return rc

    def add_requests(self, ops: np.ndarray, offsets: np.ndarray, pages: np.ndarray, first: int = 0,
                     count: int | None = None) -> tuple[int, int]:
        """Queue requests first..first+count-1 of a request table; returns (status, queued)."""
        ops = np.ascontiguousarray(ops, dtype=np.int32)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        pages = np.ascontiguousarray(pages, dtype=PAGE_DTYPE)
        n = (len(ops) - first) if count is None else count
        added = ctypes.c_size_t(0)
        rc = _lib.ms_batch_add_requests(self.handle, n, ops.ctypes.data + 4 * first,
                                        offsets.ctypes.data + 8 * first, pages.ctypes.data,
                                        ctypes.byref(added))
        if rc not in (MS_OK, MS_EBUSY):
            raise MemShieldError(rc, "ms_batch_add_requests")
        return rc, added.value

    def submit(self) -> None:
        _check(_lib.ms_batch_submit(self.handle), "ms_batch_submit")

    def stats(self) -> dict:
        st = ms_batch_stats()
        _check(_lib.ms_batch_get_stats(self.handle, ctypes.byref(st)), "ms_batch_get_stats")
        return {f: getattr(st, f) for f, _ in ms_batch_stats._fields_}

    def destroy(self) -> int:
        if self.handle:
            rc = _lib.ms_batch_destroy(self.handle)
            if rc != MS_ETIMEDOUT:  # still in use on the GPU: the handle stays valid, call again
                self.handle = None
            return rc
        return MS_OK

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()


class Server:
    """An ms_server: continuous batching of page requests over a host working set."""

    def __init__(self, ctx: Context, host_base, n_pages: int, *, staging_bytes: int = 0, max_wave_pages: int = 0,
                 waves_in_flight: int = 0, copy_threads: int | None = None, max_pending: int = 0,
                 mode: int = MS_SERVE_CONTINUOUS, zero_staging: bool = False, max_request_pages: int = 0,
                 idle_spin_us: int | None = None, zero_copy_max_pages: int | None = None):
        cfg = ms_server_config()
        _lib.ms_server_config_default(ctypes.byref(cfg))
        if staging_bytes:
            cfg.staging_bytes = staging_bytes
        if max_wave_pages:
            cfg.max_wave_pages = max_wave_pages
        if waves_in_flight:
            cfg.waves_in_flight = waves_in_flight
        if copy_threads is not None:
            cfg.copy_threads = copy_threads
        if max_pending:
            cfg.max_pending = max_pending
        cfg.mode = mode
        cfg.zero_staging = 1 if zero_staging else 0
        if max_request_pages:
            cfg.max_request_pages = max_request_pages
        if idle_spin_us is not None:
            cfg.idle_spin_us = idle_spin_us
        if zero_copy_max_pages is not None:
            cfg.zero_copy_max_pages = zero_copy_max_pages
        h = ctypes.c_void_p()
        _check(_lib.ms_server_create(ctx.handle, _ptr(host_base), n_pages, ctypes.byref(cfg), ctypes.byref(h)),
               "ms_server_create")
        self.handle = h.value
        self.ctx = ctx

    def submit(self, op: int, page_index, domain: int | None = None) -> int:
        idx = np.ascontiguousarray(page_index, dtype=np.uint64)
        t = ctypes.c_uint64()
        if domain is None:
            rc = _lib.ms_server_submit(self.handle, op, idx.ctypes.data, idx.size, ctypes.byref(t))
        else:
            rc = _lib.ms_server_submit_dom(self.handle, op, domain, idx.ctypes.data, idx.size, ctypes.byref(t))
        _check(rc, "ms_server_submit")
        return t.value

    def poll(self, ticket: int) -> int:
        return _lib.ms_server_poll(self.handle, ticket)

    def wait(self, ticket: int, timeout_ms: int = 10000) -> None:
        _check(_lib.ms_server_wait(self.handle, ticket, timeout_ms), "ms_server_wait")

    def replay(self, arrival_s, ops, offsets, page_index, timeout_ms: int = 60000, domains=None):
        """Open-loop replay; returns (latency_s array, makespan_s)."""
        arrival_s = np.ascontiguousarray(arrival_s, dtype=np.float64)
        ops = np.ascontiguousarray(ops, dtype=np.int32)
        dom = None if domains is None else np.ascontiguousarray(domains, dtype=np.uint32)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        page_index = np.ascontiguousarray(page_index, dtype=np.uint64)
        lat = np.empty(arrival_s.size, dtype=np.float64)
        mk = ctypes.c_double()
        _check(_lib.ms_server_replay(self.handle, arrival_s.size, arrival_s.ctypes.data, ops.ctypes.data,
                                     None if dom is None else dom.ctypes.data,
                                     offsets.ctypes.data, page_index.ctypes.data, lat.ctypes.data,
                                     ctypes.byref(mk), timeout_ms), "ms_server_replay")
        return lat, mk.value

    def run_window_clients(self, window_pages: int, evict_batch: int, clients, timeout_ms: int = 60000,
                           background_free: int = 0, sync_evict: bool = False):
        """Sliding-window clients: `clients` is a list of (domain, first_page, n_pages, trace).
        background_free = T > 0 adds a background evictor per client that keeps T
        window slots free; sync_evict makes each client wait for its own overflow
        evictions.  Returns (per-client stats dicts, per-client final windows as
        lists of page indices)."""
        return _run_window(lambda cfg, arr, n, st, fw: _lib.ms_window_run(self.handle, cfg, arr, n, st, fw, timeout_ms),
                           "ms_window_run", window_pages, evict_batch, clients, background_free, sync_evict)

    def stats(self) -> dict:
        st = ms_server_stats()
        _check(_lib.ms_server_get_stats(self.handle, ctypes.byref(st)), "ms_server_get_stats")
        return {f: getattr(st, f) for f, _ in ms_server_stats._fields_}

    def destroy(self) -> int:
        if self.handle:
            rc = _lib.ms_server_destroy(self.handle)
            if rc != MS_ETIMEDOUT:  # still in use on the GPU: the handle stays valid, call again
                self.handle = None
            return rc
        return MS_OK

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()


def _run_window(call, name: str, window_pages: int, evict_batch: int, clients, background_free: int = 0,
                sync_evict: bool = False):
    cfg = ms_window_config(window_pages, evict_batch, background_free, 1 if sync_evict else 0)
    arr = (ms_window_client * len(clients))()
    keep = []
    for i, (dom, first, n, trace) in enumerate(clients):
        tr = np.ascontiguousarray(trace, dtype=np.uint64)
        keep.append(tr)
        arr[i] = ms_window_client(dom, 0, first, n, tr.ctypes.data, tr.size)
    st = (ms_window_stats * len(clients))()
    fw = np.empty(len(clients) * (window_pages + 1), dtype=np.uint64)
    _check(call(ctypes.byref(cfg), arr, len(clients), st, fw.ctypes.data), name)
    stats = [{f: getattr(st[i], f) for f, _ in ms_window_stats._fields_} for i in range(len(clients))]
    wins = []
    for i in range(len(clients)):
        w = fw[i * (window_pages + 1):(i + 1) * (window_pages + 1)]
        wins.append([int(x) for x in w if x != np.uint64(0xFFFFFFFFFFFFFFFF)])
    return stats, wins


class Resident:
    """An ms_resident: worker kernels that keep running and take single pages from mapped rings."""

    def __init__(self, ctx: Context, workers: int = 0, ring_entries: int = 0, idle_exit_us: int = 0,
                 max_run_ms: int = 0):
        cfg = ms_resident_config()
        _lib.ms_resident_config_default(ctypes.byref(cfg))
        if workers:
            cfg.workers = workers
        if ring_entries:
            cfg.ring_entries = ring_entries
        if idle_exit_us:
            cfg.idle_exit_us = idle_exit_us
        if max_run_ms:
            cfg.max_run_ms = max_run_ms
        h = ctypes.c_void_p()
        _check(_lib.ms_resident_create(ctx.handle, ctypes.byref(cfg), ctypes.byref(h)), "ms_resident_create")
        self.handle = h.value
        self.ctx = ctx

    def submit(self, addr: int, page_id: int, domain: int = 0) -> int:
        """Queue one page; returns its ticket, or -1 when the worker's ring is full."""
        e = pages_dom_array([addr], [page_id], [domain])
        t = ctypes.c_uint64()
        rc = _lib.ms_resident_submit(self.handle, e.ctypes.data, ctypes.byref(t))
        if rc == MS_EBUSY:
            return -1
        _check(rc, "ms_resident_submit")
        return t.value

    def poll(self, ticket: int) -> int:
        return _lib.ms_resident_poll(self.handle, ticket)

    def wait(self, ticket: int, timeout_ms: int = 10000) -> None:
        _check(_lib.ms_resident_wait(self.handle, ticket, timeout_ms), "ms_resident_wait")

    def stats(self) -> dict:
        st = ms_resident_stats()
        _check(_lib.ms_resident_get_stats(self.handle, ctypes.byref(st)), "ms_resident_get_stats")
        return {f: getattr(st, f) for f, _ in ms_resident_stats._fields_}

    def replay(self, host_base, n_pages: int, arrival_s, offsets, page_index, domains=None, timeout_ms: int = 60000):
        arrival_s = np.ascontiguousarray(arrival_s, dtype=np.float64)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        page_index = np.ascontiguousarray(page_index, dtype=np.uint64)
        dom = None if domains is None else np.ascontiguousarray(domains, dtype=np.uint32)
        lat = np.empty(arrival_s.size, dtype=np.float64)
        mk = ctypes.c_double()
        _check(_lib.ms_resident_replay(self.handle, _ptr(host_base), n_pages, arrival_s.size, arrival_s.ctypes.data,
                                       None if dom is None else dom.ctypes.data, offsets.ctypes.data,
                                       page_index.ctypes.data, lat.ctypes.data, ctypes.byref(mk), timeout_ms),
               "ms_resident_replay")
        return lat, mk.value

    def run_window_clients(self, host_base, n_pages: int, window_pages: int, evict_batch: int, clients,
                           timeout_ms: int = 60000, background_free: int = 0, sync_evict: bool = False):
        """The sliding-window clients of Server.run_window_clients, served by these
        workers in place on a pinned, mapped working set of n_pages pages."""
        base = _ptr(host_base)
        return _run_window(lambda cfg, arr, n, st, fw: _lib.ms_window_run_resident(
            self.handle, base, n_pages, cfg, arr, n, st, fw, timeout_ms),
            "ms_window_run_resident", window_pages, evict_batch, clients, background_free, sync_evict)

    def destroy(self) -> int:
        if self.handle:
            rc = _lib.ms_resident_destroy(self.handle)
            if rc != MS_ETIMEDOUT:  # still in use on the GPU: the handle stays valid, call again
                self.handle = None
            return rc
        return MS_OK

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()
