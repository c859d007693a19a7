"""GPU tests of the served form (continuous batching over a pinned host
working set): results match the oracle, each request's result is the same
alone and in the mix, admission respects page conflicts and the budget."""
import numpy as np
import pytest

import oracle
import synth
from helpers import PAGE

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_09252_b300 import memshield
    return memshield


def working_set(seed, n):
    h = torch.empty(n * PAGE, dtype=torch.uint8).pin_memory()
    synth.fill_pages(h.data_ptr(), seed, 0, n)
    return h


def distinct_workload(seed, n_req, n_pages, rate):
    """Serving recipe (80 % 1-page decrypts, 20 % 8..64-page encrypts, Poisson
    arrivals) with every page used by at most one request, so each request's
    output is just its pages' final contents."""
    arrival, ops, offsets, _ = synth.serving_workload(seed, n_req, rate, n_pages)
    total = int(offsets[-1])
    pages = synth.scattered_slots(seed + 7, n_pages, total)
    return arrival, ops, offsets, pages


def oracle_ws(key, plain, pages):
    want = plain.copy()
    oracle.crypt_pages(key, want, pages, pages, threads=8)
    return want


def test_submit_wait_matches_oracle(ms, key1):
    n = 2048
    h = working_set(70, n)
    plain = h.numpy().copy()
    reqs = [(1, [5]), (0, list(range(100, 140))), (1, [2047]), (0, [7, 9, 11, 1000, 3])]
    with ms.Context(key1) as ctx, ms.Server(ctx, h, n) as srv:
        tickets = [srv.submit(op, pg) for op, pg in reqs]
        for t in tickets:
            srv.wait(t)
            assert srv.poll(t) == 1
        st = srv.stats()
    touched = np.array(sorted({p for _, pg in reqs for p in pg}), dtype=np.uint64)
    assert np.array_equal(h.numpy(), oracle_ws(key1, plain, touched))
    assert st["requests_done"] == len(reqs) and st["pages_done"] == len(touched)


@pytest.mark.parametrize("mode,zc_pages,rate", [(0, 0, 2e6), (0, None, 2e6), (0, None, 3e4), (0, 16, 3e4),
                                                (0, 512, 2e5), (1, None, 2e6), (2, None, 2e6)])
def test_alone_equals_mix(ms, key1, mode, zc_pages, rate):
    """Each request's result is identical when served alone (submit, wait, one
    at a time) and when served in an open-loop mix (bit-exact), and both equal
    the oracle; at the lower rates the in-place lane carries waves."""
    n, n_req = 16384, 1500
    arrival, ops, offsets, pages = distinct_workload(71, n_req, n, rate)
    plain = synth.page_bytes_fast(72, 0, n)
    alone = torch.from_numpy(plain.copy()).pin_memory()
    mix = torch.from_numpy(plain.copy()).pin_memory()
    with ms.Context(key1) as ctx:
        with ms.Server(ctx, alone, n) as srv:
            for r in range(n_req):
                srv.wait(srv.submit(int(ops[r]), pages[offsets[r]:offsets[r + 1]]))
        with ms.Server(ctx, mix, n, mode=mode, zero_copy_max_pages=zc_pages) as srv:
            lat, makespan = srv.replay(arrival, ops, offsets, pages)
            st = srv.stats()
    assert (lat >= 0).all() and makespan > 0
    a, b = alone.numpy().reshape(n, PAGE), mix.numpy().reshape(n, PAGE)
    for r in range(n_req):
        sel = pages[offsets[r]:offsets[r + 1]]
        assert np.array_equal(a[sel], b[sel]), f"request {r} differs alone vs mix"
    assert np.array_equal(alone.numpy(), oracle_ws(key1, plain, pages))
    if mode == 1:
        assert st["max_wave_requests"] == 1 and st["waves"] == n_req and st["staged_waves"] == n_req
    elif mode == 2:
        assert st["staged_waves"] == 0                    # no staging copies in zero-copy mode
    else:
        assert st["waves"] <= n_req
        # continuous mode over mapped memory stages only with the lane off
        assert st["staged_waves"] == (st["waves"] if zc_pages == 0 else 0)
    if mode != 0 or zc_pages == 0:                        # the in-place lane is continuous mode's only
        assert st["inplace_waves"] == 0
    elif rate < 1e6:                                      # short queues: the lane carries waves
        assert 0 < st["inplace_waves"] <= st["waves"]


@pytest.mark.parametrize("rounds", [20, 12, 8])
def test_zero_copy_large_waves(ms, key1, rounds):
    """Every request arrives at once, so zero-copy waves hold hundreds to
    thousands of pages: the bounded-grid kernel that works on the mapped
    working set takes several blocks per thread, with a ragged last step.
    The working set equals the oracle's, for each round count."""
    n, n_req = 16384, 1200
    _, ops, offsets, pages = distinct_workload(78, n_req, n, 2e6)
    arrival = np.zeros(n_req)
    plain = synth.page_bytes_fast(79, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    with ms.Context(key1, rounds=rounds) as ctx, ms.Server(ctx, h, n, mode=ms.MS_SERVE_ZERO_COPY) as srv:
        lat, makespan = srv.replay(arrival, ops, offsets, pages)
        st = srv.stats()
    assert (lat >= 0).all() and makespan > 0
    assert st["pages_done"] == int(offsets[-1]) and st["max_wave_pages"] > 256
    want = plain.copy()
    oracle.crypt_pages(key1, want, pages, pages, rounds=rounds, threads=8)
    assert np.array_equal(h.numpy(), want)


def test_conflicting_requests_serialise(ms, key1):
    """Requests on the same pages wait for each other; k applications of the
    same XOR leave p ^ K for odd k and p for even k."""
    n = 256
    h = working_set(73, n)
    plain = h.numpy().copy()
    rng = synth.splitmix64(74, 0, 4000)
    counts = np.zeros(n, dtype=np.int64)
    with ms.Context(key1) as ctx, ms.Server(ctx, h, n, max_request_pages=16) as srv:
        tickets = []
        for r in range(200):
            k = 1 + int(rng[r] % np.uint64(16))
            sel = np.unique((rng[200 + 16 * r:200 + 16 * r + k] % np.uint64(32)).astype(np.int64))
            counts[sel] += 1
            tickets.append(srv.submit(r % 2, sel))
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
    odd = np.nonzero(counts % 2)[0].astype(np.uint64)
    assert np.array_equal(h.numpy(), oracle_ws(key1, plain, odd))
    assert st["conflict_waits"] > 0


@pytest.mark.parametrize("lane", [None, 0])
def test_concurrent_submitters(ms, key1, lane):
    """Four threads submit at once (each ctypes call releases the GIL) on
    overlapping pages, waiting for some of their tickets as they go: the
    inbox takes every request, admission serialises requests that share a
    page, and the final state is the closed form of the application counts,
    with the in-place waves and with every wave staged."""
    import threading
    n, per_thread, n_threads = 256, 300, 4
    h = working_set(84, n)
    plain = h.numpy().copy()
    rng = synth.splitmix64(85, 0, n_threads * per_thread * 17)
    reqs = []
    for th in range(n_threads):
        mine = []
        for r in range(per_thread):
            i = (th * per_thread + r) * 17
            k = 1 + int(rng[i] % np.uint64(16))
            sel = np.unique((rng[i + 1:i + 1 + k] % np.uint64(64)).astype(np.int64))
            mine.append((r % 2, sel))
        reqs.append(mine)
    counts = np.zeros(n, dtype=np.int64)
    for mine in reqs:
        for _, sel in mine:
            counts[sel] += 1
    errors = []
    with ms.Context(key1) as ctx, ms.Server(ctx, h, n, max_request_pages=16, zero_copy_max_pages=lane) as srv:
        def client(mine):
            try:
                pending = []
                for j, (op, sel) in enumerate(mine):
                    pending.append(srv.submit(op, sel))
                    if j % 7 == 6:
                        srv.wait(pending.pop(0))
                for t in pending:
                    srv.wait(t)
            except Exception as e:  # noqa: BLE001  (reported below)
                errors.append(e)
        threads = [threading.Thread(target=client, args=(m,)) for m in reqs]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        st = srv.stats()
    assert not errors, errors
    odd = np.nonzero(counts % 2)[0].astype(np.uint64)
    assert np.array_equal(h.numpy(), oracle_ws(key1, plain, odd))
    assert st["requests_done"] == n_threads * per_thread
    assert (st["staged_waves"] == st["waves"]) if lane == 0 else (st["staged_waves"] == 0)


def test_in_place_lane_with_conflicts(ms, key1):
    """Requests submitted a few at a time on overlapping pages, with the
    in-place lane on: short queues go through the lane, longer ones form
    entry-list waves (in place as well), and a request on a page still in
    flight in either kind of wave waits for it.  The final state is the
    closed form of the application counts."""
    n = 512
    h = working_set(76, n)
    plain = h.numpy().copy()
    rng = synth.splitmix64(77, 0, 20000)
    counts = np.zeros(n, dtype=np.int64)
    with ms.Context(key1) as ctx, ms.Server(ctx, h, n, zero_copy_max_pages=16) as srv:
        pending = []
        for r in range(600):
            x = int(rng[r] % np.uint64(64))
            # every fifth request is 20 pages (never in the 16-page lane), the others one page
            sel = (x + np.arange(20)) % 64 if r % 5 == 0 else np.array([x])
            counts[sel] += 1
            pending.append(srv.submit(r % 2, sel))
            if r % 3 == 2:                 # let the queue drain now and then
                srv.wait(pending.pop(0))
        for t in pending:
            srv.wait(t)
        st = srv.stats()
    odd = np.nonzero(counts % 2)[0].astype(np.uint64)
    assert np.array_equal(h.numpy(), oracle_ws(key1, plain, odd))
    assert st["inplace_waves"] > 0 and st["waves"] > st["inplace_waves"] and st["staged_waves"] == 0


def test_in_place_lane_limit(ms, key1):
    h = working_set(78, 64)
    with ms.Context(key1) as ctx:
        with pytest.raises(ms.MemShieldError) as e:
            ms.Server(ctx, h, 64, zero_copy_max_pages=513)
        assert e.value.code == ms.MS_EINVAL


def test_small_staging_budget(ms, key1):
    n, n_req = 4096, 400
    arrival, ops, offsets, pages = distinct_workload(75, n_req, n, 5e5)
    sizes = np.diff(offsets)
    keep = sizes <= 32
    # requests of at most 32 pages through a 64-page staging ring
    sel_req = np.nonzero(keep)[0]
    new_off = np.concatenate([[0], np.cumsum(sizes[sel_req])]).astype(np.uint64)
    new_pages = np.concatenate([pages[offsets[r]:offsets[r + 1]] for r in sel_req])
    plain = synth.page_bytes_fast(76, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    # four waves of up to 32 pages may be in flight, so the 64-page ring is what limits admission
    with ms.Context(key1) as ctx, ms.Server(ctx, h, n, staging_bytes=64 * PAGE, max_request_pages=32,
                                            max_wave_pages=32, waves_in_flight=4, zero_staging=True) as srv:
        lat, _ = srv.replay(arrival[sel_req], ops[sel_req], new_off, new_pages)
        st = srv.stats()
    assert np.array_equal(h.numpy(), oracle_ws(key1, plain, new_pages))
    assert st["max_wave_pages"] <= 32 and 0 < st["max_staged_pages"] <= 64


def test_limits(ms, key1):
    n = 64
    h = working_set(77, n)
    plain = h.numpy().copy()
    with ms.Context(key1) as ctx, ms.Server(ctx, h, n, max_request_pages=8) as srv:
        for bad, code in (([1] * 2, ms.MS_EINVAL), ([64], ms.MS_EINVAL), (list(range(9)), ms.MS_ERANGE)):
            with pytest.raises(ms.MemShieldError) as e:
                srv.submit(ms.MS_ENCRYPT, bad)
            assert e.value.code == code
        with pytest.raises(ms.MemShieldError):
            srv.submit(3, [1])
        assert srv.poll(10**9) == ms.MS_EINVAL
    assert np.array_equal(h.numpy(), plain)
    with ms.Context(key1) as ctx:
        with pytest.raises(ms.MemShieldError):
            ms.Server(ctx, h, n, staging_bytes=1000)      # not a multiple of 4096


def test_zero_copy_needs_pinned_memory(ms, key1):
    import numpy as np
    pageable = np.zeros(16 * PAGE, dtype=np.uint8)
    with ms.Context(key1) as ctx:
        with pytest.raises(ms.MemShieldError) as e:
            ms.Server(ctx, pageable, 16, mode=ms.MS_SERVE_ZERO_COPY)
        assert e.value.code == ms.MS_EINVAL


def test_pageable_working_set_is_staged(ms, key1):
    """Continuous mode over pageable memory: every wave is staged (no in-place waves)."""
    n = 256
    plain = synth.page_bytes(78, 0, n)
    ws = plain.copy()
    pages = synth.scattered_slots(79, n, 100)
    with ms.Context(key1) as ctx, ms.Server(ctx, ws, n) as srv:
        ts = [srv.submit(ms.MS_ENCRYPT, pages[i:i + 5]) for i in range(0, 100, 5)]
        for t in ts:
            srv.wait(t)
        st = srv.stats()
    assert np.array_equal(ws, oracle_ws(key1, plain, pages.astype(np.uint64)))
    assert st["gather_ns"] > 0 and st["staged_waves"] == st["waves"] > 0 and st["inplace_waves"] == 0


def test_in_place_lane_at_its_parameter_limit(ms, key1):
    """One request of exactly 512 pages (the lane's kernel-parameter limit)
    goes through the lane; one of 513 forms an entry-list wave, in place as
    well; both match the oracle."""
    n = 4096
    h = working_set(79, n)
    plain = h.numpy().copy()
    p512 = synth.scattered_slots(80, n, 512)
    rest = np.setdiff1d(np.arange(n), p512)
    p513 = rest[synth.scattered_slots(81, len(rest), 513)]
    with ms.Context(key1) as ctx, ms.Server(ctx, h, n) as srv:
        srv.wait(srv.submit(ms.MS_ENCRYPT, p512))
        st = srv.stats()
        assert st["inplace_waves"] == 1 and st["max_wave_pages"] == 512
        srv.wait(srv.submit(ms.MS_DECRYPT, p513))
        st = srv.stats()
        assert st["inplace_waves"] == 1 and st["waves"] == 2 and st["max_wave_pages"] == 513
        assert st["staged_waves"] == 0
    touched = np.concatenate([p512, p513]).astype(np.uint64)
    assert np.array_equal(h.numpy(), oracle_ws(key1, plain, touched))


def test_destroy_with_in_place_waves_in_flight(ms, key1):
    """Destroying a server right after queueing short requests waits (bounded)
    for the in-place waves it issued and completes every request."""
    n = 2048
    h = working_set(82, n)
    plain = h.numpy().copy()
    pages = synth.scattered_slots(83, n, 400)
    with ms.Context(key1) as ctx:
        srv = ms.Server(ctx, h, n)
        tickets = [srv.submit(ms.MS_ENCRYPT, pages[i:i + 4]) for i in range(0, 400, 4)]
        assert srv.destroy() == ms.MS_OK
    assert np.array_equal(h.numpy(), oracle_ws(key1, plain, pages.astype(np.uint64)))
    assert len(tickets) == 100
