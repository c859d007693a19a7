"""Resident workers (the paper's always-running kernel fed through queues in
mapped memory, Sec. 4.4), with bounded lifetimes: parity with the oracle for
pages in pinned host memory and in device memory, and restart after the
idle and maximum-run exits."""
import time

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


def submit_all(res, addrs, ids, doms):
    tickets = []
    for a, i, d in zip(addrs, ids, doms):
        t = res.submit(int(a), int(i), int(d))
        while t < 0:                               # ring full: wait for room
            time.sleep(0.0001)
            t = res.submit(int(a), int(i), int(d))
        tickets.append(t)
    return tickets


def expected(key, plain, slots, ids, doms):
    out = plain.copy()
    for d in np.unique(doms):
        sel = doms == d
        oracle.crypt_pages(key, out, slots[sel], ids[sel], domain=int(d))
    return out


@pytest.mark.parametrize("workers,ring", [(1, 4), (2, 64), (4, 4096)])
def test_pinned_host_pages(ms, key1, workers, ring):
    n = 512
    plain = synth.page_bytes(110, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    slots = synth.scattered_slots(111, n, 300).astype(np.uint64)
    ids = synth.splitmix64(112, 0, 300).astype(np.uint64)
    doms = (synth.splitmix64(113, 0, 300) % np.uint64(3)).astype(np.uint32)
    with ms.Context(key1) as ctx, ms.Resident(ctx, workers=workers, ring_entries=ring) as res:
        ts = submit_all(res, h.data_ptr() + PAGE * slots, ids, doms)
        for t in ts:
            res.wait(t)
        st = res.stats()
    assert np.array_equal(h.numpy(), expected(key1, plain, slots, ids, doms))
    assert st["requests"] == 300 and st["launches"] >= 1


def test_device_pages(ms, key1):
    n = 256
    plain = synth.page_bytes(114, 0, n)
    d = torch.from_numpy(plain).cuda()
    slots = np.arange(n, dtype=np.uint64)
    with ms.Context(key1, domain=0) as ctx, ms.Resident(ctx, workers=3) as res:
        ts = submit_all(res, d.data_ptr() + PAGE * slots, slots, np.zeros(n, np.uint32))
        for t in ts:
            res.wait(t)
    assert np.array_equal(d.cpu().numpy(), expected(key1, plain, slots, slots, np.zeros(n, np.uint32)))


def test_idle_exit_and_restart(ms, key1):
    n = 64
    plain = synth.page_bytes(115, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    with ms.Context(key1) as ctx, ms.Resident(ctx, workers=1, idle_exit_us=2000) as res:
        res.wait(res.submit(h.data_ptr(), 0))
        deadline = time.time() + 5
        while res.stats()["workers_running"] and time.time() < deadline:
            time.sleep(0.005)
        assert res.stats()["workers_running"] == 0          # left after 2 ms idle
        res.wait(res.submit(h.data_ptr() + PAGE, 1))        # launched again on demand
        assert res.stats()["launches"] >= 2
    want = plain.copy()
    oracle.crypt_pages(key1, want, np.array([0, 1]), np.array([0, 1]))
    assert np.array_equal(h.numpy(), want)


def test_max_run_exit_keeps_serving(ms, key1):
    """A worker leaves after max_run_ms even with requests queued; waits launch it again."""
    n = 2048
    plain = synth.page_bytes_fast(116, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    slots = np.arange(n, dtype=np.uint64)
    with ms.Context(key1) as ctx, ms.Resident(ctx, workers=2, max_run_ms=2) as res:
        ts = []
        t_end = time.time() + 0.05
        k = 0
        while time.time() < t_end and k < n:                # keep submitting past several 2 ms lifetimes
            ts += submit_all(res, [h.data_ptr() + PAGE * k], [k], [0])
            k += 1
        for t in ts:
            res.wait(t)
        st = res.stats()
    done = slots[:k]
    assert np.array_equal(h.numpy(), expected(key1, plain, done, done, np.zeros(k, np.uint32)))
    assert st["max_run_exits"] >= 1 and st["launches"] >= 2


def test_replay_matches_oracle(ms, key1):
    n, n_req = 4096, 600
    arrival, ops, offsets, pages = synth.serving_workload(117, n_req, 2e5, n)
    plain = synth.page_bytes_fast(118, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    with ms.Context(key1) as ctx, ms.Resident(ctx, workers=4) as res:
        lat, makespan = res.replay(h, n, arrival, offsets, pages)
    assert (lat >= 0).all() and makespan > 0
    counts = np.bincount(pages.astype(np.int64), minlength=n)
    odd = np.nonzero(counts % 2)[0].astype(np.uint64)
    want = plain.copy()
    oracle.crypt_pages(key1, want, odd, odd)
    assert np.array_equal(h.numpy(), want)


@pytest.mark.parametrize("workers,ring", [(16, 4), (32, 64)])
def test_replay_full_rings(ms, key1, workers, ring):
    """Every request arrives at once, so the rings fill and the replay waits
    for room on the worker whose turn it is: the pages still go round the
    workers in rotation, and the result matches the oracle."""
    n, n_req = 4096, 3000
    _, _, offsets, pages = synth.serving_workload(119, n_req, 2e5, n)
    arrival = np.zeros(n_req)
    plain = synth.page_bytes_fast(120, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    with ms.Context(key1) as ctx, ms.Resident(ctx, workers=workers, ring_entries=ring) as res:
        lat, makespan = res.replay(h, n, arrival, offsets, pages)
        st = res.stats()
    assert (lat >= 0).all() and makespan > 0 and st["requests"] == int(offsets[-1])
    counts = np.bincount(pages.astype(np.int64), minlength=n)
    odd = np.nonzero(counts % 2)[0].astype(np.uint64)
    want = plain.copy()
    oracle.crypt_pages(key1, want, odd, odd)
    assert np.array_equal(h.numpy(), want)


def test_concurrent_submitters(ms, key1):
    """Four threads submit single pages at once (disjoint pages: a page is not
    resubmitted while pending) and wait for their own tickets; every worker
    ring is shared by all four threads.  The result matches the oracle."""
    import threading
    n, per = 2048, 400
    plain = synth.page_bytes_fast(121, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    slots = synth.scattered_slots(122, n, 4 * per).astype(np.uint64)
    errors = []
    with ms.Context(key1) as ctx, ms.Resident(ctx, workers=4, ring_entries=64) as res:
        def client(mine):
            try:
                ts = submit_all(res, h.data_ptr() + PAGE * mine, mine, np.zeros(len(mine), np.uint32))
                for t in ts:
                    res.wait(t)
            except Exception as e:  # noqa: BLE001  (reported below)
                errors.append(e)
        threads = [threading.Thread(target=client, args=(slots[i * per:(i + 1) * per],)) for i in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        st = res.stats()
    assert not errors, errors
    assert st["requests"] == 4 * per
    assert np.array_equal(h.numpy(), expected(key1, plain, slots, slots, np.zeros(4 * per, np.uint32)))


def test_config_checks(ms, key1):
    with ms.Context(key1, rounds=12) as ctx:
        with pytest.raises(ms.MemShieldError):
            ms.Resident(ctx)
    with ms.Context(key1) as ctx:
        for kw in ({"ring_entries": 100}, {"workers": 65}, {"max_run_ms": 700000}):
            with pytest.raises(ms.MemShieldError):
                ms.Resident(ctx, **kw)
