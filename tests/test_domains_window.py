"""Per-page domains (the paper's client PID in the nonce) and the
sliding-window client driver (the fault / eviction stream of Sec. 4.3),
checked against the oracle on the GPU."""
import numpy as np
import pytest

import oracle
import synth
from helpers import PAGE, oracle_expected

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_09252_b300 import memshield
    return memshield


def oracle_by_domain(key, plain, slots, ids, domains):
    out = plain.copy()
    for dom in np.unique(domains):
        sel = domains == dom
        oracle.crypt_pages(key, out, slots[sel], ids[sel], domain=int(dom))
    return out


@pytest.mark.parametrize("n", [1, 16, 129, 512, 513])
def test_per_page_domains_short_host_lists(ms, key1, n):
    """Host lists with a domain per entry: up to 512 travel in the kernel's
    parameters, 513 takes the staged path."""
    n_slots = n + 11
    plain = synth.page_bytes(95, 0, n_slots)
    slots = synth.scattered_slots(96, n_slots, n).astype(np.uint64)
    ids = synth.splitmix64(97, 0, n).astype(np.uint64)
    doms = (synth.splitmix64(98, 0, n) % np.uint64(7)).astype(np.uint32) * np.uint32(0x10001)
    want = oracle_by_domain(key1, plain, slots, ids, doms)
    with ms.Context(key1, stream=torch.cuda.current_stream(), domain=999) as ctx:
        d = torch.from_numpy(plain).cuda()
        ctx.crypt_pages_dom(ms.pages_dom_array(d.data_ptr() + PAGE * slots, ids, doms))
        ctx.sync_checked()
        assert np.array_equal(d.cpu().numpy(), want)


@pytest.mark.parametrize("shape", [None, (1, 256, 10, 1, 0), (4, 128, 10, 1, 0), (2, 512, 10, 0, 1)])
def test_per_page_domains_host_and_device_lists(ms, key1, shape):
    n_slots, n = 300, 257
    plain = synth.page_bytes(90, 0, n_slots)
    slots = synth.scattered_slots(91, n_slots, n).astype(np.uint64)
    ids = synth.splitmix64(92, 0, n).astype(np.uint64)
    doms = (synth.splitmix64(93, 0, n) % np.uint64(5)).astype(np.uint32) * np.uint32(0x1234567)
    want = oracle_by_domain(key1, plain, slots, ids, doms)
    with ms.Context(key1, stream=torch.cuda.current_stream(), domain=999) as ctx:
        if shape:
            ctx.set_shape(*shape)
        d = torch.from_numpy(plain).cuda()
        ctx.crypt_pages_dom(ms.pages_dom_array(d.data_ptr() + PAGE * slots, ids, doms))
        ctx.sync_checked()
        assert np.array_equal(d.cpu().numpy(), want)
        d2 = torch.from_numpy(plain).cuda()
        lst = torch.from_numpy(ms.pages_dom_array(d2.data_ptr() + PAGE * slots, ids, doms).view(np.uint8)).cuda()
        ctx.crypt_pages_dom_dev(lst, n)
        ctx.sync_checked()
        assert np.array_equal(d2.cpu().numpy(), want)


@pytest.mark.parametrize("n,lane,zc", [(512, None, False), (4096, None, False), (4096, 0, False),
                                       (4096, None, True)])
def test_server_requests_with_domains(ms, key1, n, lane, zc):
    """Requests with their own domain words through the in-place lane (short
    queue), through long in-place waves (thousands of pages queued at once),
    staged (lane off) and in zero-copy mode."""
    plain = synth.page_bytes(94, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    m = 400 if n == 512 else 4000
    pages = synth.scattered_slots(95, n, m)
    doms = np.repeat(np.array([7, 11, 13, 7], dtype=np.uint32), m // 4)
    mode = ms.MS_SERVE_ZERO_COPY if zc else ms.MS_SERVE_CONTINUOUS
    n_req = m // 4
    offsets = (np.arange(n_req + 1) * 4).astype(np.uint64)
    ops = np.full(n_req, ms.MS_ENCRYPT, dtype=np.int32)
    with ms.Context(key1, domain=5) as ctx, ms.Server(ctx, h, n, mode=mode, zero_copy_max_pages=lane) as srv:
        if n == 512:   # one at a time from Python: short queues, the lane
            ts = [srv.submit(ms.MS_ENCRYPT, pages[i:i + 4], domain=int(doms[i])) for i in range(0, m, 4)]
            for t in ts:
                srv.wait(t)
        else:          # all at once from the replay: the queue outgrows the lane
            srv.replay(np.zeros(n_req), ops, offsets, pages, domains=doms[::4].copy())
        st = srv.stats()
    want = oracle_by_domain(key1, plain, pages.astype(np.uint64), pages.astype(np.uint64), doms)
    assert np.array_equal(h.numpy(), want)
    assert (st["staged_waves"] == st["waves"]) if lane == 0 else (st["staged_waves"] == 0)
    if n > 512 and lane is None and not zc:
        assert st["waves"] > st["inplace_waves"]       # long in-place waves formed


@pytest.mark.parametrize("window,batch", [(4, 1), (8, 1), (8, 4), (16, 9)])
def test_sliding_window_clients(ms, key1, window, batch):
    """Three clients with their own PIDs fault through FIFO windows; afterwards
    exactly their final-window pages are in clear, the rest encrypted."""
    per, n_clients = 128, 3
    n = per * n_clients
    plain = synth.page_bytes_fast(96, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    doms = [1001, 2002, 3003]
    clients = [(doms[c], c * per, per, synth.window_trace(97 + c, per, 1500)) for c in range(n_clients)]
    with ms.Context(key1) as ctx, ms.Server(ctx, h, n) as srv:
        for c in range(n_clients):             # every client page starts encrypted
            srv.wait(srv.submit(ms.MS_ENCRYPT, np.arange(c * per, (c + 1) * per), domain=doms[c]))
        stats, wins = srv.run_window_clients(window, batch, clients)
    ws = h.numpy()
    for c in range(n_clients):
        st, win = stats[c], wins[c]
        assert st["accesses"] == 1500 and st["hits"] + st["faults"] == 1500
        assert st["faults"] - st["evictions"] == len(win) == st["final_window_pages"] <= window
        assert len(set(win)) == len(win) and all(c * per <= p < (c + 1) * per for p in win)
        enc = np.array(sorted(set(range(c * per, (c + 1) * per)) - set(win)), dtype=np.uint64)
        want = plain[c * per * PAGE:(c + 1) * per * PAGE].copy()
        rel = enc - np.uint64(c * per)
        oracle.crypt_pages(key1, want, rel, enc, domain=doms[c])
        assert np.array_equal(ws[c * per * PAGE:(c + 1) * per * PAGE], want), f"client {c}"
        assert st["fault_p50_us"] > 0 and st["fault_p99_us"] >= st["fault_p50_us"]


@pytest.mark.parametrize("window,batch", [(4, 1), (8, 4), (16, 9)])
def test_sliding_window_clients_on_resident_workers(ms, key1, window, batch):
    """The same clients served by resident workers in place on the pinned working
    set: the same final state (final-window pages in clear, the rest encrypted
    under each client's PID)."""
    per, n_clients = 128, 3
    n = per * n_clients + 5                     # pages past the clients stay untouched
    plain = synth.page_bytes_fast(196, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    doms = [11, 22, 33]
    clients = [(doms[c], c * per, per, synth.window_trace(197 + c, per, 1500)) for c in range(n_clients)]
    with ms.Context(key1) as ctx:
        with ms.Server(ctx, h, n) as srv:
            for c in range(n_clients):
                srv.wait(srv.submit(ms.MS_ENCRYPT, np.arange(c * per, (c + 1) * per), domain=doms[c]))
        with ms.Resident(ctx, workers=4) as res:
            stats, wins = res.run_window_clients(h, n, window, batch, clients)
    ws = h.numpy()
    for c in range(n_clients):
        st, win = stats[c], wins[c]
        assert st["accesses"] == 1500 and st["hits"] + st["faults"] == 1500
        assert st["faults"] - st["evictions"] == len(win) <= window
        enc = np.array(sorted(set(range(c * per, (c + 1) * per)) - set(win)), dtype=np.uint64)
        want = plain[c * per * PAGE:(c + 1) * per * PAGE].copy()
        oracle.crypt_pages(key1, want, enc - np.uint64(c * per), enc, domain=doms[c])
        assert np.array_equal(ws[c * per * PAGE:(c + 1) * per * PAGE], want), f"client {c}"
    assert np.array_equal(ws[n_clients * per * PAGE:], plain[n_clients * per * PAGE:])
    with ms.Context(key1) as ctx, ms.Resident(ctx) as res:
        with pytest.raises(ms.MemShieldError):                 # a client range past the working set
            res.run_window_clients(h, n, 4, 1, [(1, n - 4, 8, np.zeros(2, dtype=np.uint64))])


@pytest.mark.parametrize("window,batch", [(4, 1), (16, 9)])
def test_sliding_window_clients_on_ticketed_launches(ms, key1, window, batch):
    """The same clients served by one ticketed launch per fault and per eviction,
    each client on its own clone of the context (its PID, its stream): the same
    final state."""
    per, n_clients = 128, 3
    n = per * n_clients
    plain = synth.page_bytes_fast(296, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    doms = [501, 502, 503]
    clients = [(doms[c], c * per, per, synth.window_trace(297 + c, per, 1500)) for c in range(n_clients)]
    with ms.Context(key1) as ctx:
        base = ms.host_device_address(h)
        for c in range(n_clients):                             # all start encrypted under their PID
            ids = np.arange(c * per, (c + 1) * per, dtype=np.uint64)
            k = ctx.clone(doms[c])
            k.wait(k.submit_host(ms.MS_ENCRYPT, ms.pages_array(base + PAGE * ids, ids)))
            k.shutdown()
        stats, wins = ctx.run_window_clients(h, n, window, batch, clients)
    ws = h.numpy()
    for c in range(n_clients):
        st, win = stats[c], wins[c]
        assert st["accesses"] == 1500 and st["faults"] - st["evictions"] == len(win) <= window
        enc = np.array(sorted(set(range(c * per, (c + 1) * per)) - set(win)), dtype=np.uint64)
        want = plain[c * per * PAGE:(c + 1) * per * PAGE].copy()
        oracle.crypt_pages(key1, want, enc - np.uint64(c * per), enc, domain=doms[c])
        assert np.array_equal(ws[c * per * PAGE:(c + 1) * per * PAGE], want), f"client {c}"


def test_clone_keeps_the_key_and_takes_its_domain(ms, key1):
    """A clone encrypts with the parent's key under its own domain, on its own
    stream; the parent is unchanged; a clone of a clone works too."""
    n = 40
    plain = synth.page_bytes(298, 0, n)
    ids = np.arange(n, dtype=np.uint64)
    with ms.Context(key1, domain=7) as ctx:
        ctx.set_shape(2, 256, 10, 1)
        k = ctx.clone(9)
        k2 = k.clone(11)
        assert k.get_shape() == ctx.get_shape()
        for c, dom in ((ctx, 7), (k, 9), (k2, 11)):
            d = torch.from_numpy(plain).cuda()
            torch.cuda.synchronize()
            c.encrypt_pages(ms.pages_array(d.data_ptr() + PAGE * ids, ids))
            c.sync_checked()
            assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, ids, ids, domain=dom))
        k2.shutdown()
        k.shutdown()
    with ms.Context(None) as rnd:                              # a random key: the clone matches it
        k = rnd.clone(0)
        a, b = torch.from_numpy(plain).cuda(), torch.from_numpy(plain).cuda()
        torch.cuda.synchronize()
        rnd.encrypt_pages(ms.pages_array(a.data_ptr() + PAGE * ids, ids))
        k.encrypt_pages(ms.pages_array(b.data_ptr() + PAGE * ids, ids))
        rnd.sync_checked()
        k.sync_checked()
        assert torch.equal(a, b) and not np.array_equal(a.cpu().numpy(), plain)
        k.shutdown()


def test_window_rejects_bad_configs(ms, key1):
    n = 64
    h = torch.zeros(n * PAGE, dtype=torch.uint8).pin_memory()
    with ms.Context(key1) as ctx, ms.Server(ctx, h, n) as srv:
        tr = np.zeros(4, dtype=np.uint64)
        with pytest.raises(ms.MemShieldError):
            srv.run_window_clients(0, 1, [(1, 0, 32, tr)])          # empty window
        with pytest.raises(ms.MemShieldError):
            srv.run_window_clients(4, 1, [(1, 0, 32, tr), (2, 16, 32, tr)])   # overlapping clients
        with pytest.raises(ms.MemShieldError):
            srv.run_window_clients(4, 1, [(1, 0, 32, np.array([40], dtype=np.uint64))])  # outside the client


@pytest.mark.parametrize("use_graph", [True, False])
def test_batched_form_with_per_page_domains(ms, key1, use_graph):
    n_slots, n = 1024, 700
    plain = synth.page_bytes_fast(98, 0, n_slots)
    d = torch.from_numpy(plain).cuda()
    slots = synth.scattered_slots(99, n_slots, n).astype(np.uint64)
    doms = (synth.splitmix64(100, 0, n) % np.uint64(4) + np.uint64(40)).astype(np.uint32)
    doms[600:] = 5                                         # these go through ms_batch_add: context domain
    with ms.Context(key1, stream=torch.cuda.current_stream(), domain=5) as ctx:
        with ctx.batch(capacity=300, use_graph=use_graph, per_page_domain=True) as b:
            for lo in range(0, 600, 50):
                sel = slice(lo, lo + 50)
                e = ms.pages_dom_array(d.data_ptr() + PAGE * slots[sel], slots[sel], doms[sel])
                if b.add_dom(ms.MS_ENCRYPT, e) == ms.MS_EBUSY:
                    b.submit()
                    assert b.add_dom(ms.MS_ENCRYPT, e) == ms.MS_OK
            b.submit()
            assert b.add(ms.MS_ENCRYPT, ms.pages_array(d.data_ptr() + PAGE * slots[600:], slots[600:])) == ms.MS_OK
            b.submit()
            ctx.sync_checked()
        with ctx.batch(capacity=16) as plain_batch:
            with pytest.raises(ms.MemShieldError):
                plain_batch.add_dom(ms.MS_ENCRYPT, ms.pages_dom_array([d.data_ptr()], [0], [1]))
    assert np.array_equal(d.cpu().numpy(), oracle_by_domain(key1, plain, slots, slots, doms))


@pytest.mark.parametrize("backend", ["server", "resident", "ticketed"])
@pytest.mark.parametrize("window,batch,free", [(4, 1, 1), (8, 1, 3), (16, 4, 6), (32, 8, 31)])
def test_background_eviction_final_state(ms, key1, backend, window, batch, free):
    """Background eviction (the paper's conclusions: encrypt window pages ahead
    of need once the free slots fall below a threshold): every client's
    evictor keeps `free` window slots free off the fault path.  Afterwards the
    final-window pages are in clear and every other page of the client is
    encrypted under its PID (the oracle); the final window holds at most
    window - free pages and the evictor did run."""
    per, n_clients = 128, 3
    n = per * n_clients
    plain = synth.page_bytes_fast(396, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    doms = [701, 702, 703]
    clients = [(doms[c], c * per, per, synth.window_trace(397 + c, per, 1500)) for c in range(n_clients)]
    with ms.Context(key1) as ctx:
        with ms.Server(ctx, h, n) as srv:
            for c in range(n_clients):             # every client page starts encrypted
                srv.wait(srv.submit(ms.MS_ENCRYPT, np.arange(c * per, (c + 1) * per), domain=doms[c]))
            if backend == "server":
                stats, wins = srv.run_window_clients(window, batch, clients, background_free=free)
        if backend == "resident":
            with ms.Resident(ctx, workers=4) as res:
                stats, wins = res.run_window_clients(h, n, window, batch, clients, background_free=free)
        elif backend == "ticketed":
            stats, wins = ctx.run_window_clients(h, n, window, batch, clients, background_free=free)
    ws = h.numpy()
    for c in range(n_clients):
        st, win = stats[c], wins[c]
        assert st["accesses"] == 1500 and st["hits"] + st["faults"] == 1500
        assert st["faults"] - st["evictions"] == len(win) == st["final_window_pages"] <= window - free
        assert 0 < st["background_evictions"] <= st["evictions"]
        assert 0 < st["background_requests"] <= st["evict_requests"]
        assert len(set(win)) == len(win) and all(c * per <= p < (c + 1) * per for p in win)
        enc = np.array(sorted(set(range(c * per, (c + 1) * per)) - set(win)), dtype=np.uint64)
        want = plain[c * per * PAGE:(c + 1) * per * PAGE].copy()
        oracle.crypt_pages(key1, want, enc - np.uint64(c * per), enc, domain=doms[c])
        assert np.array_equal(ws[c * per * PAGE:(c + 1) * per * PAGE], want), f"client {c}"


def test_background_eviction_rejects_bad_thresholds(ms, key1):
    n = 64
    h = torch.from_numpy(synth.page_bytes(399, 0, n)).pin_memory()
    tr = np.zeros(4, dtype=np.uint64)
    with ms.Context(key1) as ctx, ms.Server(ctx, h, n) as srv:
        for free in (4, 9):                         # the threshold must leave room for a page
            with pytest.raises(ms.MemShieldError) as e:
                srv.run_window_clients(4, 1, [(1, 0, 32, tr)], background_free=free)
            assert e.value.code == ms.MS_EINVAL


@pytest.mark.parametrize("backend", ["server", "resident", "ticketed"])
@pytest.mark.parametrize("window,batch,free", [(8, 1, 0), (16, 4, 0), (8, 1, 3)])
def test_synchronous_eviction_final_state(ms, key1, backend, window, batch, free):
    """Each client waits for its own overflow evictions (the paper's per-client
    server finishes an eviction before the next fault), alone and beside a
    background evictor: the same final state as the asynchronous policies."""
    per, n_clients = 128, 2
    n = per * n_clients
    plain = synth.page_bytes_fast(496, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    doms = [801, 802]
    clients = [(doms[c], c * per, per, synth.window_trace(497 + c, per, 1500)) for c in range(n_clients)]
    kw = dict(background_free=free, sync_evict=True)
    with ms.Context(key1) as ctx:
        with ms.Server(ctx, h, n) as srv:
            for c in range(n_clients):
                srv.wait(srv.submit(ms.MS_ENCRYPT, np.arange(c * per, (c + 1) * per), domain=doms[c]))
            if backend == "server":
                stats, wins = srv.run_window_clients(window, batch, clients, **kw)
        if backend == "resident":
            with ms.Resident(ctx, workers=4) as res:
                stats, wins = res.run_window_clients(h, n, window, batch, clients, **kw)
        elif backend == "ticketed":
            stats, wins = ctx.run_window_clients(h, n, window, batch, clients, **kw)
    ws = h.numpy()
    for c in range(n_clients):
        st, win = stats[c], wins[c]
        assert st["accesses"] == 1500 and st["faults"] - st["evictions"] == len(win) <= window - free
        enc = np.array(sorted(set(range(c * per, (c + 1) * per)) - set(win)), dtype=np.uint64)
        want = plain[c * per * PAGE:(c + 1) * per * PAGE].copy()
        oracle.crypt_pages(key1, want, enc - np.uint64(c * per), enc, domain=doms[c])
        assert np.array_equal(ws[c * per * PAGE:(c + 1) * per * PAGE], want), f"client {c}"
