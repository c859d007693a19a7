"""GPU parity of the batched form (persistent kernel K2 fed by a device work
queue, launched through CUDA graphs) and of the autotuner, against the oracle."""
import os
import tempfile

import numpy as np
import pytest

import synth
from helpers import PAGE, check_sampled_pages, check_whole_buffer, fill_device, oracle_expected, oracle_pages, sample_pages

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_09252_b300 import memshield
    return memshield


def make_ctx(ms, key, **kw):
    return ms.Context(key, stream=torch.cuda.current_stream(), **kw)


def requests(seed, n_slots, n_req, kmax):
    """Zipf(1.2) request sizes truncated to 1..kmax, pages scattered without replacement."""
    sizes = synth.zipf_sizes(seed, n_req, 1.2, kmax)
    total = int(sizes.sum())
    assert total <= n_slots
    slots = synth.scattered_slots(seed + 1, n_slots, total)
    ops = (synth.splitmix64(seed + 2, 0, n_req) >> np.uint64(63)).astype(int)
    return sizes, slots, ops


def run_batched(ms, ctx, d, sizes, slots, ops, batch_requests, **bkw):
    base = d.data_ptr()
    with ctx.batch(**bkw) as b:
        off = 0
        for r, sz in enumerate(sizes):
            sl = slots[off:off + sz].astype(np.uint64)
            rc = b.add(int(ops[r]), ms.pages_array(base + PAGE * sl, sl))
            if rc == ms.MS_EBUSY:
                b.submit()
                assert b.add(int(ops[r]), ms.pages_array(base + PAGE * sl, sl)) == ms.MS_OK
            off += sz
            if (r + 1) % batch_requests == 0:
                b.submit()
        b.submit()
        ctx.sync_checked()
        return b.stats()


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("bpt,tpc,hoist", [(1, 256, 0), (2, 128, 0), (4, 512, 0), (4, 256, 1), (2, 512, 1)])
@pytest.mark.parametrize("grab", [1, 7, 64])
def test_batched_matches_oracle(ms, key1, use_graph, bpt, tpc, hoist, grab):
    n_slots = 4096
    sizes, slots, ops = requests(40, n_slots, 120, 64)
    plain = synth.page_bytes_fast(41, 0, n_slots)
    d = torch.from_numpy(plain).cuda()
    with make_ctx(ms, key1) as ctx:
        ctx.set_shape(bpt, tpc, 10, 1, hoist)
        st = run_batched(ms, ctx, d, sizes, slots, ops, batch_requests=17, use_graph=use_graph, grab=grab)
    want = oracle_expected(key1, plain, slots, slots)
    assert np.array_equal(d.cpu().numpy(), want)
    assert st["requests"] == len(sizes) and st["pages"] == sizes.sum()
    assert st["graph_launches"] == (st["submits"] if use_graph else 0)
    assert st["submits"] == -(-len(sizes) // 17)


def test_add_requests_table(ms, key1):
    n_slots = 3000
    sizes, slots, ops = requests(50, n_slots, 90, 80)
    plain = synth.page_bytes_fast(51, 0, n_slots)
    d = torch.from_numpy(plain).cuda()
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    table = ms.pages_array(d.data_ptr() + PAGE * slots.astype(np.uint64), slots)
    with make_ctx(ms, key1) as ctx, ctx.batch(capacity=500) as b:
        first = 0
        while first < len(sizes):
            rc, added = b.add_requests(ops, offsets, table, first)
            first += added
            if rc == ms.MS_EBUSY:
                assert added < len(sizes)
            b.submit()
        ctx.sync_checked()
        assert b.stats()["requests"] == len(sizes)
    assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, slots, slots))


def test_batch_full_returns_busy_and_recovers(ms, key1):
    n_slots = 600
    sizes, slots, ops = requests(42, n_slots, 40, 30)
    plain = synth.page_bytes(43, 0, n_slots)
    d = torch.from_numpy(plain).cuda()
    with make_ctx(ms, key1) as ctx:
        st = run_batched(ms, ctx, d, sizes, slots, ops, batch_requests=10**9, capacity=64)
    assert st["submits"] > 2                   # several forced submits, buffers alternated
    assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, slots, slots))


def test_batch_rejects_bad_entries_and_empty_submit(ms, key1):
    plain = synth.page_bytes(44, 0, 4)
    d = torch.from_numpy(plain).cuda()
    ids = np.arange(4, dtype=np.uint64)
    with make_ctx(ms, key1) as ctx, ctx.batch(capacity=16) as b:
        b.submit()                             # empty: no-op
        bad = ms.pages_array(d.data_ptr() + PAGE * ids, ids)
        bad["addr"][1] = 0
        with pytest.raises(ms.MemShieldError) as e:
            b.add(ms.MS_ENCRYPT, bad)
        assert e.value.code == ms.MS_EINVAL
        with pytest.raises(ms.MemShieldError):
            b.add(5, ms.pages_array(d.data_ptr() + PAGE * ids, ids))
        big = ms.pages_array(np.full(17, d.data_ptr(), np.uint64), np.arange(17))
        with pytest.raises(ms.MemShieldError) as e:
            b.add(ms.MS_ENCRYPT, big)                  # larger than the whole batch
        assert e.value.code == ms.MS_ERANGE
        assert b.add(ms.MS_ENCRYPT, ms.pages_array(d.data_ptr() + PAGE * ids, ids)) == ms.MS_OK
        b.submit()
        ctx.sync_checked()
        assert b.stats()["submits"] == 1
    assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, ids, ids))


def test_batch_reduced_rounds(ms, key1):
    n_slots = 300
    sizes, slots, ops = requests(45, n_slots, 20, 12)
    plain = synth.page_bytes(46, 0, n_slots)
    for rounds in (8, 12):
        d = torch.from_numpy(plain).cuda()
        with make_ctx(ms, key1, rounds=rounds) as ctx:
            run_batched(ms, ctx, d, sizes, slots, ops, batch_requests=7)
        assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, slots, slots, rounds=rounds))


def test_autotune_then_parity_and_table(ms, key1):
    with make_ctx(ms, key1) as ctx:
        r = ctx.autotune(8192)
        assert r["tried"] > 50 and r["k1_gbs"] > 0 and r["queue_gbs"] > 0
        assert r["grab"] in (1, 2, 4, 8, 16, 32, 64)
        assert ctx.get_shape() == r["shape"]
        # the tuned shapes still give the oracle's bytes, one launch and batched
        n_slots = 2000
        sizes, slots, ops = requests(47, n_slots, 60, 40)
        plain = synth.page_bytes_fast(48, 0, n_slots)
        d = torch.from_numpy(plain).cuda()
        run_batched(ms, ctx, d, sizes, slots, ops, batch_requests=25)
        want = oracle_expected(key1, plain, slots, slots)
        assert np.array_equal(d.cpu().numpy(), want)
        d2 = torch.from_numpy(plain).cuda()
        ids = np.arange(n_slots, dtype=np.uint64)
        ctx.encrypt_pages(ms.pages_array(d2.data_ptr() + PAGE * ids, ids))
        ctx.sync_checked()
        assert np.array_equal(d2.cpu().numpy(), oracle_expected(key1, plain, ids, ids))
        with tempfile.TemporaryDirectory() as tmp:
            path = os.path.join(tmp, "tune.txt")
            ctx.tune_save(path)
            ctx.set_shape(1, 128, 2, 0)
            assert ctx.tune_load(path) == ms.MS_OK
            assert ctx.get_shape() == r["shape"]
            line = open(path).read().split()
            line[1] = "Some_Other_GPU"
            open(path, "w").write(" ".join(line) + "\n")
            assert ctx.tune_load(path) == ms.MS_EINVAL
            assert ctx.tune_load(os.path.join(tmp, "missing.txt")) == ms.MS_EINVAL


@pytest.mark.slow
@pytest.mark.parametrize("form", ["batch", "feed"])
def test_batching_config_full_size(ms, key1, form):
    """The batching configuration at full size: 20,000 Zipf(1.2) requests (1..512
    pages) scattered without replacement over an 8 GiB buffer of SplitMix64
    seed-3 bytes.  The persistent batched path (graph-launched submits, or one
    fed launch) and one launch per request give identical 8 GiB buffers; the
    whole result equals the oracle's (every touched page XORed once, the rest
    unchanged), byte for byte and by SHA-256; and a seeded 1/16 of the touched
    pages, recomputed one by one, matches."""
    n_slots = 2097152
    sizes, slots, ops = synth.batching_workload(3)
    a = torch.empty(n_slots * PAGE, dtype=torch.uint8, device="cuda")
    fill_device(a, 3, n_slots)
    b = a.clone()
    with make_ctx(ms, key1) as ctx:
        if form == "batch":
            run_batched(ms, ctx, a, sizes, slots, ops, batch_requests=500)
        else:
            offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
            sl = slots.astype(np.uint64)
            table = ms.pages_array(a.data_ptr() + PAGE * sl, sl)
            with ctx.feed(capacity=len(slots)) as f:
                f.open()
                first = 0
                while first < len(sizes):
                    first += f.add_requests(ops.astype(np.int32), offsets, table, first, min(700, len(sizes) - first))
                f.close()
                ctx.sync_checked()
        off = 0
        base = b.data_ptr()
        for sz in sizes:
            sl = slots[off:off + sz].astype(np.uint64)
            ctx.encrypt_pages(ms.pages_array(base + PAGE * sl, sl))
            off += sz
        ctx.sync_checked()
    assert torch.equal(a, b)
    del b
    odd = np.bincount(slots.astype(np.int64), minlength=n_slots) % 2 == 1
    assert odd.sum() == len(slots)                      # without replacement: each touched page once
    h = torch.empty(262144 * PAGE, dtype=torch.uint8).pin_memory()

    def chunk(p0, m):
        h[:m * PAGE].copy_(a[p0 * PAGE:(p0 + m) * PAGE])
        return h[:m * PAGE].numpy()
    got_sha, want_sha = check_whole_buffer(key1, 3, n_slots, odd, chunk)
    assert got_sha == want_sha
    av = a.view(n_slots, PAGE)
    n = check_sampled_pages(key1, 3, np.unique(slots.astype(np.int64)), odd,
                            lambda pick: av[torch.from_numpy(pick).cuda()].cpu().numpy(), 49)
    assert n > len(slots) // 20


def test_shutdown_refused_while_children_live(ms, key1):
    ctx = ms.Context(key1)
    b = ctx.batch(capacity=16)
    h = torch.zeros(16 * PAGE, dtype=torch.uint8).pin_memory()
    srv = ms.Server(ctx, h, 16)
    assert ms.lib.ms_shutdown(ctx.handle) == ms.MS_EBUSY      # the context stays usable
    b.destroy()
    assert ms.lib.ms_shutdown(ctx.handle) == ms.MS_EBUSY
    srv.wait(srv.submit(ms.MS_ENCRYPT, [1]))
    srv.destroy()
    assert ctx.shutdown() == ms.MS_OK
