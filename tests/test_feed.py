"""The fed form (ms_feed): one persistent kernel drains a queue the host is
still filling.  Bit-exact against the oracle; a feed that is not fed runs
out its bounded wait and reports MS_ESTARVED without faulting anything."""
import numpy as np
import pytest

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


def request_table(seed, n_slots, n_req, max_pages):
    sizes = (synth.splitmix64(seed, 0, n_req) % np.uint64(max_pages) + np.uint64(1)).astype(np.int64)
    total = int(sizes.sum())
    slots = synth.scattered_slots(seed + 1, n_slots, total).astype(np.uint64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    ops = (synth.splitmix64(seed + 2, 0, n_req) % np.uint64(2)).astype(np.int32)
    return slots, offsets, ops


@pytest.mark.parametrize("chunk,per_call", [(1024, 7), (4096, 300), (65536, 50)])
def test_fed_queue_matches_oracle(ms, key1, chunk, per_call):
    """Ragged requests over scattered slots, appended a few at a time while the
    kernel runs; many publications (chunk 1024) or one at the close."""
    n_slots = 12000
    slots, offsets, ops = request_table(180, n_slots, 400, 40)
    plain = synth.page_bytes_fast(181, 0, n_slots)
    d = torch.from_numpy(plain).cuda()
    torch.cuda.synchronize()
    table = ms.pages_array(d.data_ptr() + PAGE * slots, slots)
    with ms.Context(key1) as ctx:
        with ctx.feed(capacity=len(slots), chunk=chunk) as f:
            f.open()
            first = 0
            while first < len(ops):
                first += f.add_requests(ops, offsets, table, first, min(per_call, len(ops) - first))
            f.close()
            st = f.stats()
            ctx.sync_checked()
        assert st["pages"] == len(slots) and st["requests"] == 400
        assert st["publications"] >= (len(slots) // chunk)
    assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, slots, slots))


def test_feeds_one_after_another_and_empty(ms, key1):
    n_slots = 3000
    plain = synth.page_bytes_fast(182, 0, n_slots)
    d = torch.from_numpy(plain).cuda()
    torch.cuda.synchronize()
    ids = np.arange(n_slots, dtype=np.uint64)
    table = ms.pages_array(d.data_ptr() + PAGE * ids, ids)
    offsets = np.array([0, 1000, 2999, 3000], dtype=np.uint64)
    ops = np.zeros(3, dtype=np.int32)
    with ms.Context(key1) as ctx:
        for _ in range(3):                                    # odd: encrypted once net
            with ctx.feed(capacity=n_slots, chunk=1024) as f:
                assert f.open().add_requests(ops, offsets, table) == 3
        with ctx.feed(capacity=n_slots, chunk=1024) as f:     # one feed, two runs: even, no net change
            for _ in range(2):
                f.open()
                assert f.add_requests(ops, offsets, table) == 3
                f.close()
            assert f.stats()["runs"] == 2
        with ctx.feed() as f:                                 # opened and closed with nothing in it
            f.open().close()
        ctx.sync_checked()
    assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, ids, ids))


def test_feed_checks_on_the_host(ms, key1):
    d = torch.zeros(8 * PAGE, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    ids = np.arange(8, dtype=np.uint64)
    good = ms.pages_array(d.data_ptr() + PAGE * ids, ids)
    bad = good.copy()
    bad["addr"][3] += 8
    offsets = np.array([0, 8], dtype=np.uint64)
    ops = np.zeros(1, dtype=np.int32)
    with ms.Context(key1) as ctx:
        with ctx.feed(capacity=8, chunk=1024) as f:
            with pytest.raises(ms.MemShieldError):
                f.add_requests(ops, offsets, good)              # not open yet
            f.open()
            with pytest.raises(ms.MemShieldError) as e:
                f.open()                                        # already open
            assert e.value.code == ms.MS_EBUSY
            with pytest.raises(ms.MemShieldError) as e:
                f.add_requests(ops, offsets, bad)
            assert e.value.code == ms.MS_EINVAL
            with pytest.raises(ms.MemShieldError) as e:
                f.add_requests(np.zeros(2, dtype=np.int32), np.array([0, 8, 16], dtype=np.uint64),
                               np.concatenate([good, good]))   # 16 entries in a feed of 8
            assert e.value.code == ms.MS_ERANGE
            f.close()
            with pytest.raises(ms.MemShieldError):
                f.add_requests(ops, offsets, good)              # closed
        ctx.sync_checked()
        with pytest.raises(ms.MemShieldError):
            ctx.feed(chunk=100)                                 # chunk below 1024


def test_a_starved_feed_reports_and_the_context_recovers(ms, key1):
    """Entries are published but the feed is never closed: CTAs whose claims lie
    beyond them wait wait_ms (50 ms), set the starved bit and leave.  The next
    ms_sync returns MS_ESTARVED; the context then works as before."""
    n = 2048
    plain = synth.page_bytes_fast(183, 0, n)
    d = torch.from_numpy(plain).cuda()
    torch.cuda.synchronize()
    ids = np.arange(n, dtype=np.uint64)
    table = ms.pages_array(d.data_ptr() + PAGE * ids, ids)
    with ms.Context(key1) as ctx:
        f = ctx.feed(capacity=n, chunk=1024, wait_ms=50).open()
        assert f.add_requests(np.zeros(1, dtype=np.int32), np.array([0, 1024], dtype=np.uint64), table) == 1
        assert ctx.sync_for(60000) == ms.MS_ESTARVED     # the kernel left by its bounded wait
        assert f.destroy() == ms.MS_OK                   # closing a feed whose kernel left is fine
        assert ctx.sync() == 0
        d2 = torch.from_numpy(plain).cuda()
        torch.cuda.synchronize()
        ctx.encrypt_pages(ms.pages_array(d2.data_ptr() + PAGE * ids, ids))
        ctx.sync_checked()
        assert np.array_equal(d2.cpu().numpy(), oracle_expected(key1, plain, ids, ids))


@pytest.mark.parametrize("rounds,bpt", [(12, 4), (8, 2), (20, 1), (20, 2)])
def test_fed_queue_reduced_rounds_and_shapes(ms, key1, rounds, bpt):
    """The fed kernel's other instances: ChaCha12 / ChaCha8 and 1 or 2 blocks
    per thread (taken from the context's shape)."""
    n_slots = 5000
    slots, offsets, ops = request_table(185, n_slots, 150, 30)
    plain = synth.page_bytes_fast(186, 0, n_slots)
    d = torch.from_numpy(plain).cuda()
    torch.cuda.synchronize()
    table = ms.pages_array(d.data_ptr() + PAGE * slots, slots)
    with ms.Context(key1, rounds=rounds) as ctx:
        if bpt != 4:
            ctx.set_shape(bpt, 128, rounds // 2, 1, 1 if bpt >= 2 else 0)
        with ctx.feed(capacity=len(slots), chunk=1024) as f:
            f.open()
            assert f.add_requests(ops, offsets, table) == len(ops)
            f.close()
            ctx.sync_checked()
    assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, slots, slots, rounds=rounds))
