"""Failure detection without a GPU fault: every host-side wait is bounded and a
wait that runs out returns MS_ETIMEDOUT with the context still usable; no
status report is lost across a timed-out ms_sync."""
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


def test_sync_times_out_then_completes(ms, key1):
    n = 262144
    d = torch.zeros(n * PAGE, dtype=torch.uint8, device="cuda")
    with ms.Context(key1, stream=torch.cuda.current_stream()) as ctx:
        for _ in range(20):                       # ~12 ms of queued work
            ctx.crypt_range(ms.MS_ENCRYPT, d, 0, n)
        assert ctx.sync_for(0) == ms.MS_ETIMEDOUT
        assert ctx.sync_for(60000) == ms.MS_OK
        assert int(d[:4096].sum()) == 0          # an even number of XORs


def test_status_survives_a_timed_out_sync(ms, key1):
    n_big = 262144
    big = torch.zeros(n_big * PAGE, dtype=torch.uint8, device="cuda")
    plain = synth.page_bytes(80, 0, 4)
    d = torch.from_numpy(plain).cuda()
    ids = np.arange(4, dtype=np.uint64)
    lst = ms.pages_array(d.data_ptr() + PAGE * ids, ids)
    lst["addr"][2] = 0
    dl = torch.from_numpy(lst.view(np.uint8)).cuda()
    with ms.Context(key1, stream=torch.cuda.current_stream()) as ctx:
        ctx.encrypt_pages_dev(dl, 4)              # reports a bad entry in the status word
        for _ in range(10):
            ctx.crypt_range(ms.MS_ENCRYPT, big, 0, n_big)
        assert ctx.sync_for(0) == ms.MS_ETIMEDOUT
        assert ctx.sync_for(60000) == ms.MS_EINVAL   # the report was not lost
        assert ctx.sync_for(60000) == ms.MS_OK
    good = np.array([0, 1, 3], dtype=np.uint64)
    assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, good, good))


def test_server_wait_times_out(ms, key1):
    n = 1024
    h = torch.empty(n * PAGE, dtype=torch.uint8).pin_memory()
    with ms.Context(key1) as ctx, ms.Server(ctx, h, n) as srv:
        t = srv.submit(ms.MS_ENCRYPT, np.arange(512))
        rc = ms.lib.ms_server_wait(srv.handle, t, 0)
        assert rc in (ms.MS_OK, ms.MS_ETIMEDOUT)
        srv.wait(t, 10000)
        assert srv.poll(t) == 1


def test_ticket_wait_is_not_held_up_by_a_sync(ms, key1):
    """A client waiting on its own ticket is not blocked by another thread's
    ms_sync that waits for later work (ms_poll takes no lock)."""
    import threading
    import time
    n_big = 262144
    big = torch.zeros(n_big * PAGE, dtype=torch.uint8, device="cuda")
    small = torch.zeros(4 * PAGE, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    ids = np.arange(4, dtype=np.uint64)
    with ms.Context(key1) as ctx:
        t = ctx.submit_host(ms.MS_ENCRYPT, ms.pages_array(small.data_ptr() + PAGE * ids, ids))
        for _ in range(40):                                   # ~25 ms of later work
            ctx.crypt_range(ms.MS_ENCRYPT, big, 0, n_big)
        done = {}
        def syncer():
            done["sync_rc"] = ctx.sync_for(60000)
            done["sync_t"] = time.perf_counter()
        th = threading.Thread(target=syncer)
        th.start()
        time.sleep(0.002)                                     # the sync now holds the context lock
        ctx.wait(t, 60000)
        t_ticket = time.perf_counter()
        th.join()
        assert done["sync_rc"] == ms.MS_OK
        assert t_ticket < done["sync_t"]


def test_shutdown_with_work_still_queued_times_out_and_keeps_the_context(ms, key1):
    """A shutdown whose bounded wait runs out touches nothing: the queued work
    finishes with the key intact, and a later shutdown succeeds."""
    n = 262144
    plain = synth.page_bytes_fast(84, 0, 64)
    d = torch.zeros(n * PAGE, dtype=torch.uint8, device="cuda")
    d[:64 * PAGE] = torch.from_numpy(plain).cuda()
    torch.cuda.synchronize()
    ctx = ms.Context(key1, timeout_ms=1)
    for _ in range(41):                                   # ~25 ms of queued work, odd count
        ctx.crypt_range(ms.MS_ENCRYPT, d, 0, n)
    assert ctx.shutdown() == ms.MS_ETIMEDOUT               # 1 ms is not enough
    assert ctx.handle is not None
    while ctx.sync_for(10) == ms.MS_ETIMEDOUT:             # the context still works
        pass
    assert ctx.shutdown() == ms.MS_OK
    ids = np.arange(64, dtype=np.uint64)
    assert np.array_equal(d[:64 * PAGE].cpu().numpy(), oracle_expected(key1, plain, ids, ids))
