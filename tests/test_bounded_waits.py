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
