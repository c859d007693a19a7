"""Error handling under host-side fault injection: a CUDA call that fails
(simulated on the host, the real call skipped; no GPU fault) gives MS_ECUDA
and the error code, and the context keeps working afterwards."""
import numpy as np
import pytest

import oracle
import synth
from helpers import PAGE, oracle_expected

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ERR = 719  # cudaErrorLaunchFailure, as reported by the injected failure


@pytest.fixture(scope="module")
def ms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_09252_b300 import memshield
    yield memshield
    memshield.inject_fault(0)


def test_inject_rejects_bad_arguments(ms):
    with pytest.raises(ms.MemShieldError):
        ms.inject_fault(64)
    with pytest.raises(ms.MemShieldError):
        ms.inject_fault(ms.MS_FAULT_LAUNCH, -1)
    ms.inject_fault(0)


@pytest.mark.parametrize("site", ["launch", "copy"])
def test_one_launch_form_recovers(ms, key1, site):
    n = 32
    plain = synth.page_bytes(120, 0, n)
    d = torch.from_numpy(plain).cuda()
    ids = np.arange(n, dtype=np.uint64)
    pages = ms.pages_array(d.data_ptr() + PAGE * ids, ids)
    with ms.Context(key1, stream=torch.cuda.current_stream()) as ctx:
        ms.inject_fault(ms.MS_FAULT_LAUNCH if site == "launch" else ms.MS_FAULT_COPY, 0, ERR)
        with pytest.raises(ms.MemShieldError) as e:
            ctx.encrypt_pages(pages)
        assert e.value.code == ms.MS_ECUDA and ctx.last_cuda_error() == ERR
        ctx.sync_checked()
        assert np.array_equal(d.cpu().numpy(), plain)       # nothing was applied
        ctx.encrypt_pages(pages)                            # the context still works
        ctx.sync_checked()
    assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, ids, ids))


def test_countdown_skips_earlier_calls(ms, key1):
    n = 8
    plain = synth.page_bytes(121, 0, n)
    d = torch.from_numpy(plain).cuda()
    with ms.Context(key1, stream=torch.cuda.current_stream()) as ctx:
        ms.inject_fault(ms.MS_FAULT_LAUNCH, 2, ERR)          # the third launch fails
        ctx.crypt_range(ms.MS_ENCRYPT, d, 0, n)
        ctx.crypt_range(ms.MS_ENCRYPT, d, 0, n)
        with pytest.raises(ms.MemShieldError):
            ctx.crypt_range(ms.MS_ENCRYPT, d, 0, n)
        ctx.crypt_range(ms.MS_ENCRYPT, d, 0, n)
        ctx.sync_checked()
    # three applications went through: odd, so the pages are encrypted once
    ids = np.arange(n, dtype=np.uint64)
    assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, ids, ids))


def test_host_stream_copy_failure(ms, key1):
    n = 600
    plain = synth.page_bytes(122, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    with ms.Context(key1) as ctx:
        ms.inject_fault(ms.MS_FAULT_COPY, 1, ERR)           # the second chunk's copy fails
        with pytest.raises(ms.MemShieldError):
            ctx.crypt_host(ms.MS_ENCRYPT, h, 0, n, chunk_bytes=256 * PAGE, n_streams=2)
        ctx.sync_checked()
        h.copy_(torch.from_numpy(plain))
        ctx.crypt_host(ms.MS_ENCRYPT, h, 0, n, chunk_bytes=256 * PAGE, n_streams=2)
    ids = np.arange(n, dtype=np.uint64)
    assert np.array_equal(h.numpy(), oracle_expected(key1, plain, ids, ids))


def test_batch_graph_failure_then_retry(ms, key1):
    n = 64
    plain = synth.page_bytes(123, 0, n)
    d = torch.from_numpy(plain).cuda()
    ids = np.arange(n, dtype=np.uint64)
    with ms.Context(key1, stream=torch.cuda.current_stream()) as ctx, ctx.batch(capacity=128) as b:
        assert b.add(ms.MS_ENCRYPT, ms.pages_array(d.data_ptr() + PAGE * ids, ids)) == ms.MS_OK
        ms.inject_fault(ms.MS_FAULT_GRAPH, 0, ERR)
        with pytest.raises(ms.MemShieldError):
            b.submit()
        b.submit()                                          # the queued requests are still there
        ctx.sync_checked()
        assert b.stats()["submits"] == 1
    assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, ids, ids))


def test_server_failure_fails_requests_cleanly(ms, key1):
    n = 256
    plain = synth.page_bytes(124, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    with ms.Context(key1) as ctx:
        srv = ms.Server(ctx, h, n)
        ms.inject_fault(ms.MS_FAULT_SERVER, 0, ERR)
        t = srv.submit(ms.MS_ENCRYPT, [3, 4, 5])
        with pytest.raises(ms.MemShieldError) as e:
            srv.wait(t, 5000)
        assert e.value.code == ms.MS_ECUDA
        with pytest.raises(ms.MemShieldError):
            srv.submit(ms.MS_ENCRYPT, [6])                  # a failed server takes no new work
        srv.destroy()
        with ms.Server(ctx, h, n) as srv2:                  # a new server on the same context works
            srv2.wait(srv2.submit(ms.MS_ENCRYPT, [7, 8]))
    want = plain.copy()
    oracle.crypt_pages(key1, want, np.array([7, 8]), np.array([7, 8]))
    assert np.array_equal(h.numpy(), want)
