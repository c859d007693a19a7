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


@pytest.mark.parametrize("site,n", [("launch", 32), ("launch", 2000), ("copy", 2000)])
def test_one_launch_form_recovers(ms, key1, site, n):
    # 32 entries travel in the kernel parameters; 2000 take the staged copy
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


def test_host_in_place_launch_failure(ms, key1):
    """A failed launch of the host-link kernel (ms_crypt_host_inplace) leaves
    the pinned pages untouched, reports the error, and the next call works."""
    n = 300
    plain = synth.page_bytes(123, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    with ms.Context(key1) as ctx:
        ms.inject_fault(ms.MS_FAULT_LAUNCH, 0, ERR)
        with pytest.raises(ms.MemShieldError) as e:
            ctx.crypt_host_inplace(ms.MS_ENCRYPT, h, 0, n)
        assert e.value.code == ms.MS_ECUDA and ctx.last_cuda_error() == ERR
        ctx.sync_checked()
        assert np.array_equal(h.numpy(), plain)
        ctx.crypt_host_inplace(ms.MS_ENCRYPT, h, 0, n)
        ctx.sync_checked()
    ids = np.arange(n, dtype=np.uint64)
    assert np.array_equal(h.numpy(), oracle_expected(key1, plain, ids, ids))


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


def test_server_replay_failure_returns_cleanly(ms, key1):
    """A wave that fails in the middle of an open-loop replay ends the replay with
    MS_ECUDA; requests still outstanding no longer write to the caller's latency
    array, and the context serves a new server afterwards."""
    n = 512
    plain = synth.page_bytes(125, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    n_req = 200
    arrival = np.linspace(0.0, 0.004, n_req)
    ops = np.full(n_req, ms.MS_ENCRYPT, dtype=np.int32)
    offsets = np.arange(n_req + 1, dtype=np.uint64)
    pages = np.arange(n_req, dtype=np.uint64)
    with ms.Context(key1) as ctx:
        srv = ms.Server(ctx, h, n, mode=ms.MS_SERVE_ONE_PER_LAUNCH)
        ms.inject_fault(ms.MS_FAULT_SERVER, 20, ERR)        # the 21st wave fails
        with pytest.raises(ms.MemShieldError) as e:
            srv.replay(arrival, ops, offsets, pages, timeout_ms=5000)
        assert e.value.code == ms.MS_ECUDA
        srv.destroy()
        with ms.Server(ctx, h, n) as srv2:
            srv2.wait(srv2.submit(ms.MS_ENCRYPT, [n - 1]))
    last = slice((n - 1) * PAGE, n * PAGE)
    want = oracle_expected(key1, plain[last], np.array([0]), np.array([n - 1]))
    assert np.array_equal(h.numpy()[last], want)


def test_server_replay_checks_every_request_first(ms, key1):
    n = 64
    h = torch.zeros(n * PAGE, dtype=torch.uint8).pin_memory()
    arrival = np.zeros(3)
    ops = np.full(3, ms.MS_ENCRYPT, dtype=np.int32)
    with ms.Context(key1) as ctx, ms.Server(ctx, h, n) as srv:
        for offsets, pages in (([0, 1, 2, 3], [1, 2, n]),       # page out of range in the last request
                               ([0, 1, 1, 2], [1, 2]),          # empty request
                               ([0, 1, 3, 4], [1, 2, 2, 3])):   # page repeated within a request
            with pytest.raises(ms.MemShieldError) as e:
                srv.replay(arrival, ops, np.array(offsets, dtype=np.uint64), np.array(pages, dtype=np.uint64))
            assert e.value.code == ms.MS_EINVAL
        assert srv.stats()["requests_done"] == 0                 # nothing was submitted
    assert not h.numpy().any()
