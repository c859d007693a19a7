"""Parity at the full sizes of the host configuration (4 GiB pinned host
buffer, streamed through the copy engines and in place over the link) and
serving (16 GiB pinned working set) configurations, each compared whole
with the oracle, in the launch configurations the benchmark uses."""
import numpy as np
import pytest

import oracle
import synth
from helpers import PAGE, check_sampled_pages, check_whole_buffer

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def ms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_09252_b300 import memshield
    return memshield


def test_host_config_4gib(ms, key1):
    """1,048,576 pages of seed 4 streamed in 16 MiB chunks on 2 streams: the
    whole 4 GiB result against the oracle (run over all host cores), then the
    decrypted buffer against the input."""
    import os
    n = 1048576
    h = torch.empty(n * PAGE, dtype=torch.uint8).pin_memory()
    synth.fill_pages(h.data_ptr(), 4, 0, n)
    want = np.empty(n * PAGE, dtype=np.uint8)
    synth.fill_pages(want.ctypes.data, 4, 0, n)
    ids = np.arange(n, dtype=np.uint64)
    threads = max(1, os.cpu_count() or 1)
    with ms.Context(key1) as ctx:
        ctx.crypt_host(ms.MS_ENCRYPT, h, 0, n, 16 << 20, 2)
        oracle.crypt_pages(key1, want, ids, ids, threads=threads)
        assert np.array_equal(h.numpy(), want)
        ctx.crypt_host(ms.MS_DECRYPT, h, 0, n, 16 << 20, 2)
    oracle.crypt_pages(key1, want, ids, ids, threads=threads)  # the same XOR again: the input
    assert np.array_equal(h.numpy(), want)


def test_host_config_4gib_in_place(ms, key1):
    """The same 4 GiB buffer encrypted in place over the host link
    (ms_crypt_host_inplace, the bounded-grid kernel): the whole result
    against the oracle, then decrypted back to the input."""
    import os
    n = 1048576
    h = torch.empty(n * PAGE, dtype=torch.uint8).pin_memory()
    synth.fill_pages(h.data_ptr(), 4, 0, n)
    want = np.empty(n * PAGE, dtype=np.uint8)
    synth.fill_pages(want.ctypes.data, 4, 0, n)
    ids = np.arange(n, dtype=np.uint64)
    threads = max(1, os.cpu_count() or 1)
    with ms.Context(key1) as ctx:
        ctx.crypt_host_inplace(ms.MS_ENCRYPT, h, 0, n)
        ctx.sync_checked()
        oracle.crypt_pages(key1, want, ids, ids, threads=threads)
        assert np.array_equal(h.numpy(), want)
        ctx.crypt_host_inplace(ms.MS_DECRYPT, h, 0, n)
        ctx.sync_checked()
    oracle.crypt_pages(key1, want, ids, ids, threads=threads)
    assert np.array_equal(h.numpy(), want)


@pytest.mark.parametrize("form,rate,n_req", [("continuous", 1.41e5, 17625), ("continuous", 2e6, 250000),
                                             ("resident", 2e6, 250000)])
def test_serving_config_16gib(ms, key1, form, rate, n_req):
    """The serving mix over the 16 GiB working set (seed 5): one second at
    141k pages/s and one at 2M pages/s through continuous batching (in-place
    lane and entry-list waves), and one second at 2M pages/s through resident
    workers (8 workers, in place).  The whole 16 GiB result
    equals the closed form computed by the oracle (a page applied an odd
    number of times is encrypted, every other page unchanged), byte for byte
    and by SHA-256, and a seeded 1/16 of the touched pages, recomputed one by
    one, matches."""
    n = 4194304
    ws = torch.empty(n * PAGE, dtype=torch.uint8).pin_memory()
    synth.fill_pages(ws.data_ptr(), 5, 0, n)
    arrival, ops, offsets, pages = synth.serving_workload(5, n_req, rate, n)
    with ms.Context(key1) as ctx:
        if form == "resident":
            with ms.Resident(ctx, workers=8) as res:
                lat, makespan = res.replay(ws, n, arrival, offsets, pages)
        else:
            with ms.Server(ctx, ws, n) as srv:
                lat, makespan = srv.replay(arrival, ops, offsets, pages)
    assert (lat >= 0).all()
    counts = np.bincount(pages.astype(np.int64), minlength=n)
    odd = counts % 2 == 1
    touched = np.nonzero(counts)[0]
    wv = ws.numpy()
    got_sha, want_sha = check_whole_buffer(key1, 5, n, odd, lambda p0, m: wv[p0 * PAGE:(p0 + m) * PAGE])
    assert got_sha == want_sha
    k = check_sampled_pages(key1, 5, touched, odd, lambda pick: wv.reshape(n, PAGE)[pick], 132)
    assert k > len(touched) // 20
