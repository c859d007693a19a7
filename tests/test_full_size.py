"""Parity at the full sizes of the host-streaming (4 GiB pinned host buffer,
compared whole) and serving (16 GiB pinned working set, sampled pages)
configurations, in the launch configurations the benchmark uses."""
import numpy as np
import pytest

import oracle
import synth
from helpers import PAGE

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


@pytest.mark.parametrize("form,rate,n_req", [("continuous", 1.41e5, 17625), ("resident", 2e6, 250000)])
def test_serving_config_16gib(ms, key1, form, rate, n_req):
    """The serving mix over the 16 GiB working set (seed 5): one second at
    141k pages/s through continuous batching, and one second at 2M pages/s
    through resident workers (8 workers, in place). Every touched page ends as
    the closed form says (odd number of applications = encrypted)."""
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
    touched = np.nonzero(counts)[0]
    pick = touched[(synth.splitmix64(132, 0, 256) % np.uint64(len(touched))).astype(np.int64)]
    wv = ws.numpy().reshape(n, PAGE)
    for p in pick:
        pg = synth.page_bytes(5, int(p), 1)
        if counts[p] % 2:
            oracle.page_xor(key1, int(p), pg)
        assert np.array_equal(wv[p], pg), f"page {p}"
    untouched = np.setdiff1d(np.arange(0, n, 65537), touched)
    for p in untouched[:16]:
        assert np.array_equal(wv[p], synth.page_bytes(5, int(p), 1))
