"""In-place host pages (ms_crypt_host_inplace): the bounded-grid kernel that
works on pinned, mapped host memory over the host link, against the oracle
at sizes below, at and above one grid step (16 CTAs x 512 threads = 128
pages), with a ragged last step, for every round count, a domain word and
ids at the top of the 64-bit range; memory that is not pinned and mapped,
misaligned bases and wrapping ids are refused before any launch."""
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


@pytest.mark.parametrize("n", [1, 7, 127, 128, 129, 1000, 4097])
def test_matches_oracle(ms, key1, n):
    plain = synth.page_bytes_fast(130, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    first = 5000 + n
    with ms.Context(key1) as ctx:
        ctx.crypt_host_inplace(ms.MS_ENCRYPT, h, first, n)
        ctx.sync_checked()
    want = plain.copy()
    ids = np.arange(first, first + n, dtype=np.uint64)
    oracle.crypt_pages(key1, want, np.arange(n, dtype=np.uint64), ids, threads=8)
    assert np.array_equal(h.numpy(), want)


@pytest.mark.parametrize("rounds", [8, 12])
def test_round_counts_and_domain(ms, key1, rounds):
    n = 300
    plain = synth.page_bytes_fast(131, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    with ms.Context(key1, rounds=rounds, domain=0xA5A5) as ctx:
        ctx.crypt_host_inplace(ms.MS_DECRYPT, h, 0, n)
        ctx.sync_checked()
    want = plain.copy()
    ids = np.arange(n, dtype=np.uint64)
    oracle.crypt_pages(key1, want, ids, ids, domain=0xA5A5, rounds=rounds, threads=8)
    assert np.array_equal(h.numpy(), want)


def test_top_ids_and_round_trip(ms, key1):
    n = 200
    first = 2**64 - n                         # the last id is 2^64 - 1
    plain = synth.page_bytes_fast(132, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    with ms.Context(key1) as ctx:
        ctx.crypt_host_inplace(ms.MS_ENCRYPT, h, first, n)
        ctx.sync_checked()
        want = plain.copy()
        ids = np.arange(n, dtype=np.uint64) + np.uint64(first)
        oracle.crypt_pages(key1, want, np.arange(n, dtype=np.uint64), ids, threads=8)
        assert np.array_equal(h.numpy(), want)
        ctx.crypt_host_inplace(ms.MS_DECRYPT, h, first, n)
        ctx.sync_checked()
    assert np.array_equal(h.numpy(), plain)


def test_refusals(ms, key1):
    pageable = np.zeros(4 * PAGE, dtype=np.uint8)
    h = torch.zeros(4 * PAGE, dtype=torch.uint8).pin_memory()
    with ms.Context(key1) as ctx:
        for args, what in (((pageable, 0, 4), "pageable"), ((h.data_ptr() + 8, 0, 3), "misaligned"),
                           ((h, 2**64 - 2, 4), "wrapping ids"), ((h, 0, 4, 7), "bad op")):
            op = args[3] if len(args) == 4 else ms.MS_ENCRYPT
            with pytest.raises(ms.MemShieldError) as e:
                ctx.crypt_host_inplace(op, *args[:3])
            assert e.value.code == ms.MS_EINVAL, what
        ctx.crypt_host_inplace(ms.MS_ENCRYPT, h, 0, 0)   # n = 0: nothing to do
        ctx.sync_checked()
    assert not h.numpy().any()
    assert not pageable.any()
