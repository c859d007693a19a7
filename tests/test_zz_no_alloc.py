"""The allocation-free entry point (ms_crypt_pages_noalloc) against ms_encrypt_pages
and against the oracle.

Some callers cannot allocate device memory at the moment they encrypt or
decrypt a page -- for example code resolving a page fault, where cudaMalloc
can stall the device or fail because a caching allocator holds the memory.
ms_crypt_pages_noalloc serves them from a fixed device array inside the
library.  This file runs last so that a failure here never hides the other
tests; it must pass on its own in a fresh process as well.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PAGE = 4096


@pytest.fixture(scope="module")
def ms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_09252_b300 import memshield
    return memshield


def run_both(ms, ctx, plain, slots, ids, op):
    """Apply the same list through the no-alloc call and through ms_encrypt_pages."""
    a = torch.from_numpy(plain).cuda()
    b = torch.from_numpy(plain).cuda()
    la = ms.pages_array(a.data_ptr() + PAGE * slots.astype(np.uint64), ids)
    lb = ms.pages_array(b.data_ptr() + PAGE * slots.astype(np.uint64), ids)
    ctx.crypt_pages_noalloc(op, la)          # waits for its own kernel
    ctx.encrypt_pages(lb)
    ctx.sync_checked()
    return a, b


def test_noalloc_matches_existing_entry_point_twice(ms):
    key = synth.key_bytes(1)
    with ms.Context(key, stream=torch.cuda.current_stream()) as ctx:
        # first call: a long scattered list
        n_slots, n1 = 3000, 2500
        plain = synth.page_bytes_fast(31, 0, n_slots)
        slots = synth.scattered_slots(32, n_slots, n1)
        ids = synth.splitmix64(33, 0, n1).astype(np.uint64)
        a, b = run_both(ms, ctx, plain, slots, ids, ms.MS_ENCRYPT)
        assert torch.equal(a, b)
        assert not torch.equal(a, torch.from_numpy(plain).cuda())
        # second call in a row: a shorter list, so stale entries from the first
        # call sit past its end in the shared array and must be ignored
        n2 = 700
        slots2 = synth.scattered_slots(34, n_slots, n2)
        ids2 = np.arange(n2, dtype=np.uint64) + 10**12
        a2, b2 = run_both(ms, ctx, plain, slots2, ids2, ms.MS_DECRYPT)
        assert torch.equal(a2, b2)
        untouched = np.setdiff1d(np.arange(n_slots), slots2)
        idx = torch.from_numpy(untouched).cuda()
        assert torch.equal(a2.view(n_slots, PAGE)[idx], torch.from_numpy(plain).cuda().view(n_slots, PAGE)[idx])


def test_noalloc_limits_and_bad_entries(ms):
    key = synth.key_bytes(1)
    plain = synth.page_bytes(35, 0, 4)
    d = torch.from_numpy(plain).cuda()
    ids = np.arange(4, dtype=np.uint64)
    with ms.Context(key, stream=torch.cuda.current_stream()) as ctx:
        too_many = ms.pages_array(np.full(ms.MS_NOALLOC_MAX_PAGES + 1, d.data_ptr(), np.uint64),
                                  np.arange(ms.MS_NOALLOC_MAX_PAGES + 1))
        with pytest.raises(ms.MemShieldError) as e:
            ctx.crypt_pages_noalloc(ms.MS_ENCRYPT, too_many)
        assert e.value.code == ms.MS_ERANGE
        bad = ms.pages_array(d.data_ptr() + PAGE * ids, ids)
        bad["addr"][3] += 4
        with pytest.raises(ms.MemShieldError) as e:
            ctx.crypt_pages_noalloc(ms.MS_ENCRYPT, bad)
        assert e.value.code == ms.MS_EINVAL
        ctx.crypt_pages_noalloc(ms.MS_ENCRYPT, ms.pages_array([], []))   # n = 0: no-op
        ctx.sync_checked()
        assert torch.equal(d, torch.from_numpy(plain).cuda())


def test_noalloc_matches_the_oracle_at_the_largest_list(ms):
    """A list of exactly MS_NOALLOC_MAX_PAGES scattered pages (the last entry
    sits at the end of the shared array), ids unrelated to the slots and a
    non-zero domain word, twice in a row: each result against the oracle."""
    oracle.build()
    key = synth.key_bytes(1)
    n = ms.MS_NOALLOC_MAX_PAGES
    n_slots = n + 1024
    plain = synth.page_bytes_fast(36, 0, n_slots)
    slots = synth.scattered_slots(37, n_slots, n)
    ids = synth.splitmix64(38, 0, n).astype(np.uint64)
    dom = 0x9E3779B9
    d = torch.from_numpy(plain).cuda()
    lst = ms.pages_array(d.data_ptr() + PAGE * slots.astype(np.uint64), ids)
    want = plain.copy()
    oracle.crypt_pages(key, want, slots, ids, domain=dom, threads=8)
    with ms.Context(key, stream=torch.cuda.current_stream(), domain=dom) as ctx:
        ctx.crypt_pages_noalloc(ms.MS_ENCRYPT, lst)
        assert np.array_equal(d.cpu().numpy(), want)
        ctx.crypt_pages_noalloc(ms.MS_DECRYPT, lst)
        assert np.array_equal(d.cpu().numpy(), plain)


def test_noalloc_rejects_repeated_pages_when_asked(ms):
    """With check_duplicates the call refuses a list that names a page twice,
    as ms_encrypt_pages does, and changes nothing; without it the same list is
    accepted (its result is then undefined, so it is not compared)."""
    key = synth.key_bytes(1)
    plain = synth.page_bytes(39, 0, 8)
    d = torch.from_numpy(plain).cuda()
    slots = np.array([0, 1, 2, 3, 4, 5, 6, 2], dtype=np.uint64)
    lst = ms.pages_array(d.data_ptr() + PAGE * slots, slots)
    with ms.Context(key, stream=torch.cuda.current_stream(), check_duplicates=True) as ctx:
        with pytest.raises(ms.MemShieldError) as e:
            ctx.encrypt_pages(lst)
        assert e.value.code == ms.MS_EINVAL
        with pytest.raises(ms.MemShieldError) as e:
            ctx.crypt_pages_noalloc(ms.MS_ENCRYPT, lst)
        assert e.value.code == ms.MS_EINVAL
        ctx.sync_checked()
        assert np.array_equal(d.cpu().numpy(), plain)
        ok = lst[:7]                           # the same pages without the repeat go through
        ctx.crypt_pages_noalloc(ms.MS_ENCRYPT, ok)
        want = plain.copy()
        oracle.build()
        oracle.crypt_pages(key, want, slots[:7], slots[:7])
        assert np.array_equal(d.cpu().numpy(), want)


def test_noalloc_refuses_a_capturing_stream(ms):
    """The call waits for its own kernel, which a stream under capture cannot
    do: it returns MS_EINVAL before touching the stream, the capture stays
    valid, and the context works once the capture has ended."""
    key = synth.key_bytes(1)
    plain = synth.page_bytes(40, 0, 4)
    d = torch.from_numpy(plain).cuda()
    ids = np.arange(4, dtype=np.uint64)
    lst = ms.pages_array(d.data_ptr() + PAGE * ids, ids)
    side = torch.cuda.Stream()
    x = torch.zeros(16, device="cuda")
    with ms.Context(key, stream=side) as ctx:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            rc = ms.lib.ms_crypt_pages_noalloc(ctx.handle, ms.MS_ENCRYPT, lst.ctypes.data, 4)
            x.add_(1)                          # the capture still records work of its own
        assert rc == ms.MS_EINVAL
        g.replay()
        torch.cuda.synchronize()
        assert float(x[0]) == 1.0
        assert np.array_equal(d.cpu().numpy(), plain)
        ctx.crypt_pages_noalloc(ms.MS_ENCRYPT, lst)
        want = plain.copy()
        oracle.build()
        oracle.crypt_pages(key, want, ids, ids)
        assert np.array_equal(d.cpu().numpy(), want)
