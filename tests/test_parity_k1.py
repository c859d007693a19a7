"""GPU parity of the one-launch page kernel (K1) against the CPU oracle: bit-exact."""
import numpy as np
import pytest

import synth
from helpers import PAGE, oracle_expected, oracle_pages, sample_pages

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_09252_b300 import memshield
    return memshield


def dev(a: np.ndarray):
    return torch.from_numpy(a).cuda()


def make_ctx(ms, key, **kw):
    return ms.Context(key, stream=torch.cuda.current_stream().cuda_stream, **kw)


def test_small_config_encrypt_then_decrypt(ms, key1):
    """256 pages of seed 0, ids 0..255, one encrypt launch then one decrypt launch."""
    n = 256
    plain = synth.page_bytes(0, 0, n)
    d = dev(plain)
    base = d.data_ptr()
    ids = np.arange(n, dtype=np.uint64)
    pages = ms.pages_array(base + PAGE * ids, ids)
    with make_ctx(ms, key1) as ctx:
        ctx.encrypt_pages(pages)
        ctx.sync_checked()
        got = d.cpu().numpy()
        want = oracle_expected(key1, plain, ids, ids)
        assert np.array_equal(got, want)
        ctx.decrypt_pages(pages)
        ctx.sync_checked()
        assert np.array_equal(d.cpu().numpy(), plain)


SHAPES = [(b, u, p) for (b, u, p) in [
    (1, 1, 0), (1, 2, 0), (1, 10, 0), (1, 1, 1), (1, 2, 1), (1, 10, 1), (1, 1, 2), (1, 2, 2), (1, 10, 2),
    (2, 2, 0), (2, 10, 0), (2, 2, 1), (2, 10, 1), (2, 2, 2), (2, 10, 2),
    (4, 2, 1), (4, 10, 1), (4, 2, 2), (4, 10, 2),
    (1, 10, 3), (2, 10, 3), (4, 10, 3), (1, 2, 3), (1, 10, 4), (2, 10, 4), (4, 10, 4),
    (1, 10, 5), (2, 10, 5), (4, 10, 5), (1, 10, 6), (2, 10, 6), (4, 10, 6),
    (1, 10, 7), (2, 10, 7), (4, 10, 7)]]


@pytest.mark.parametrize("bpt,unr,pol", SHAPES)
@pytest.mark.parametrize("tpc", [128, 512])
def test_every_shape_scattered_ragged(ms, key1, bpt, unr, pol, tpc):
    """Every compiled shape on a ragged, scattered list with ids that differ from slots."""
    n_slots, n = 97, 61                      # 61 pages: several CTAs and a ragged tail
    plain = synth.page_bytes(7, 0, n_slots)
    d = dev(plain)
    slots = synth.scattered_slots(8, n_slots, n)
    ids = (synth.splitmix64(9, 0, n)).astype(np.uint64)   # full 64-bit ids
    pages = ms.pages_array(d.data_ptr() + PAGE * slots.astype(np.uint64), ids)
    with make_ctx(ms, key1) as ctx:
        ctx.set_shape(bpt, tpc, unr, pol)
        assert ctx.get_shape() == {"blocks_per_thread": bpt, "threads_per_cta": tpc, "dr_unroll": unr,
                                   "rot_policy": pol, "hoist": 0}
        ctx.encrypt_pages(pages)
        ctx.sync_checked()
    assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, slots, ids))


@pytest.mark.parametrize("rounds,bpt,pol", [(20, 2, 1), (20, 4, 1), (20, 2, 0), (20, 4, 0), (12, 2, 1),
                                            (12, 4, 1), (8, 2, 1), (8, 4, 1)])
@pytest.mark.parametrize("tpc", [128, 512])
def test_hoisted_prelude_shapes(ms, key1, rounds, bpt, pol, tpc):
    """The shapes that compute the counter-free prelude once per page, in list and range mode."""
    n_slots, n = 97, 61
    plain = synth.page_bytes(17, 0, n_slots)
    d = dev(plain)
    slots = synth.scattered_slots(18, n_slots, n)
    ids = (synth.splitmix64(19, 0, n)).astype(np.uint64)
    with make_ctx(ms, key1, rounds=rounds, domain=77) as ctx:
        ctx.set_shape(bpt, tpc, rounds // 2, pol, 1)
        assert ctx.get_shape()["hoist"] == 1
        ctx.encrypt_pages(ms.pages_array(d.data_ptr() + PAGE * slots.astype(np.uint64), ids))
        ctx.sync_checked()
        assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, slots, ids, domain=77, rounds=rounds))
        r = dev(plain)
        ctx.crypt_range(ms.MS_ENCRYPT, r, 1 << 40, n_slots)
        ctx.sync_checked()
        ids_r = (np.arange(n_slots, dtype=np.uint64) + np.uint64(1 << 40))
        assert np.array_equal(r.cpu().numpy(), oracle_expected(key1, plain, np.arange(n_slots), ids_r, domain=77,
                                                               rounds=rounds))
    with make_ctx(ms, key1) as ctx:
        with pytest.raises(ms.MemShieldError):
            ctx.set_shape(1, 256, 10, 1, 1)         # hoisting needs >= 2 blocks per thread


@pytest.mark.parametrize("rounds", [8, 12])
def test_reduced_rounds(ms, key1, rounds):
    n = 33
    plain = synth.page_bytes(10, 0, n)
    d = dev(plain)
    ids = np.arange(100, 100 + n, dtype=np.uint64)
    slots = np.arange(n, dtype=np.uint64)
    with make_ctx(ms, key1, rounds=rounds) as ctx:
        ctx.encrypt_pages(ms.pages_array(d.data_ptr() + PAGE * slots, ids))
        ctx.sync_checked()
    assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, slots, ids, rounds=rounds))


def test_domain_word(ms, key1):
    n = 8
    plain = synth.page_bytes(11, 0, n)
    d = dev(plain)
    ids = np.arange(n, dtype=np.uint64)
    with make_ctx(ms, key1, domain=0xDEADBEEF) as ctx:
        ctx.encrypt_pages(ms.pages_array(d.data_ptr() + PAGE * ids, ids))
        ctx.sync_checked()
    assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, ids, ids, domain=0xDEADBEEF))


def test_device_list_and_range_forms(ms, key1):
    n = 130
    plain = synth.page_bytes(12, 0, n)
    ids = np.arange(5000, 5000 + n, dtype=np.uint64)
    slots = np.arange(n, dtype=np.uint64)
    want = oracle_expected(key1, plain, slots, ids)
    with make_ctx(ms, key1) as ctx:
        d = dev(plain)
        lst = torch.from_numpy(ms.pages_array(d.data_ptr() + PAGE * slots, ids).view(np.uint8)).cuda()
        ctx.encrypt_pages_dev(lst, n)
        assert ctx.sync() == 0
        assert np.array_equal(d.cpu().numpy(), want)
        d2 = dev(plain)
        ctx.crypt_range(ms.MS_ENCRYPT, d2, 5000, n)
        assert ctx.sync() == 0
        assert np.array_equal(d2.cpu().numpy(), want)
        ctx.crypt_range(ms.MS_DECRYPT, d2, 5000, n)
        assert ctx.sync() == 0
        assert np.array_equal(d2.cpu().numpy(), plain)


def test_empty_and_bad_entries(ms, key1):
    n = 4
    plain = synth.page_bytes(13, 0, n)
    d = dev(plain)
    ids = np.arange(n, dtype=np.uint64)
    with make_ctx(ms, key1) as ctx:
        ctx.encrypt_pages(ms.pages_array([], []))          # n = 0 is a no-op
        ctx.crypt_range(ms.MS_ENCRYPT, d, 0, 0)
        assert ctx.sync() == 0
        assert np.array_equal(d.cpu().numpy(), plain)
        bad = ms.pages_array(d.data_ptr() + PAGE * ids, ids)
        bad["addr"][2] += 8                                  # misaligned: rejected on the host
        with pytest.raises(ms.MemShieldError) as e:
            ctx.encrypt_pages(bad)
        assert e.value.code == ms.MS_EINVAL
        assert ctx.sync() == 0
        assert np.array_equal(d.cpu().numpy(), plain)       # nothing was launched
        # device-side check: the bad entry is skipped, the others are processed
        lst = ms.pages_array(d.data_ptr() + PAGE * ids, ids)
        lst["addr"][1] = 0
        dl = torch.from_numpy(lst.view(np.uint8)).cuda()
        ctx.encrypt_pages_dev(dl, n)
        assert ctx.sync() == ms.MS_EINVAL
        assert ctx.sync() == 0                               # the status word was cleared
        want = oracle_expected(key1, plain, np.array([0, 2, 3], np.uint64), np.array([0, 2, 3], np.uint64))
        assert np.array_equal(d.cpu().numpy(), want)
        with pytest.raises(ms.MemShieldError):
            ctx.crypt_range(7, d, 0, 1)                      # bad op


def test_duplicate_check(ms, key1):
    plain = synth.page_bytes(14, 0, 2)
    d = dev(plain)
    with make_ctx(ms, key1, check_duplicates=True) as ctx:
        dup = ms.pages_array([d.data_ptr(), d.data_ptr()], [0, 1])
        with pytest.raises(ms.MemShieldError):
            ctx.encrypt_pages(dup)


def test_list_longer_than_staging_slot(ms, key1):
    """A host list longer than one staging slot (and than the parameter-space
    limit of 1024 entries) is cut into several staged launches."""
    n = 1500
    plain = synth.page_bytes(15, 0, n)
    d = dev(plain)
    ids = np.arange(n, dtype=np.uint64)
    with make_ctx(ms, key1, list_capacity=64) as ctx:
        for _ in range(3):                                   # odd count: encrypted once net
            ctx.encrypt_pages(ms.pages_array(d.data_ptr() + PAGE * ids, ids))
        ctx.sync_checked()
    assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, ids, ids))


@pytest.mark.parametrize("rounds", [20, 12, 8])
@pytest.mark.parametrize("n", [1, 16, 17, 128, 129, 1000, 1024, 1025])
def test_short_host_lists_in_kernel_parameters(ms, key1, n, rounds):
    """Host lists of up to 1024 entries travel in the kernel's parameters (16-,
    128- and 1024-entry blocks); 1025 takes the staged path.  Scattered slots,
    full 64-bit ids, a non-zero domain."""
    n_slots = n + 37
    plain = synth.page_bytes(150 + n, 0, n_slots)
    d = dev(plain)
    slots = synth.scattered_slots(151 + n, n_slots, n)
    ids = synth.splitmix64(152 + n, 0, n).astype(np.uint64)
    with make_ctx(ms, key1, rounds=rounds, domain=0x5A5A5A5A) as ctx:
        ctx.encrypt_pages(ms.pages_array(d.data_ptr() + PAGE * slots.astype(np.uint64), ids))
        ctx.sync_checked()
        want = oracle_expected(key1, plain, slots, ids, domain=0x5A5A5A5A, rounds=rounds)
        assert np.array_equal(d.cpu().numpy(), want)
        ctx.decrypt_pages(ms.pages_array(d.data_ptr() + PAGE * slots.astype(np.uint64), ids))
        ctx.sync_checked()
        assert np.array_equal(d.cpu().numpy(), plain)


def test_short_host_lists_back_to_back(ms, key1):
    """Many short launches queued without a wait: every parameter block is the
    caller's list at the time of the call, even though the caller reuses its
    array at once."""
    n_slots = 4096
    plain = synth.page_bytes(160, 0, n_slots)
    d = dev(plain)
    lst = ms.pages_array(np.zeros(8, np.uint64), np.zeros(8, np.uint64))
    with make_ctx(ms, key1) as ctx:
        for r in range(n_slots // 8):
            sl = np.arange(8 * r, 8 * r + 8, dtype=np.uint64)
            lst["addr"] = d.data_ptr() + PAGE * sl
            lst["page_id"] = sl
            ctx.encrypt_pages(lst)
        ctx.sync_checked()
    all_ = np.arange(n_slots)
    assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, all_, all_))


def test_extreme_ids_and_domains(ms, key1):
    """Ids at the edges of the 64-bit range (nonce words 13 and 14 all ones, or
    one of them zero) and the largest domain word, through the host list, the
    device list and the range form; a range whose ids would wrap is refused."""
    ids = np.array([0, 1, 2**32 - 1, 2**32, 2**63, 2**64 - 2, 2**64 - 1, 0xFFFFFFFF00000000], dtype=np.uint64)
    n = ids.size
    plain = synth.page_bytes(170, 0, n)
    slots = np.arange(n, dtype=np.uint64)
    for dom in (0, 0xFFFFFFFF):
        want = oracle_expected(key1, plain, slots, ids, domain=dom)
        with make_ctx(ms, key1, domain=dom) as ctx:
            d = dev(plain)
            ctx.encrypt_pages(ms.pages_array(d.data_ptr() + PAGE * slots, ids))
            ctx.sync_checked()
            assert np.array_equal(d.cpu().numpy(), want)
            d = dev(plain)
            lst = torch.from_numpy(ms.pages_array(d.data_ptr() + PAGE * slots, ids).view(np.uint8)).cuda()
            ctx.encrypt_pages_dev(lst, n)
            ctx.sync_checked()
            assert np.array_equal(d.cpu().numpy(), want)
            d = dev(plain[:2 * PAGE])                      # the last two ids of the space
            ctx.crypt_range(ms.MS_ENCRYPT, d, 2**64 - 2, 2)
            ctx.sync_checked()
            assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain[:2 * PAGE], np.arange(2), ids[5:7],
                                                                   domain=dom))
            with pytest.raises(ms.MemShieldError) as e:   # 2^64 - 1, then 0: refused, nothing runs
                ctx.crypt_range(ms.MS_ENCRYPT, d, 2**64 - 1, 2)
            assert e.value.code == ms.MS_EINVAL
            h = torch.from_numpy(plain[:2 * PAGE].copy()).pin_memory()
            with pytest.raises(ms.MemShieldError):
                ctx.crypt_host(ms.MS_ENCRYPT, h, 2**64 - 1, 2)
            assert np.array_equal(h.numpy(), plain[:2 * PAGE])


@pytest.mark.slow
def test_bulk_1gib_whole(ms, key1):
    """The 1 GiB bulk configuration in the launch shape the benchmark times:
    262,144 pages of seed 2, ids 0..262143, one encrypt then one decrypt launch.
    The whole encrypted GiB is compared with the oracle's (run over all host
    cores), and the round trip restores the input."""
    import os
    n = 262144
    plain = synth.page_bytes_fast(2, 0, n)
    d = dev(plain)
    ids = np.arange(n, dtype=np.uint64)
    lst = torch.from_numpy(ms.pages_array(d.data_ptr() + PAGE * ids, ids).view(np.uint8)).cuda()
    with make_ctx(ms, key1) as ctx:
        ctx.encrypt_pages_dev(lst, n)
        ctx.sync_checked()
        got = d.cpu().numpy()
        want = oracle_expected(key1, plain, ids, ids, threads=max(1, os.cpu_count() or 1))
        bad = np.nonzero((got.reshape(n, PAGE) != want.reshape(n, PAGE)).any(axis=1))[0]
        assert bad.size == 0, f"{bad.size} pages differ, first {bad[:8]}"
        ctx.decrypt_pages_dev(lst, n)
        ctx.sync_checked()
        assert torch.equal(d, torch.from_numpy(plain).cuda())


def test_host_streamed_pages(ms, key1):
    """Host pages streamed through the device in chunks on two streams."""
    n = 3000                                                   # 11.7 MiB, ragged last chunk
    plain = synth.page_bytes_fast(4, 0, n)
    h = torch.from_numpy(plain.copy()).pin_memory()
    with make_ctx(ms, key1) as ctx:
        ctx.crypt_host(ms.MS_ENCRYPT, h, 0, n, chunk_bytes=2 << 20, n_streams=2)
        sample = sample_pages(22, n, 64)
        assert np.array_equal(h.numpy().reshape(n, PAGE)[sample], oracle_pages(key1, 4, sample, sample))
        for ns in (1, 3, 4):
            ctx.crypt_host(ms.MS_DECRYPT, h, 0, n, chunk_bytes=4096 * 7, n_streams=ns)
            ctx.crypt_host(ms.MS_ENCRYPT, h, 0, n, chunk_bytes=1 << 20, n_streams=ns)
        ctx.crypt_host(ms.MS_DECRYPT, h, 0, n)
        assert np.array_equal(h.numpy(), plain)


def test_launches_follow_the_callers_stream(ms, key1):
    """With the caller's stream given (torch's default stream has handle 0), later
    work on that stream sees the encrypted bytes without any ms_sync."""
    n = 16384                                                  # 64 MiB: long enough to race
    plain = synth.page_bytes_fast(16, 0, n)
    d = dev(plain)
    with make_ctx(ms, key1) as ctx:
        assert torch.cuda.current_stream().cuda_stream == 0 or True
        ctx.crypt_range(ms.MS_ENCRYPT, d, 0, n)
        snap = d.clone()                                       # same stream, no ms_sync
        ctx.sync_checked()
        assert torch.equal(snap, d)
        assert not torch.equal(snap[:PAGE], torch.from_numpy(plain[:PAGE]).cuda())


def test_launch_size_beyond_grid_limit_is_rejected_before_launch(ms, key1):
    """A page count whose grid exceeds the launch limit is refused on the host
    (MS_ECUDA, invalid configuration) and nothing is launched."""
    d = torch.zeros(PAGE, dtype=torch.uint8, device="cuda")
    with make_ctx(ms, key1) as ctx:
        with pytest.raises(ms.MemShieldError) as e:
            ctx.crypt_range(ms.MS_ENCRYPT, d, 0, 1 << 40)   # 2^40 pages: grid far above 2^31 - 1
        assert e.value.code == ms.MS_ECUDA and ctx.last_cuda_error() == 9   # cudaErrorInvalidConfiguration
        ctx.sync_checked()
        assert int(d.sum()) == 0


def test_random_key_from_the_os(ms):
    """key = NULL draws the key with getrandom (Sec. 4.4): two contexts give
    different ciphertexts, each decrypts its own, and neither is the plaintext."""
    n = 8
    plain = synth.page_bytes(140, 0, n)
    ids = np.arange(n, dtype=np.uint64)
    outs = []
    for _ in range(2):
        d = dev(plain)
        with ms.Context(None, stream=torch.cuda.current_stream().cuda_stream) as ctx:
            ctx.encrypt_pages(ms.pages_array(d.data_ptr() + PAGE * ids, ids))
            ctx.sync_checked()
            outs.append(d.cpu().numpy())
            ctx.decrypt_pages(ms.pages_array(d.data_ptr() + PAGE * ids, ids))
            ctx.sync_checked()
            assert np.array_equal(d.cpu().numpy(), plain)
    assert not np.array_equal(outs[0], outs[1])
    assert not np.array_equal(outs[0], plain)


def test_ticketed_submissions(ms, key1):
    """ms_submit_host / ms_poll / ms_wait: per-submission completion, on device
    pages and on pinned host pages the kernel works on in place."""
    n = 600
    plain = synth.page_bytes(175, 0, n)
    d = dev(plain)
    h = torch.from_numpy(plain.copy()).pin_memory()
    hbase = ms.host_device_address(h)
    with ms.Context(key1) as ctx:
        tickets = []
        for lo in range(0, n, 100):                     # six requests of 100 pages, each side
            ids = np.arange(lo, lo + 100, dtype=np.uint64)
            tickets.append(ctx.submit_host(ms.MS_ENCRYPT, ms.pages_array(d.data_ptr() + PAGE * ids, ids)))
            tickets.append(ctx.submit_host(ms.MS_ENCRYPT, ms.pages_array(hbase + PAGE * ids, ids)))
        assert tickets == list(range(tickets[0], tickets[0] + len(tickets)))
        for t in tickets:
            ctx.wait(t, 10000)
            assert ctx.poll(t) == 1
        marker = ctx.submit_host(ms.MS_ENCRYPT, ms.pages_array([], []))   # empty: completes after the rest
        ctx.wait(marker)
        assert ctx.poll(marker + 1) == ms.MS_EINVAL                        # never issued
        with pytest.raises(ms.MemShieldError):
            ms.host_device_address(d)                                       # device memory is not host memory
    all_ = np.arange(n, dtype=np.uint64)
    want = oracle_expected(key1, plain, all_, all_)
    assert np.array_equal(d.cpu().numpy(), want)
    assert np.array_equal(h.numpy(), want)


def test_concurrent_submitters_on_one_context(ms, key1):
    """Four host threads submit and wait on one context at once (the paper's
    many clients feeding one GPU module): every thread's pages end as the
    oracle says, and every ticket completes."""
    import threading
    n_threads, per, reqs = 4, 800, 200
    n = n_threads * per
    plain = synth.page_bytes_fast(177, 0, n)
    d = dev(plain)
    torch.cuda.synchronize()
    errors = []
    with ms.Context(key1) as ctx:
        def client(k):
            try:
                rng_sizes = (synth.splitmix64(178 + k, 0, reqs) % np.uint64(4) + np.uint64(1)).astype(int)
                pages = synth.scattered_slots(190 + k, per, int(rng_sizes.sum())).astype(np.uint64) + np.uint64(k * per)
                off = 0
                for sz in rng_sizes:
                    sl = pages[off:off + sz]
                    t = ctx.submit_host(ms.MS_ENCRYPT, ms.pages_array(d.data_ptr() + PAGE * sl, sl))
                    ctx.wait(t, 10000)
                    off += sz
                rest = np.setdiff1d(np.arange(k * per, (k + 1) * per, dtype=np.uint64), pages)
                ctx.encrypt_pages(ms.pages_array(d.data_ptr() + PAGE * rest, rest))   # the rest, untracked
            except Exception as e:  # surfaced below
                errors.append(e)
        th = [threading.Thread(target=client, args=(k,)) for k in range(n_threads)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        ctx.sync_checked()
    assert not errors, errors
    all_ = np.arange(n, dtype=np.uint64)
    assert np.array_equal(d.cpu().numpy(), oracle_expected(key1, plain, all_, all_))
