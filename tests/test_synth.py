"""The seeded input generators: counter form = sequential form, numpy = C, recipe shapes."""
import numpy as np
import pytest

import synth


def test_counter_form_equals_sequential_splitmix():
    seed = 123456789
    state = seed
    seq = []
    for _ in range(16):
        state = (state + 0x9E3779B97F4A7C15) & (2**64 - 1)
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & (2**64 - 1)
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & (2**64 - 1)
        seq.append(z ^ (z >> 31))
    assert [int(v) for v in synth.splitmix64(seed, 0, 16)] == seq
    assert [int(v) for v in synth.splitmix64(seed, 5, 4)] == seq[5:9]


def test_numpy_and_c_fill_agree():
    a = synth.page_bytes(4, 1000, 9)
    b = synth.page_bytes_fast(4, 1000, 9)
    assert (a == b).all()
    big = synth.page_bytes_fast(5, 0, 40)      # crosses the threading threshold
    assert (big[4096 * 17:4096 * 18] == synth.page_bytes(5, 17, 1)).all()


def test_key_is_first_32_bytes_of_seed1():
    assert synth.key_bytes(1) == synth.page_bytes(1, 0, 1)[:32].tobytes()


def test_zipf_recipe():
    s = synth.zipf_sizes(3, 20000)
    assert s.min() >= 1 and s.max() <= 512
    assert abs(synth.zipf_mean() - 44.08) < 0.01
    assert abs(s.mean() - synth.zipf_mean()) < 3.0
    # P(size = 1) for Zipf(1.2) truncated at 512
    k = np.arange(1, 513, dtype=np.float64)
    p1 = 1.0 / (k ** -1.2).sum()
    assert abs((s == 1).mean() - p1) < 0.02


def test_scattered_slots_without_replacement():
    x = synth.scattered_slots(3, 1000, 900)
    assert len(np.unique(x)) == 900 and x.min() >= 0 and x.max() < 1000


def test_serving_recipe():
    arr, ops, off, pages = synth.serving_workload(5, 5000, 80000.0, 1 << 20)
    sizes = np.diff(off)
    assert abs((ops == 1).mean() - 0.8) < 0.03
    assert set(np.unique(sizes[ops == 1])) == {1}
    assert sizes[ops == 0].min() >= 8 and sizes[ops == 0].max() <= 64
    assert abs(sizes.mean() - 8.0) < 0.6
    assert np.all(np.diff(arr) >= 0)
    assert abs(len(arr) / arr[-1] - 10000.0) / 10000.0 < 0.05
    for r in range(0, 5000, 97):
        seg = pages[off[r]:off[r + 1]]
        assert len(np.unique(seg)) == len(seg)


@pytest.mark.parametrize("n_ws", [1 << 20, 4096, 70])
def test_serving_duplicates_fixed_as_walked(n_ws):
    """The duplicate fix-up finds its requests with one sort; the result is
    the same as walking every multi-page request in order, and every
    request's pages are distinct (small working sets force many repeats)."""
    arr, ops, off, pages = synth.serving_workload(9, 3000, 80000.0, n_ws)
    raw = (synth.splitmix64(9 ^ 0x3333, 0, int(off[-1])) % np.uint64(n_ws)).astype(np.int64)
    walked = raw.copy()
    for r in range(len(off) - 1):
        seg = walked[off[r]:off[r + 1]]
        if len(seg) > 1 and len(np.unique(seg)) != len(seg):
            seen = set()
            for i in range(len(seg)):
                v = int(seg[i])
                while v in seen:
                    v = (v + 1) % n_ws
                seen.add(v)
                seg[i] = v
    assert np.array_equal(pages, walked)
    for r in range(len(off) - 1):
        seg = pages[off[r]:off[r + 1]]
        assert len(np.unique(seg)) == len(seg)


def test_window_trace_recipe():
    n, length = 1000, 20000
    t = synth.window_trace(7, n, length)
    assert t.dtype == np.uint64 and len(t) == length and t.max() < n
    assert np.array_equal(t, synth.window_trace(7, n, length))          # seeded
    assert not np.array_equal(t, synth.window_trace(8, n, length))
    # the scan part advances by one page per scan access
    d = np.diff(t.astype(np.int64)) % n
    assert (d == 1).mean() > 0.15
    # the hot part concentrates on a few pages (Zipf 1.1)
    counts = np.bincount(t.astype(np.int64), minlength=n)
    assert np.sort(counts)[-10:].sum() > 0.15 * length
