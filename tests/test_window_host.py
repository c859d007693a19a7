"""The sliding-window clients and their background evictors, tested on the
CPU: the same header the GPU backends use (csrc/ms_window_client.h, no CUDA)
driven by a fake GPU whose executors apply each request after a random
delay.  Checks that no request finds its page in the wrong state, that the
final states match the final windows, and the counters; a fake that breaks
the per-page order must be caught."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2004_09252_b300", "csrc")
INCLUDE = os.path.join(ROOT, "include")
SRC = os.path.join(ROOT, "tests", "window_sim.cpp")


@pytest.fixture(scope="module")
def sim(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("win") / "window_sim")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-pthread", "-I", CSRC, "-I", INCLUDE, SRC, "-o", exe])
    return exe


CASES = [
    # seed, clients, client_pages, trace_len, window, evict_batch, background_free, executors
    (1, 1, 64, 4000, 4, 1, 0, 1),      # the paper's policy, stream order
    (2, 3, 64, 3000, 8, 1, 0, 4),      # several clients, in-flight rule
    (3, 1, 64, 4000, 4, 1, 1, 1),      # background eviction, one free slot
    (4, 3, 64, 3000, 8, 1, 3, 4),
    (5, 2, 128, 3000, 16, 4, 6, 4),    # background requests of up to 4 pages
    (6, 4, 48, 2500, 32, 8, 31, 2),    # the evictor keeps one page at rest
    (7, 2, 40, 3000, 8, 9, 2, 1),      # overflow batches larger than the window
]
SYNC_CASES = [  # the client waits for its own overflow evictions (the paper's server), with and without an evictor
    (8, 2, 64, 3000, 8, 1, 0, 4),
    (9, 3, 64, 3000, 8, 4, 2, 4),
]


@pytest.mark.parametrize("case", CASES)
def test_window_invariants(sim, case):
    r = subprocess.run([sim] + [str(v) for v in case] + ["0"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr


@pytest.mark.parametrize("case", SYNC_CASES)
def test_window_invariants_with_synchronous_eviction(sim, case):
    r = subprocess.run([sim] + [str(v) for v in case] + ["0", "1"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr


def test_a_reordering_backend_is_caught(sim):
    """Executors that ignore the per-page order must break an invariant."""
    caught = 0
    for seed in range(1, 6):
        r = subprocess.run([sim, str(seed), "3", "32", "3000", "8", "1", "3", "4", "1"], capture_output=True,
                           text=True, timeout=120)
        caught += r.stdout.startswith("FAIL")
    assert caught >= 4
