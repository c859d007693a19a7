"""The served form's admission policy, tested on the CPU: the same header the
server uses (csrc/ms_admission.h, no CUDA) driven by a random simulator that
checks ring bounds, slot and page exclusivity, per-page arrival order and
progress on every step."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2004_09252_b300", "csrc")
SRC = os.path.join(ROOT, "tests", "admission_sim.cpp")


@pytest.fixture(scope="module")
def sim(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("adm") / "admission_sim")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", CSRC, SRC, "-o", exe])
    return exe


CASES = [
    # seed, slots, max_wave, one_per_launch, n_pages, n_req, max_req_pages, depth, inplace_max
    (1, 64, 32, 0, 200, 3000, 8, 2, 0),       # small ring, frequent wrap, many conflicts
    (2, 64, 32, 0, 40, 3000, 8, 4, 0),        # tiny page space: conflicts everywhere
    (3, 100, 50, 0, 1000, 5000, 50, 3, 0),    # requests as large as the wave
    (4, 128, 64, 1, 300, 3000, 16, 2, 0),     # one request per wave
    (5, 4096, 2048, 0, 100000, 20000, 64, 2, 0),
    (6, 37, 37, 0, 50, 2000, 37, 8, 0),       # odd ring size, requests filling the ring
    (7, 64, 32, 0, 200, 3000, 4, 4, 32),      # in-place waves mixed in, completing in any order
    (8, 64, 32, 0, 40, 3000, 3, 4, 24),       # ... with conflicts everywhere
    (9, 4096, 2048, 0, 100000, 20000, 64, 2, 64),
    (10, 256, 128, 0, 2000, 5000, 8, 3, 48),
]


@pytest.mark.parametrize("case", CASES)
def test_admission_invariants(sim, case):
    r = subprocess.run([sim] + [str(v) for v in case], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr
