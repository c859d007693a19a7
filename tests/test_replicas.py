"""Multi-GPU is replicas only (pages shard with no exchange step): the bench's
whole-job aggregation over ranks, checked with world_size 2 over gloo on CPU."""
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took 10 * (r + 1) ms for 1e9 * (r + 1) bytes
    ms, gbs = bench.aggregate_replicas(10.0 * (rank + 1), 1e9 * (rank + 1), world)
    out[rank] = (ms, gbs)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_over_gloo():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        ms, gbs = res[r]
        assert ms == pytest.approx(20.0)                 # max over ranks
        assert gbs == pytest.approx(3e9 / 0.020 / 1e9)   # all ranks' bytes / max time


def test_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    ms, gbs = bench.aggregate_replicas(5.0, 1e9, 1)
    assert ms == 5.0 and gbs == pytest.approx(200.0)


def test_reference_arm_non_zero_rank_exits_silently():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
