"""The multi-GPU path of bench.py on CPU: world-size-2 gloo ranks.

bench.py runs one replica of the workload per rank (the solve has no
exchange step) and reports the slowest rank's time; these tests check that
aggregation and the reference arm's rank-0-only rule with a real process
group, without a GPU."""

import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r measured (r + 1) ms per solve and a wall time of 10 - r s
        ms_max, wall_max = bench.max_over_ranks([rank + 1.0, 10.0 - rank], dist, "cpu")
        out[rank] = (ms_max, wall_max, bench.job_throughput(world, ms_max))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # every rank sees the slowest rank's time; the job's throughput counts both replicas
    for r in range(world):
        assert res[r] == (2.0, 10.0, 1000.0)


def test_max_over_ranks_single_process():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], None, "cpu") == [3.0, 4.0]
    assert bench.job_throughput(1, 4.0) == 250.0


@pytest.mark.parametrize("rank", [1])
def test_reference_arm_prints_on_rank0_only(rank):
    """Under torchrun only rank 0 times the oracle; other ranks exit 0 silently."""
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_bench_help_lists_contract_flags():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0
    for flag in ("--gpus", "--steps", "--warmup", "--impl"):
        assert flag in r.stdout
