"""The N > 1 host logic of bench.py on CPU: two gloo ranks (max over ranks, disjoint problem seeds, the
whole-job rate) and the reference arm's non-zero ranks, which exit without work."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.5 + rank)
    seeds = bench.rank_seed_offsets(rank, 3)
    dist.barrier()
    q.put((rank, t, seeds))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_step_time_and_shard_the_problems():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [t for _, t, _ in out] == [2.5, 2.5]  # every rank gets the slowest rank's time
    s0, s1 = out[0][2], out[1][2]
    assert s0 == [0, 1, 2] and s1 == [3, 4, 5]  # disjoint problems per rank (weak scaling)
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(2, 3, 0.5) == 12.0
    assert bench.max_over_ranks(3.25) == 3.25  # no process group: the value itself


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
