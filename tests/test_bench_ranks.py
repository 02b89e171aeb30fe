"""bench.py's multi-rank logic on CPU: two gloo ranks, each with its own
disjoint run of slices (weak scaling), the step time taken as the maximum
over ranks, and the reference arm printing from rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = bench.shard_workload("stack512", 4, rank)
    seeds = [s.seed for s in wl.slices]
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    slowest = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    single = bench.shard_workload("slice2048", None, rank)
    q.put((rank, gathered, slowest, [s.seed for s in single.slices]))
    dist.destroy_process_group()


def test_two_ranks_shard_and_take_the_max():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, slowest, single in res:
        a, b = gathered
        assert len(a) == len(b) == 4 and not set(a) & set(b)  # disjoint runs of the stack
        assert a == [1000 + k for k in range(4)] and b == [1004 + k for k in range(4)]
        assert slowest == 15.0
        assert single == [0]  # single-slice workloads are replicated


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
