"""Host logic of the benchmark's multi-GPU path, run as two gloo ranks on the CPU:
disjoint receiver shards of the same shape on every rank (weak scaling, no data-path
collective), whole-job time as the slowest rank's, whole-job units as the sum; and
the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ids = bench.rank_receiver_ids(rank, 4)
        all_ids = [None] * world
        dist.all_gather_object(all_ids, ids)
        t = bench.job_time(10.0 + rank, world, torch.device("cpu"))
        u = bench.job_units(1000 * (rank + 1), world, torch.device("cpu"))
        out.put((rank, all_ids, t, u))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, all_ids, t, u in res:
        flat = [i for ids in all_ids for i in ids]
        assert sorted(flat) == list(range(8))                  # disjoint, complete
        assert all(len(ids) == 4 for ids in all_ids)           # same shape on every rank
        assert t == 11.0                                       # slowest rank
        assert u == 3000                                       # sum over ranks


def test_weak_scaling_shards_have_identical_shape():
    sys.path.insert(0, ROOT)
    import bench
    a = bench.workload(0, 2, 3)
    b = bench.workload(1, 2, 3)
    assert [r.meta for r in a] != [r.meta for r in b]
    for x, y in zip(a, b):
        assert (x.fs, x.block_samples, len(x.channels), x.n_taps, x.integ_blocks) == \
               (y.fs, y.block_samples, len(y.channels), y.n_taps, y.integ_blocks)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
