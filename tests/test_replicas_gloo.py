"""Multi-process host logic of N-GPU runs (independent replicas), on CPU with
gloo at world size 2: rank discovery, per-rank tables, the max-over-ranks
time and the whole-job value; and the reference arm's rank > 0 behaviour."""
import os
import socket
import subprocess
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1901_01488_gb300 import datagen, replicas

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert replicas.env_rank() == (rank, world, rank)
        t = datagen.skewed_table(1000, seed=replicas.table_seed(rank))
        digest = int(t.col("key").data.sum())
        dist.barrier()
        ms = replicas.max_over_ranks(10.0 + 5.0 * rank, dist)
        value = replicas.job_value(1000 * 200, world, ms)
        seeds = [None] * world
        dist.all_gather_object(seeds, (replicas.table_seed(rank), digest))
        q.put((rank, ms, value, seeds))
    finally:
        dist.destroy_process_group()


def test_two_replicas_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, seeds in out:
        assert ms == 15.0                               # the slowest rank's time, on every rank
        assert value == 1000 * 200 * 2 / 0.015          # units of both ranks over that time
        assert seeds[0][0] != seeds[1][0] and seeds[0][1] != seeds[1][1]   # distinct tables


def test_single_process_needs_no_collective():
    assert replicas.max_over_ranks(7.5) == 7.5
    assert replicas.job_value(10, 1, 1000.0) == 10.0


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
