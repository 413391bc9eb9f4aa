"""The N > 1 path of the benchmark on CPU: two gloo ranks, each timing its own replica;
barrier, max over ranks and sum of units give the whole-job throughput."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    from paper_2103_07925_gb300.replicas import from_env
    rep, local = from_env("gloo")
    try:
        assert (rep.rank, rep.world, local) == (rank, world, rank)
        rep.barrier()
        # rank r processed 100 (r + 1) units in 2 (r + 1) seconds
        units, secs = 100.0 * (rank + 1), 2.0 * (rank + 1)
        q.put((rank, rep.max(secs), rep.sum(units), rep.throughput(units, secs)))
        rep.barrier()
    finally:
        rep.dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, tmax, usum, thr in res:
        assert tmax == 4.0 and usum == 300.0 and thr == 75.0


def test_single_process_needs_no_group():
    from paper_2103_07925_gb300.replicas import Replicas
    rep = Replicas(None)
    rep.barrier()
    assert (rep.rank, rep.world) == (0, 1)
    assert rep.throughput(120.0, 3.0) == 40.0


def test_reference_arm_on_a_non_zero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
