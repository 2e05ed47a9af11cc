"""The N > 1 path of bench.py: independent replicas, timing combined over ranks.

Runs as two `gloo` ranks on the CPU (world size 2): the barrier, the maximum of
the ranks' times and the whole-job rate; and the reference arm, which only
rank 0 runs under torchrun.
"""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    rep = bench.Replicas("gloo")
    rep.barrier()
    slowest = rep.max_over_ranks(1.0 + rank)          # rank r "took" 1 + r seconds
    rate = bench.replica_throughput(rep.world, 8 * 20, slowest)
    rep.barrier()
    rep.close()
    out.put((rank, rep.world, slowest, rate))


def test_two_gloo_ranks_combine_max_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, world, slowest, rate in res:
        assert world == 2
        assert slowest == 2.0                          # max over ranks, seen by both
        assert rate == pytest.approx(2 * 160 / 2.0)    # all ranks' units / slowest time


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    env_backup = {k: os.environ.pop(k, None) for k in ("WORLD_SIZE", "RANK")}
    try:
        rep = bench.Replicas("gloo")
        assert rep.world == 1 and rep.dist is None
        assert rep.max_over_ranks(3.5) == 3.5
        rep.barrier()
    finally:
        for k, v in env_backup.items():
            if v is not None:
                os.environ[k] = v


def test_reference_arm_runs_on_rank_0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
