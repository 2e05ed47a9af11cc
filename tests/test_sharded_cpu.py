"""Host side of the term-sharded apply, no GPU: the partition of the term
list over parts, and the integer reduction of the parts' accumulators over two
gloo ranks (the collective a multi-GPU apply uses between its parts)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp

import paper_2111_13655_gb300 as sg
from paper_2111_13655_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("nparts", [1, 2, 3, 8])
def test_parts_cover_every_term_once_and_balance_the_cost(nparts):
    p = synth.workload_C3(L=8)
    with sg.sg_plan(p, "mixed") as ctx:
        sizes = [sg.sg_part_size(ctx, r, nparts) for r in range(nparts)]
    assert sum(n for n, _ in sizes) == ctx.n_terms
    costs = np.array([c for _, c in sizes], float)
    assert costs.max() / costs.mean() < 1.01      # round robin over terms sorted by cost


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


M64 = 1 << 64


def _accumulators(rank):
    """Rank-specific int64 accumulators with values near the int64 limits, so
    that the sum over ranks wraps modulo 2^64 in between."""
    rng = np.random.default_rng(100 + rank)
    a = rng.integers(-(1 << 62), 1 << 62, size=4096, dtype=np.int64)
    a[:16] = (1 << 63) - 1 - rank            # large positive: the sum overflows
    a[16:32] = -(1 << 63) + rank             # large negative: the sum underflows
    return a


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2111_13655_gb300 import sharded
    dist.init_process_group("gloo")
    acc = torch.from_numpy(_accumulators(rank))
    sharded.reduce_accumulators(acc)
    dist.destroy_process_group()
    out.put((rank, acc.numpy().tobytes()))


def test_two_gloo_ranks_sum_accumulators_exactly_modulo_2_64():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts = [_accumulators(r) for r in range(2)]
    expect = [((int(a) + int(b)) % M64) for a, b in zip(*parts)]
    expect = np.array([v - M64 if v >= 1 << 63 else v for v in expect], dtype=np.int64)
    for rank in range(2):
        got = np.frombuffer(res[rank], dtype=np.int64)
        assert np.array_equal(got, expect)
