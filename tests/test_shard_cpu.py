"""Multi-GPU sharding of one volume, run as CPU ranks: two gloo processes each enumerate their
shard of the work list with the host emulation and exchange the partial sums by the same
all-reduce the GPU ranks use.  The combined volume must equal the oracle's; a tie in any
shard must reach every rank."""

import os
import random
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle.lifts import lifts as oracle_lifts
from oracle.volume import nvol_placing


def _port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, cases, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_1501_02237_gb300 as bd
    from paper_1501_02237_gb300 import shard
    out = []
    for pts, lf, items in cases:
        part = bd.host_volume_lifted(np.array(pts), np.array(lf), item_subsets=items, shard=rank, shards=world)
        out.append((part, shard.combine(part)))
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def run_ranks(world, cases):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, cases, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def _cases():
    rng = random.Random(77)
    cases = []
    for i in range(6):
        k = rng.choice([2, 3, 4, 5])
        n = rng.randint(k + 3, 11)
        pts = [tuple(rng.randint(-2, 2) for _ in range(k)) for _ in range(n)]
        cases.append((pts, oracle_lifts(n, i), 1 + 30 * (i % 2)))
    return cases


def test_two_cpu_ranks_sum_to_the_oracle_volume():
    cases = _cases()
    res = run_ranks(2, cases)
    for c, (pts, lf, items) in enumerate(cases):
        p0, t0 = res[0][c]
        p1, t1 = res[1][c]
        ref = nvol_placing(pts)
        assert t0["nvol"] == t1["nvol"] == ref == p0["nvol"] + p1["nvol"]
        assert t0["cells"] == p0["cells"] + p1["cells"] and t0["singular"] == p0["singular"] + p1["singular"]
        assert t0["ties"] == 0


def test_a_tie_in_one_shard_reaches_every_rank():
    rng = random.Random(3)
    pts = [tuple(rng.randint(-3, 3) for _ in range(3)) for _ in range(9)]
    res = run_ranks(2, [(pts, [0] * len(pts), 1)])
    (p0, t0), (p1, t1) = res[0][0], res[1][0]
    assert t0["ties"] == t1["ties"] == p0["ties"] + p1["ties"] > 0
