"""Failure reporting on the GPU without a GPU fault: injected device-allocation failures come
back as BD_ERR_NOMEM from every kind of call that allocates, free what was allocated, and leave
the context usable (the next call gives the exact result)."""

import json
import os

import numpy as np
import pytest

import paper_1501_02237_gb300 as bd
from paper_1501_02237_gb300._lib import BD_ERR_NOMEM
from workloads import batch_systems, config_system

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_volumes.json")))["configs"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    yield
    bd.inject_alloc_failure(-1)


@pytest.mark.parametrize("after", [0, 1, 2])
def test_plan_allocation_failures_are_nomem_and_recoverable(after):
    P = bd.reduce(config_system("single_n24_k8").A)["points"]
    bd.inject_alloc_failure(after)  # the plan's three device buffers, in turn
    with pytest.raises(bd.BinodegError) as e:
        bd.Plan(P)
    assert e.value.code == BD_ERR_NOMEM
    plan = bd.Plan(P)
    assert plan.volume(seed=1)["nvol"] == GOLDEN["single_n24_k8"]["nvol"]
    plan.close()


def test_batch_server_and_pivot_report_nomem():
    systems = batch_systems(16, first_seed=500)
    b = bd.Batch()
    for s in systems:
        b.add(s.A)
    b.prepare()
    bd.inject_alloc_failure(0)
    with pytest.raises(bd.BinodegError) as e:
        b.run(mode=0)
    assert e.value.code == BD_ERR_NOMEM
    b.run(mode=0)  # recovers
    assert [r["degree"] for r in b.results()] == [bd.degree(s.A)["degree"] for s in systems]
    b.close()
    bd.inject_alloc_failure(0)
    with pytest.raises(bd.BinodegError) as e:
        bd.Server()
    assert e.value.code == BD_ERR_NOMEM
    small = np.array([[0, 0], [1, 0], [0, 1], [1, 1], [2, 1]])
    bd.inject_alloc_failure(0)
    with pytest.raises(bd.BinodegError) as e:
        bd.volume_pivot(small)
    assert e.value.code == BD_ERR_NOMEM
    assert bd.volume_pivot(small)["nvol"] == bd.volume(small)["nvol"] == 3  # NVol of the pentagon: 2 x 3/2


def test_publication_wait_runs_out_and_the_server_recovers():
    # the third admission's publication stamps are withheld (a message the test drops): the
    # kernel's bounded wait for them runs out, its request fails with BD_ERR_TIMEOUT, every
    # other request is requeued and finishes exactly, and the server keeps serving
    from paper_1501_02237_gb300._lib import BD_ERR_TIMEOUT

    systems = batch_systems(10, first_seed=600, n_range=(12, 18), k_range=(4, 6))
    srv = bd.Server(publish_wait_ms=200, test_withhold=3)
    try:
        tickets = {srv.submit(s.A, seed=1): s for s in systems}
        got, failed = {}, {}
        while len(got) + len(failed) < len(tickets):
            try:
                r = srv.poll(wait_ms=5000)
            except bd.BinodegError as e:
                failed[e.ticket] = e.code
                continue
            assert r is not None, "server stalled"
            got[r[0]] = r[1]
        st = srv.stats()
        t2 = srv.submit(systems[0].A, seed=1)
        r2 = srv.poll(wait_ms=5000)
    finally:
        srv.stop()
    assert list(failed.values()) == [BD_ERR_TIMEOUT], failed
    assert st["faults"] == 1, st
    for t, r in got.items():
        assert r["degree"] == bd.degree(tickets[t].A, seed=1)["degree"]
    assert r2 is not None and r2[0] == t2 and r2[1]["degree"] == bd.degree(systems[0].A, seed=1)["degree"]
