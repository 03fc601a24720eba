"""Serving with continuous batching: every result equals the single-system result, whatever
arrives while others run, under both admission orders and a tight device budget."""

import time

import numpy as np
import pytest

import paper_1501_02237_gb300 as bd
from workloads import batch_systems, master_space_system, poisson_arrivals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    yield


def served_systems(count, first_seed):
    return batch_systems(count, first_seed=first_seed, n_range=(12, 22), k_range=(4, 8))


def run_stream(server, systems, rate, seed):
    arrivals = poisson_arrivals(rate, len(systems), seed)
    t0 = time.perf_counter()
    tickets = {}
    results = {}
    for s, ta in zip(systems, arrivals):
        while time.perf_counter() - t0 < ta:
            got = server.poll()
            if got:
                results[got[0]] = got
            else:
                time.sleep(0.0002)
        tickets[server.submit(s.A, seed=3)] = s  # every system is served (side route included)
    while len(results) < len(tickets):
        got = server.poll(wait_ms=2000)
        assert got is not None, "server stalled"
        results[got[0]] = got
    return tickets, results


@pytest.mark.parametrize("order", [0, 1])
def test_each_result_is_the_same_alone_and_in_the_mix(order):
    systems = served_systems(48, 30000)
    srv = bd.Server(order=order)
    try:
        tickets, results = run_stream(srv, systems, rate=400.0, seed=order)
        st = srv.stats()
    finally:
        srv.stop()
    assert len(results) == 48
    # continuous batching: systems were resident on the device together
    assert st["peak_resident"] >= 2, st
    for t, s in tickets.items():
        _, r, lat = results[t]
        alone = bd.degree(s.A, seed=3)
        assert (r["degree"], r["nvol"], r["torsion"], r["dim"]) == \
            (alone["degree"], alone["nvol"], alone["torsion"], alone["dim"]), s.name
        assert lat > 0


def test_tight_budget_queues_but_stays_exact():
    systems = served_systems(24, 31000)
    srv = bd.Server(slots=4, memory_budget=4 * 6200 + 16 * 4096, max_inflight_items=2000)
    try:
        tickets, results = run_stream(srv, systems, rate=2000.0, seed=7)
        st = srv.stats()
    finally:
        srv.stop()
    assert st["slots"] == 4 and st["ring_items"] <= 4096
    for t, s in tickets.items():
        assert results[t][1]["degree"] == bd.degree(s.A, seed=1)["degree"]


def test_master_space_and_dimension_zero_through_the_server():
    srv = bd.Server()
    try:
        s = master_space_system(2, 3)
        t1 = srv.submit(s.A, s.coef.reshape(-1, 4))
        t2 = srv.submit(np.array([[2, 0], [0, 3]]))  # isolated points: no GPU work
        got = {}
        while len(got) < 2:
            r = srv.poll(wait_ms=2000)
            assert r is not None
            got[r[0]] = r[1]
    finally:
        srv.stop()
    assert got[t1]["degree"] == 92 and got[t2]["degree"] == 6


def wide_system(seed):
    """A binomial system whose kernel points need 128-bit minors: 10 variables, 4 binomials
    with exponent differences up to 1000, so the kernel lattice (dimension 6) has long vectors."""
    rng = np.random.default_rng(seed)
    return rng.integers(-1000, 1001, size=(10, 4)).astype(np.int64)


def test_wide_and_high_dimensional_systems_are_served_exactly():
    """128-bit systems, dimension 12 (above the persistent kernel's 10) and a master
    space go through the side route, interleaved with ordinary systems; every result
    equals bd_degree's, and the master space equals its table entry."""
    wides = [wide_system(s) for s in range(3)]
    for A in wides:
        P = bd.reduce(A)["points"]
        assert bd.volume(P)["flags"] & bd.BD_FLAG_INT128, "the case must need the 128-bit path"
    high = batch_systems(2, first_seed=41000, n_range=(20, 20), k_range=(12, 12))
    ms = master_space_system(3, 5)  # 45 variables, d = 17: the pivoting walk (Table mspace-deg: 437,038)
    ordinary = served_systems(12, 42000)
    mix = [("wide", A) for A in wides] + [("high", s.A) for s in high] + [("ms", ms.A)]
    mix += [("ord", s.A) for s in ordinary]
    order = np.random.default_rng(5).permutation(len(mix))
    srv = bd.Server()
    got, tickets = {}, {}
    try:
        for i in order:
            kind, A = mix[i]
            tickets[srv.submit(A, seed=2)] = (kind, A)
        while len(got) < len(tickets):
            r = srv.poll(wait_ms=5000)
            assert r is not None, "server stalled"
            got[r[0]] = r[1]
        st = srv.stats()
    finally:
        srv.stop()
    assert st["routed"] == len(wides) + len(high) + 1, st
    for t, (kind, A) in tickets.items():
        alone = bd.degree(A, seed=2)
        assert (got[t]["degree"], got[t]["nvol"], got[t]["dim"]) == (alone["degree"], alone["nvol"], alone["dim"]), kind
        if kind == "high":
            assert got[t]["dim"] == 12
        if kind == "ms":
            assert got[t]["degree"] == 437038 and got[t]["flags"] & bd.BD_FLAG_PIVOT
