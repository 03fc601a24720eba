"""The walk's two bottom stages on the GPU: the 5-D test (one det4 per quadruple after the Bareiss
level k-4) and the 4-D test (a det3 per triple after level k-3), each in its own kernel, give the
same exact volume as the oracle on the benchmark systems, on master spaces of Table mspace-deg and
on random point sets whose filters often take the exact routes; the per-system choice, the node
split of the 5-D stage, the batch grouping by stage and the server's choice at admission change
nothing in the results."""

import json
import os
import random

import numpy as np
import pytest

import paper_1501_02237_gb300 as bd
from oracle.lifts import lifts as oracle_lifts
from oracle.volume import nvol_placing
from workloads import batch_systems, config_system, master_space_system

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_volumes.json")))
TABLE = json.load(open(os.path.join(ROOT, "tests", "golden", "master_space_table.json")))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    yield


@pytest.mark.parametrize("name", ["small_n10_k4", "single_n24_k8", "heavy_quiver_n32_k10"])
def test_both_stages_give_the_oracle_volume(name):
    P = bd.reduce(config_system(name).A)["points"]
    want = GOLD["configs"][name]["nvol"]
    for stage in (4, 5, 0):
        p = bd.Plan(P, bottom_stage=stage)
        try:
            info = p.info()
            if stage in (4, 5):
                assert info["bottom_stage"] == stage
            assert p.volume(seed=3)["nvol"] == want, (name, stage)
        finally:
            p.close()


def test_stage_rule_on_the_benchmark_systems():
    # the headline system is mostly singular (82 % of its subsets): the 5-D stage; the n=24, k=8
    # system is mostly full-dimensional: the 4-D stage and its finer work list
    q = bd.Plan(bd.reduce(config_system("heavy_quiver_n32_k10").A)["points"])
    n = bd.Plan(bd.reduce(config_system("single_n24_k8").A)["points"])
    try:
        assert q.info()["bottom_stage"] == 5
        assert n.info()["bottom_stage"] == 4
    finally:
        q.close()
        n.close()


@pytest.mark.parametrize("mk", ["2,4", "3,3", "1,7"])
def test_both_stages_on_master_spaces(mk):
    m, k = map(int, mk.split(","))
    s = master_space_system(m, k)
    P = bd.reduce(s.A)["points"]
    for stage in (4, 5):
        p = bd.Plan(P, bottom_stage=stage)
        try:
            assert p.volume(seed=1)["nvol"] == TABLE["degree"][mk], (mk, stage)
        finally:
            p.close()


@pytest.mark.parametrize("seed", range(10))
def test_both_stages_random_sets_and_node_splits(seed):
    # k = 4..8, coordinates up to 40 (minors far from small integers: the filters' bounds decide,
    # or the exact routes do); item_subsets = 1 splits every 5-D node above 16 subsets by the
    # first point of its quadruples
    rng = random.Random(77000 + seed)
    k = 4 + seed % 5
    n = rng.randint(k + 4, 18 if k <= 6 else 15)
    span = [3, 12, 40][seed % 3]
    pts = [tuple(rng.randint(-span, span) for _ in range(k)) for _ in range(n)]
    want = nvol_placing(pts)
    lf = oracle_lifts(n, seed)
    for stage in (4, 5):
        for items in (0, 1):
            p = bd.Plan(np.array(pts), bottom_stage=stage, item_subsets=items)
            try:
                r = p.volume(seed=seed)
            finally:
                p.close()
            assert r["nvol"] == want, (k, n, span, stage, items)
    # explicit lifts through the public call, whichever stage the rule picks
    r = bd.volume_lifted(np.array(pts), np.array(lf))
    assert r["status"] in (0, 3)
    if r["status"] == 0:
        assert r["nvol"] == want


def test_batch_stage_groups_agree():
    systems = batch_systems(64, first_seed=5000)
    b = bd.Batch()
    for s in systems:
        b.add(s.A, seed=4)
    b.prepare()
    got = {}
    for stage in (0, 4, 5):
        b.run(mode=0, bottom_stage=stage)
        got[stage] = [(r["degree"], r["nvol"]) for r in b.results()]
    b.close()
    assert got[0] == got[4] == got[5]
    for i in (0, 17, 63):
        assert got[0][i][0] == bd.degree(systems[i].A, seed=4)["degree"]


@pytest.mark.parametrize("stage", [4, 5])
def test_server_with_a_fixed_stage(stage):
    systems = batch_systems(24, first_seed=6000, n_range=(12, 24), k_range=(4, 8))
    srv = bd.Server(bottom_stage=stage)
    got = {}
    try:
        tickets = {srv.submit(s.A, seed=2): s for s in systems}
        while len(got) < len(tickets):
            r = srv.poll(wait_ms=5000)
            assert r is not None, "server stalled"
            got[r[0]] = r[1]
    finally:
        srv.stop()
    for t, s in tickets.items():
        assert got[t]["degree"] == bd.degree(s.A, seed=2)["degree"]
