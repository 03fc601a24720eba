"""Batches of systems: host preparation on CPU, and on the GPU every mode of bd_batch_run against
the oracle's golden values and the single-system path (exact equality)."""

import json
import os

import numpy as np
import pytest

import paper_1501_02237_gb300 as bd
from oracle.volume import nvol_placing
from workloads import batch_systems, config_system, master_space_system, random_points

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_volumes.json")))
TABLE = json.load(open(os.path.join(ROOT, "tests", "golden", "master_space_table.json")))


def make_batch(n_random=40):
    b = bd.Batch()
    systems = batch_systems(n_random)
    for s in systems:
        b.add(s.A, seed=7)
    want = [(g["degree"], g["nvol"]) for g in GOLD["batch_first_256"][:n_random]]
    for mk in ["2,2", "2,3", "1,5"]:
        m, k = map(int, mk.split(","))
        s = master_space_system(m, k)
        b.add(s.A, s.coef.reshape(-1, 4), seed=1)
        want.append((TABLE["degree"][mk], TABLE["degree"][mk]))
    s = config_system("single_n24_k8")
    b.add(s.A, seed=2)
    g = GOLD["configs"]["single_n24_k8"]
    want.append((g["degree"], g["nvol"]))
    # a point set on the int64 path and one on the int128 path
    rng = np.random.default_rng(5)
    p64 = rng.integers(-1024, 1025, size=(12, 3))
    p128 = rng.integers(-(1 << 22), (1 << 22) + 1, size=(9, 4))
    for P in (p64, p128):
        b.add_points(P, seed=3)
        v = nvol_placing([tuple(x) for x in P.tolist()])
        want.append((v, v))
    return b, want


def test_prepare_and_features_on_host():
    b, _ = make_batch(12)
    b.prepare(threads=4)
    f = b.features()
    assert f.shape == (b.count, bd.BD_FEATURES)
    assert np.isfinite(f).all()
    # N, k of the first system agree with the host reduction
    s = batch_systems(1)[0]
    red = bd.reduce(s.A)
    assert (f[0, 0], f[0, 1]) == (red["points"].shape[0], red["dim"])
    assert set(np.unique(f[:, 4])) <= {0.0, 1.0, 2.0}


@pytest.mark.gpu
def test_batch_modes_agree_with_oracle():
    pytest.importorskip("torch").cuda.init()
    b, want = make_batch()
    b.prepare()
    for kw in [dict(mode=0), dict(mode=0, use_graph=True), dict(mode=0, use_graph=True), dict(mode=1),
               dict(mode=0, autotune=True), dict(mode=0, warps_per_block=2, item_factor=16),
               dict(mode=0, cost=np.random.default_rng(0).uniform(0.1, 10.0, size=b.count))]:
        st = b.run(**kw)
        got = [(r["degree"], r["nvol"]) for r in b.results()]
        assert got == want, kw
        assert st["subsets"] > 0


@pytest.mark.gpu
def test_batch_equals_single_system_calls():
    pytest.importorskip("torch").cuda.init()
    systems = batch_systems(30)[10:30]
    b = bd.Batch()
    for s in systems:
        b.add(s.A, seed=11)
    b.prepare()
    b.run(mode=0)
    for i, s in enumerate(systems):
        r = b.result(i)
        one = bd.degree(s.A, seed=11)
        assert (r["degree"], r["nvol"], r["cells"], r["torsion"], r["dim"]) == \
            (one["degree"], one["nvol"], one["cells"], one["torsion"], one["dim"])
        assert r["cycles"] > 0
