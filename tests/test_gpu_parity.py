"""GPU parity: the CUDA path (through the C ABI) against the oracle, bit-exact.

Small cases are compared whole (volume, cell and singular counts); the benchmark-size systems
against oracle golden values and, subset by subset, on sampled (k+1)-subsets classified by the
oracle's rational lower-facet test."""

import json
import math
import os
import random

import numpy as np
import pytest

import paper_1501_02237_gb300 as bd
from oracle.degree import degree as oracle_degree
from oracle.lifts import lifts as oracle_lifts
from oracle.lower_facet import ACCEPTED, REJECTED, SINGULAR, TIE, lower_facet_status, nvol_lifting_bruteforce
from oracle.volume import nvol_placing
from workloads import batch_systems, config_system, master_space_system, random_points

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_volumes.json")))
TABLE = json.load(open(os.path.join(ROOT, "tests", "golden", "master_space_table.json")))
STATUS = {SINGULAR: 0, REJECTED: 1, ACCEPTED: 2, TIE: 3}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    yield


@pytest.mark.parametrize("seed", range(40))
def test_volume_random_sets(seed):
    # k up to 8, up to 40 points: more than one warp slot per lane past 32 points, many work
    # items and a ragged last lane group
    rng = random.Random(seed)
    k = rng.randint(1, 8)
    npts = rng.randint(k + 1, 40 if k <= 4 else 22)
    pts = random_points(npts, k, seed, -2 - seed % 3, 2 + seed % 2)
    r = bd.volume(pts, seed=seed)
    assert r["nvol"] == nvol_placing([tuple(p) for p in pts.tolist()])
    assert r["subsets"] == math.comb(npts, k + 1)


@pytest.mark.parametrize("seed", range(20))
def test_counts_match_bruteforce_lifting(seed):
    rng = random.Random(500 + seed)
    k = rng.randint(1, 3)
    npts = rng.randint(k + 1, 9)
    pts = [tuple(rng.randint(-2, 2) for _ in range(k)) for _ in range(npts)]
    lf = oracle_lifts(npts, seed)
    total, acc, sing, ties = nvol_lifting_bruteforce(pts, lf)
    r = bd.volume_lifted(np.array(pts), np.array(lf))
    assert (r["nvol"], r["cells"], r["singular"], r["ties"]) == (total, acc, sing, ties)


@pytest.mark.parametrize("name", ["small_n10_k4", "single_n24_k8", "heavy_quiver_n32_k10"])
def test_degree_benchmark_systems(name):
    s = config_system(name)
    r = bd.degree(s.A, seed=0)
    g = GOLD["configs"][name]
    assert (r["degree"], r["nvol"], r["torsion"], r["rank"], r["dim"]) == \
        (g["degree"], g["nvol"], g["torsion"], g["rank"], g["dim"])
    assert r["subsets"] == math.comb(s.n + 1, g["dim"] + 1)


@pytest.mark.parametrize("name", ["single_n24_k8", "heavy_quiver_n32_k10"])
def test_lift_independence_full_size(name):
    s = config_system(name)
    P = bd.reduce(s.A)["points"]
    vols = {bd.volume(P, seed=sd)["nvol"] for sd in (1, 2, 77)}
    assert vols == {GOLD["configs"][name]["nvol"]}


@pytest.mark.parametrize("name", ["single_n24_k8", "heavy_quiver_n32_k10"])
def test_classify_sampled_subsets_full_size(name):
    s = config_system(name)
    P = bd.reduce(s.A)["points"]
    N, k = P.shape
    lf = np.array(oracle_lifts(N, 5))
    rng = random.Random(42)
    subs = [sorted(rng.sample(range(N), k + 1)) for _ in range(400)]
    st, ad = bd.classify(P, lf, subs)
    pts = P.tolist()
    for sub, g_st, g_ad in zip(subs, st, ad):
        o_st, o_ad = lower_facet_status(pts, lf.tolist(), sub)
        assert g_st == STATUS[o_st], sub
        assert g_ad == o_ad, sub


def test_classify_agrees_with_enumeration_counts():
    s = config_system("small_n10_k4")
    P = bd.reduce(s.A)["points"]
    N, k = P.shape
    lf = np.array(oracle_lifts(N, 0))
    subs = list(__import__("itertools").combinations(range(N), k + 1))
    st, ad = bd.classify(P, lf, subs)
    r = bd.volume_lifted(P, lf)
    assert int((st == 2).sum()) == r["cells"] and int((st == 0).sum()) == r["singular"]
    assert int(ad[st == 2].sum()) == r["nvol"]


@pytest.mark.parametrize("mk", ["1,4", "2,2", "2,3", "3,2", "1,8", "2,4", "3,3", "2,5"])
def test_master_space_degrees(mk):
    m, k = map(int, mk.split(","))
    s = master_space_system(m, k)
    r = bd.degree(s.A, s.coef.reshape(-1, 4), seed=11)
    assert r["degree"] == TABLE["degree"][mk]
    assert r["dim"] == TABLE["dimension"][mk]


def test_batch_systems_against_oracle_golden():
    systems = batch_systems(24)
    for s, g in zip(systems, GOLD["batch_first_256"]):
        r = bd.degree(s.A, seed=3)
        assert (r["degree"], r["nvol"], r["dim"]) == (g["degree"], g["nvol"], g["dim"]), s.name


def test_int128_path_forced_equals_int64():
    s = config_system("single_n24_k8")
    P = bd.reduce(s.A)["points"]
    a = bd.Plan(P).volume(seed=0)
    b = bd.Plan(P, force_int128=True)
    assert b.info()["int128"]
    assert b.volume(seed=0)["nvol"] == a["nvol"] == GOLD["configs"]["single_n24_k8"]["nvol"]


@pytest.mark.parametrize("seed", range(6))
def test_int64_path_medium_coordinates(seed):
    # |x| ~ 2^10 in k = 3: coordinate minors beyond 32 bits, lifted minors within 64
    rng = random.Random(70 + seed)
    pts = [tuple(rng.randint(-1024, 1024) for _ in range(3)) for _ in range(12)]
    p = bd.Plan(np.array(pts))
    assert p.info()["path"] == "int64"
    assert p.volume(seed=seed)["nvol"] == nvol_placing(pts)


@pytest.mark.parametrize("seed", range(6))
def test_int128_path_large_coordinates(seed):
    # coordinates near 2^22 push the Hadamard bound past 2^63: the 128-bit path must be taken
    rng = random.Random(seed)
    k = 4
    pts = [tuple(rng.randint(-(1 << 22), 1 << 22) for _ in range(k)) for _ in range(9)]
    r = bd.volume(np.array(pts), seed=seed)
    assert r["flags"] & bd.BD_FLAG_INT128
    assert r["nvol"] == nvol_placing(pts)


def test_launch_shapes_and_item_sizes_agree():
    s = config_system("single_n24_k8")
    P = bd.reduce(s.A)["points"]
    want = GOLD["configs"]["single_n24_k8"]["nvol"]
    for w, items in [(1, 64), (2, 1 << 20), (4, 0), (8, 512)]:
        p = bd.Plan(P, warps_per_block=w, item_subsets=items)
        assert p.volume(seed=4)["nvol"] == want, (w, items)


def test_ties_are_reported_not_rounded():
    S = np.array([(0, 0), (0, 1), (1, 1), (1, 0)])
    r = bd.volume_lifted(S, np.array([0, 1, 2, 1]))
    assert r["status"] == 3 and r["ties"] == 4
    # with a seeded lifting the call re-lifts and succeeds
    assert bd.volume(S, seed=0)["nvol"] == 2


def test_edge_cases():
    # fewer than k+1 points, a flat set, segments (k = 1), duplicates, the maximum point count
    assert bd.volume(np.array([[0, 0], [1, 0]]))["flags"] & bd.BD_FLAG_DEGENERATE
    flat = np.array([(0, 0, 0), (1, 0, 0), (0, 1, 0), (2, 3, 0), (1, 1, 0)])
    r = bd.volume(flat)
    assert r["nvol"] == 0 and r["flags"] & bd.BD_FLAG_DEGENERATE
    assert bd.volume(np.array([[3], [-4], [1], [0]]))["nvol"] == 7
    dup = np.array([(0, 0), (1, 0), (0, 1), (1, 0), (0, 1), (1, 1)])
    assert bd.volume(dup)["nvol"] == 2
    pts = random_points(64, 2, 9, -6, 6)
    assert bd.volume(pts)["nvol"] == nvol_placing([tuple(p) for p in pts.tolist()])
    cube = np.array(list(__import__("itertools").product((0, 1), repeat=6)))
    assert bd.volume(cube)["nvol"] == math.factorial(6)


def test_argument_errors():
    with pytest.raises(bd.BinodegError):
        bd.volume(np.zeros((5, 15), dtype=np.int64))
    with pytest.raises(bd.BinodegError):
        bd.volume(np.zeros((65, 2), dtype=np.int64))
    with pytest.raises(bd.BinodegError) as e:
        bd.volume(np.array([[1 << 39, 0, 0, 0, 0, 0, 0, 0]] + [[0] * 8] * 4 + [[(1 << 39) - 3] * 8] * 5))
    assert e.value.code in (1, 2)


def test_inconsistent_and_zero_dimensional():
    r = bd.degree(np.array([[1, 1]]), [[1, 1, -2, 1], [1, 1, -3, 1]])
    assert r["degree"] == 0 and not r["consistent"]
    r = bd.degree(np.array([[2, 0], [0, 3]]))
    assert (r["degree"], r["dim"]) == (6, 0)
    assert bd.degree(np.array([[-2], [1]]))["degree"] == 2
    assert bd.degree(np.array([[2], [2]]))["degree"] == oracle_degree([[2], [2]]).degree == 4


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["small_n10_k4", "single_n24_k8"])
def test_shards_cover_every_subset_once(name):
    # the shards of one launch (run one after another on this GPU: they never wait on each
    # other) add up to the whole enumeration, for several shard counts
    P = bd.reduce(config_system(name).A)["points"]
    plan = bd.Plan(P)
    full = plan.volume(seed=0)
    for world in (2, 3, 8):
        parts = []
        for r in range(world):
            plan.launch(seed=0, attempt=full["relifts"], shard=r, shards=world)
            parts.append(plan.read())
        for key in ("nvol", "cells", "singular", "ties"):
            assert sum(p[key] for p in parts) == full[key], (world, key)
        assert all(p["nvol"] > 0 for p in parts) or name == "small_n10_k4"
    plan.close()


@pytest.mark.gpu
def test_shard_arguments_are_checked():
    plan = bd.Plan(bd.reduce(config_system("small_n10_k4").A)["points"])
    with pytest.raises(bd.BinodegError):
        plan.launch(seed=0, shard=2, shards=2)
    plan.close()
