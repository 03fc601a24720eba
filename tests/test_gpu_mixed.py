"""Mixed volume on the GPU (bd_mixed_volume, bd_mixed_volume_lifted) against the oracle:
the same fine mixed cells and counts under the same heights on small supports; closed forms
(Bezout, the permanent of boxes) and the unmixed case against bd_volume at mid size; the host
emulation and the 128-bit path agreeing at 759k tuples; and at 85.8 million and at the
benchmark's 13.5 billion tuples of pairs (k = 7, 8 points per set) lift independence, every
listed cell confirmed one by one by the oracle's rational test, and sampled unlisted tuples
rejected by it."""

import random
from itertools import permutations
from math import prod

import numpy as np
import pytest

import paper_1501_02237_gb300 as bd
from oracle.lifts import lifts as oracle_lifts
from oracle.mixed import cell_status, mixed_cells, mixed_volume_polarization
from workloads import mixed_config

pytestmark = pytest.mark.gpu


def random_supports(rng, k, lo=2, hi=5, span=2):
    return [[tuple(rng.randint(0, span) for _ in range(k)) for _ in range(rng.randint(lo, hi))] for _ in range(k)]


@pytest.mark.parametrize("seed", range(24))
def test_gpu_mixed_cells_match_oracle(seed):
    rng = random.Random(9100 + seed)
    k = rng.choice([1, 2, 3, 3, 4])
    S = random_supports(rng, k, hi=5 if k < 4 else 4)
    W = oracle_lifts(sum(len(A) for A in S), seed)
    cells, sing, ties = mixed_cells(S, W)
    r = bd.mixed_volume_lifted(S, W, cells=True)
    if ties:
        assert r["status"] == 3 and r["ties"] == ties
        return
    assert r["status"] == 0
    assert r["cell_list"] == [c for c, _ in cells] and r["absdet"] == [v for _, v in cells]
    assert r["mv"] == sum(v for _, v in cells) and r["singular"] == sing


@pytest.mark.parametrize("seed,big", [(0, 1 << 20), (1, 1 << 20), (2, 1 << 30), (3, 1 << 30), (4, 1 << 33)])
def test_gpu_mixed_near_coplanar_lifts(seed, big):
    # every point within a few units of one plane: the exact route decides most tests
    rng = random.Random(9400 + seed)
    k = 3
    S = random_supports(rng, k, lo=3, hi=5)
    l = [rng.randint(-3, 3) for _ in range(k)]
    W = [big * sum(x * y for x, y in zip(p, l)) + rng.randint(-2, 2) for A in S for p in A]
    cells, sing, ties = mixed_cells(S, W)
    r = bd.mixed_volume_lifted(S, W, cells=True)
    if ties:
        assert r["status"] == 3 and r["ties"] == ties
        return
    assert r["cell_list"] == [c for c, _ in cells] and r["singular"] == sing


@pytest.mark.parametrize("seed,big", [(0, 1 << 24), (1, 1 << 28)])
def test_gpu_mixed_near_coplanar_mid_size(seed, big):
    # the 3-D leaf stage (1024+ nodes above it) with heights near one plane: its exact route
    S = [A.tolist() for A in mixed_config("mixed_k5_p6")]
    rng = random.Random(9500 + seed)
    l = [rng.randint(-3, 3) for _ in range(5)]
    W = [big * sum(x * y for x, y in zip(p, l)) + rng.randint(-1000, 1000) for A in S for p in A]
    g = bd.mixed_volume_lifted(S, W, cells=True)
    h = bd.host_mixed_volume_lifted(S, W, cells=True, leaf3=0)
    assert g["status"] == h["status"]
    if g["status"] == 0:
        assert (g["mv"], g["cell_list"], g["singular"]) == (h["mv"], h["cell_list"], h["singular"])
        SL = S
        for c, v in zip(g["cell_list"], g["absdet"]):
            assert cell_status(SL, W, c) == ("accepted", v)


@pytest.mark.parametrize("seed", range(6))
def test_gpu_mixed_volume_equals_polarization(seed):
    rng = random.Random(9200 + seed)
    k = rng.choice([2, 3, 4])
    S = random_supports(rng, k, lo=3, hi=4 if k == 4 else 6)
    assert bd.mixed_volume(S, seed=seed)["mv"] == mixed_volume_polarization(S)


def test_gpu_mixed_small_workload_against_oracle():
    S = [A.tolist() for A in mixed_config("mixed_k3_p5")]
    W = oracle_lifts(sum(len(A) for A in S), 0)
    cells, sing, _ = mixed_cells(S, W)
    r = bd.mixed_volume_lifted(S, W, cells=True)
    assert r["cell_list"] == [c for c, _ in cells] and r["singular"] == sing
    assert r["mv"] == mixed_volume_polarization(S) == 18


def _simplex_points(d, k):
    out = []

    def rec(prefix, left):
        if len(prefix) == k:
            out.append(tuple(prefix))
            return
        for v in range(left + 1):
            rec(prefix + [v], left - v)
    rec([], d)
    return out


@pytest.mark.parametrize("degs", [(2, 1, 2, 2), (1, 2, 1, 1, 2), (1, 1, 2, 1, 1, 1)])
def test_gpu_bezout(degs):
    k = len(degs)
    S = [_simplex_points(d, k) for d in degs]
    r = bd.mixed_volume(S, seed=1)
    assert r["mv"] == prod(degs)


@pytest.mark.parametrize("sides", [[[1, 2, 1, 3], [2, 1, 1, 1], [1, 3, 2, 1], [1, 1, 1, 2]]])
def test_gpu_boxes_permanent(sides):
    k = len(sides)
    S = [[tuple(r[j] if (m >> j) & 1 else 0 for j in range(k)) for m in range(1 << k)] for r in sides]
    perm = sum(prod(sides[i][s[i]] for i in range(k)) for s in permutations(range(k)))
    assert bd.mixed_volume(S)["mv"] == perm


def test_gpu_unmixed_equals_volume():
    rng = np.random.default_rng(5)
    P = rng.integers(-2, 3, size=(9, 4))
    assert bd.mixed_volume([P] * 4)["mv"] == bd.volume(P)["nvol"]


def test_gpu_mixed_mid_size_equals_host_emulation():
    S = mixed_config("mixed_k5_p6")
    W = oracle_lifts(sum(len(A) for A in S), 2)
    g = bd.mixed_volume_lifted(S, W, cells=True)
    h = bd.host_mixed_volume_lifted(S, W, cells=True, leaf3=0)  # the two-level leaf stage
    assert g["status"] == 0 and g == {**h, "device_ms": g["device_ms"]}
    g128 = bd.mixed_volume_lifted(S, W, force_int128=True)
    assert g128["flags"] & bd.BD_FLAG_INT128 and (g128["mv"], g128["cells"], g128["singular"]) == \
        (g["mv"], g["cells"], g["singular"])


@pytest.mark.parametrize("name,tuples", [("mixed_k6_p7", 21 ** 6), ("mixed_k7_p8", 28 ** 7)])
def test_gpu_mixed_full_size(name, tuples):
    S = mixed_config(name)
    n = sum(len(A) for A in S)
    res = [bd.mixed_volume(S, seed=s)["mv"] for s in (0, 1, 2)]
    assert res[0] == res[1] == res[2] > 0
    W = oracle_lifts(n, 0)
    r = bd.mixed_volume_lifted(S, W, cells=True)
    assert r["status"] == 0 and r["mv"] == res[0] and r["tuples"] == tuples
    assert sum(r["absdet"]) == r["mv"] and len(r["cell_list"]) == r["cells"]
    SL = [A.tolist() for A in S]
    for c, v in zip(r["cell_list"], r["absdet"]):
        assert cell_status(SL, W, c) == ("accepted", v)
    # random tuples outside the list are not cells
    listed = set(r["cell_list"])
    rng = random.Random(3)
    pairs = [[(p, q) for p in range(len(A)) for q in range(p + 1, len(A))] for A in S]
    for _ in range(300):
        t = tuple(rng.choice(P) for P in pairs)
        if t not in listed:
            assert cell_status(SL, W, t)[0] != "accepted"


def test_gpu_mixed_errors():
    with pytest.raises(bd.BinodegError):
        bd.mixed_volume([[(i, 0) for i in range(40)], [(0, i) for i in range(30)]])
    r = bd.mixed_volume([[(0, 0)], [(0, 0), (1, 0)]])
    assert r["mv"] == 0 and r["flags"] & bd.BD_FLAG_DEGENERATE
