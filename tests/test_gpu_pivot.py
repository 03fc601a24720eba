"""Simplicial pivoting on the GPU (bd_volume_pivot, bd_degree_pivot): the same volume as the
subset enumeration and the same cells as the host emulation on random point sets; the
master-space degrees of Table mspace-deg, which the subset enumeration cannot reach
(W_{2,7} .. W_{4,4}: 4.2e11 to 1.9e13 subsets, dimensions 16 to 18); 65 to 127 points (two-word
cell masks) against the oracle's placing volume, and bd_degree's route to the walk there."""

import json
import os
import random

import numpy as np
import pytest

import paper_1501_02237_gb300 as bd
from oracle.lifts import ATTEMPT_MULT, GOLDEN, MASK, mix
from oracle.volume import nvol_placing
from workloads import config_system, master_space_system

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLE = json.load(open(os.path.join(ROOT, "tests", "golden", "master_space_table.json")))


def wide_lifts(n, seed, attempt=0):
    """The pivoting path's heights: the top 40 bits of the SplitMix64 lift stream."""
    s = mix((seed ^ (attempt * ATTEMPT_MULT)) & MASK)
    return [1 + (mix((s + (i + 1) * GOLDEN) & MASK) >> 24) for i in range(n)]


@pytest.mark.parametrize("seed", range(16))
def test_gpu_pivot_equals_subset_enumeration(seed):
    rng = random.Random(7600 + seed)
    k = rng.choice([2, 3, 4, 5, 6, 8])
    n = rng.randint(k + 2, 24)
    P = np.array([[rng.randint(-3, 3) for _ in range(k)] for _ in range(n)])
    v = bd.volume(P, seed=seed)
    p = bd.volume_pivot(P, seed=seed)
    assert p["nvol"] == v["nvol"]
    if p["relifts"] == 0 and not (p["flags"] & bd.BD_FLAG_DEGENERATE):
        # the host emulation with the same heights walks the same cells
        h = bd.host_volume_pivot(P, wide_lifts(n, seed), cells=True)
        assert (h["nvol"], h["cells"]) == (p["nvol"], p["cells"])


def test_gpu_pivot_config_system():
    P = bd.reduce(config_system("single_n24_k8").A)["points"]
    assert bd.volume_pivot(P)["nvol"] == bd.volume(P)["nvol"] == 8271351


@pytest.mark.parametrize("mk", ["3,3", "2,6", "3,4", "4,3", "2,7", "7,2", "3,5", "5,3", "4,4", "2,8", "8,2", "3,6",
                                "6,3"])
def test_gpu_pivot_master_space_table(mk):
    m, k = map(int, mk.split(","))
    s = master_space_system(m, k)
    r = bd.degree_pivot(s.A, s.coef)
    assert r["consistent"] and r["degree"] == TABLE["degree"][mk]
    assert r["dim"] == m * k + 2


def test_gpu_pivot_lift_independence():
    s = master_space_system(2, 7)
    P = bd.reduce(s.A)["points"]
    res = {bd.volume_pivot(P, seed=sd)["nvol"] for sd in (0, 1, 2)}
    assert res == {TABLE["degree"]["2,7"]}


@pytest.mark.parametrize("mk", ["2,7", "3,5"])
def test_gpu_degree_above_kmax_walks_the_cells(mk):
    # dimension 16 / 17 > BD_KMAX: bd_degree itself takes the pivoting walk
    m, k = map(int, mk.split(","))
    s = master_space_system(m, k)
    r = bd.degree(s.A, s.coef)
    assert r["flags"] & bd.BD_FLAG_PIVOT
    assert r["dim"] == m * k + 2 > bd.KMAX and r["degree"] == TABLE["degree"][mk]


@pytest.mark.parametrize("seed", range(6))
def test_gpu_subset_cells_equal_pivot_walk(seed):
    # the GPU subset enumeration's cells (bd_cells) and the pivoting walk under the same heights
    rng = random.Random(7900 + seed)
    k = rng.choice([4, 5, 6, 8])
    n = rng.randint(k + 6, 22)
    P = np.array([[rng.randint(-3, 3) for _ in range(k)] for _ in range(n)])
    cells, vol = bd.cells(P, seed=seed, capacity=1 << 15)
    if vol["relifts"] or vol["flags"] & bd.BD_FLAG_DEGENERATE:
        return
    from oracle.lifts import lifts as oracle_lifts
    piv = bd.host_volume_pivot(P, oracle_lifts(n, seed), cells=True)
    assert piv["status"] == 0
    assert set(piv["cell_list"]) == {tuple(sorted(c["cell"])) for c in cells}
    assert piv["nvol"] == vol["nvol"]


@pytest.mark.parametrize("seed", range(8))
def test_gpu_pivot_two_word_masks_match_oracle(seed):
    # more than 64 points: cells are two-word masks; exact against the oracle's placing volume
    rng = random.Random(8400 + seed)
    k = [3, 4, 5, 6, 4, 5, 3, 4][seed]
    n = [65, 127, rng.randint(66, 126), rng.randint(66, 80), 100, 120, 127, 64][seed]
    pts = [tuple(rng.randint(-3, 3) for _ in range(k)) for _ in range(n)]
    r = bd.volume_pivot(np.array(pts), seed=seed)
    assert r["nvol"] == nvol_placing(pts)
    if r["relifts"] == 0 and not (r["flags"] & bd.BD_FLAG_DEGENERATE):
        h = bd.host_volume_pivot(np.array(pts), wide_lifts(n, seed))
        assert (h["nvol"], h["cells"]) == (r["nvol"], r["cells"])


def test_gpu_degree_beyond_64_points_walks_the_cells():
    # 89 variables, solution set of dimension 5: 90 points, past the subset enumeration
    rng = random.Random(8500)
    d, n = 5, 89
    R = np.array([[rng.randint(-2, 2) for _ in range(d)] for _ in range(n - d)], dtype=np.int64)
    A = np.vstack([-R.T, np.eye(n - d, dtype=np.int64)])  # kernel lattice spanned by [I; R]
    pts = [tuple(int(v) for v in row) for row in np.vstack([np.eye(d, dtype=np.int64), R])] + [(0,) * d]
    g = bd.degree(A)
    assert g["flags"] & bd.BD_FLAG_PIVOT
    assert g["nvol"] == nvol_placing(pts) and g["degree"] == g["nvol"] * g["torsion"]
    assert bd.degree_pivot(A)["degree"] == g["degree"]


@pytest.mark.parametrize("seed", range(6))
def test_gpu_pivot_wide_tableau_matches_oracle(seed):
    # cell-minor bounds past 2^62 (random coordinates in [-6, 6] times 2^12..2^16): the GPU walk
    # takes 128-bit tableau entries (BD_FLAG_INT128); exact against the oracle's placing volume,
    # and the same volume and cell count as the host emulation with the same heights
    rng = random.Random(8900 + seed)
    k = [4, 4, 5, 4, 5, 4][seed]
    n = [12, 24, 14, 40, 30, 80][seed]
    sh = [14, 12, 10, 16, 11, 14][seed]
    pts = sorted({tuple(rng.randint(-6, 6) << sh for _ in range(k)) for _ in range(n)})
    n = len(pts)
    r = bd.volume_pivot(np.array(pts), seed=seed)
    assert r["flags"] & bd.BD_FLAG_INT128 and r["bound_bits"] > 62
    assert r["nvol"] == nvol_placing(pts)
    if r["relifts"] == 0:
        h = bd.host_volume_pivot(np.array(pts), wide_lifts(n, seed))
        assert (h["nvol"], h["cells"]) == (r["nvol"], r["cells"])


@pytest.mark.parametrize("seed", range(4))
def test_gpu_pivot_forced_wide_tableau_two_word_masks(seed):
    # the 128-bit tableau forced (test hook) with one- and two-word masks: the same volume and cell
    # count as the 64-bit tableau on the GPU, exact against the oracle's placing volume
    rng = random.Random(8950 + seed)
    k = [3, 4, 5, 4][seed]
    n = [40, 70, 100, 127][seed]
    pts = [tuple(rng.randint(-3, 3) for _ in range(k)) for _ in range(n)]
    narrow = bd.volume_pivot(np.array(pts), seed=seed)
    prev = bd.pivot_force_wide(True)
    try:
        wide = bd.volume_pivot(np.array(pts), seed=seed)
    finally:
        bd.pivot_force_wide(prev)
    assert wide["flags"] & bd.BD_FLAG_INT128 and not narrow["flags"] & bd.BD_FLAG_INT128
    assert (wide["nvol"], wide["cells"], wide["relifts"]) == (narrow["nvol"], narrow["cells"], narrow["relifts"])
    assert wide["nvol"] == nvol_placing(pts)


@pytest.mark.parametrize("seed", range(3))
def test_gpu_pivot_random_large_coordinates(seed):
    # random coordinates up to 2^16 (Z^4) and 2^13 (Z^5): bounds past 2^62 and start cells formed
    # in 256-bit steps; exact against the oracle's placing volume
    rng = random.Random(8980 + seed)
    k, bits, n = [(4, 16, 40), (5, 13, 30), (4, 17, 70)][seed]
    pts = set()
    while len(pts) < n:
        pts.add(tuple(rng.randint(-(1 << bits) + 1, (1 << bits) - 1) for _ in range(k)))
    pts = sorted(pts)
    r = bd.volume_pivot(np.array(pts), seed=seed)
    assert r["flags"] & bd.BD_FLAG_INT128 and r["bound_bits"] > 62
    assert r["nvol"] == nvol_placing(pts)
