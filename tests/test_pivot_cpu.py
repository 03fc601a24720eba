"""Simplicial pivoting (bd_pivot.cuh) through its host emulation: the cells it walks are exactly
the oracle's lower facets of the same lifting (oracle/cells.py, rational arithmetic) and its
volume the oracle's placing-triangulation volume, for one-lane teams and a lockstep team of 7
lanes, with every cell eliminated or cells entered in place by tableau pivots; the master-space degrees of Table mspace-deg far beyond the subset enumeration
(W_{2,6}, W_{3,4}, W_{4,3}, W_{2,7}: 9.4e9 and 4.2e11 subsets); degenerate inputs, ties and
argument errors."""

import json
import os
import random

import numpy as np
import pytest

import paper_1501_02237_gb300 as bd
from paper_1501_02237_gb300._lib import BD_ERR_CUDA
from oracle.cells import lower_cells
from oracle.lifts import lifts as oracle_lifts
from oracle.volume import nvol_placing
from workloads import master_space_system

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLE = json.load(open(os.path.join(ROOT, "tests", "golden", "master_space_table.json")))


@pytest.mark.parametrize("seed", range(24))
def test_host_pivot_cells_match_oracle(seed):
    rng = random.Random(7300 + seed)
    k = rng.choice([1, 2, 3, 4, 5])
    n = rng.randint(k + 2, 11)
    pts = [tuple(rng.randint(-2, 2) for _ in range(k)) for _ in range(n)]
    W = oracle_lifts(n, seed)
    ref = lower_cells(pts, W)
    # one lane and a 7-lane team; every cell eliminated (budget 0) or walked into in place
    for width, budget in [(1, 0), (7, 0), (1, 1), (1, 64), (7, 64)]:
        r = bd.host_volume_pivot(np.array(pts), W, team_width=width, cells=True, walk_budget=budget)
        if r["flags"] & bd.BD_FLAG_DEGENERATE:
            assert nvol_placing(pts) == 0
            continue
        assert r["status"] == 0
        assert set(r["cell_list"]) == {tuple(sorted(c[0])) for c in ref}
        assert r["nvol"] == sum(c[1] for c in ref) == nvol_placing(pts)
        assert r["cells"] == len(ref) and r["subsets"] == (k + 1) * len(ref)


@pytest.mark.parametrize("seed", range(6))
def test_host_pivot_larger_sets_match_placing(seed):
    rng = random.Random(7400 + seed)
    k = rng.choice([3, 4, 5, 6])
    n = rng.randint(12, 20)
    pts = [tuple(rng.randint(-3, 3) for _ in range(k)) for _ in range(n)]
    r = bd.host_volume_pivot(np.array(pts), oracle_lifts(n, seed))
    if r["status"] == 0:
        assert r["nvol"] == nvol_placing(pts)


@pytest.mark.parametrize("mk", ["3,3", "2,5", "2,6", "3,4", "4,3"])
def test_host_pivot_master_space_table(mk):
    m, k = map(int, mk.split(","))
    s = master_space_system(m, k)
    red = bd.reduce(s.A)
    P = red["points"]
    for budget in (0, 64):
        r = bd.host_volume_pivot(P, oracle_lifts(P.shape[0], 0), walk_budget=budget)
        assert r["status"] == 0
        assert r["nvol"] * red["torsion"] == TABLE["degree"][mk]


def test_host_pivot_degenerate_ties_and_errors():
    # points on a plane in Z^3: not full-dimensional
    flat = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [2, 1, 0]])
    r = bd.host_volume_pivot(flat, [1, 5, 2, 9, 4])
    assert r["nvol"] == 0 and r["flags"] & bd.BD_FLAG_DEGENERATE
    # constant heights on the unit square: the two triangulations tie
    sq = np.array([[0, 0], [1, 0], [0, 1], [1, 1]])
    assert bd.host_volume_pivot(sq, [5, 5, 5, 5])["status"] == 3
    # affine heights (x + y): all four lifted points on one plane
    assert bd.host_volume_pivot(sq, [0, 1, 1, 2])["status"] == 3
    with pytest.raises(bd.BinodegError):
        bd.host_volume_pivot(np.zeros((3, 31), dtype=np.int64), [1, 2, 3])  # k above 30
    with pytest.raises(bd.BinodegError):
        bd.host_volume_pivot(np.array([[0], [1 << 21]]), [1, 2])  # coordinate range
    with pytest.raises(bd.BinodegError):
        bd.host_volume_pivot(sq, [1, 2, 3, 4], team_width=40)


@pytest.mark.parametrize("seed", range(6))
def test_host_pivot_cells_equal_subset_enumeration(seed):
    # the two walkers of the library, under the same heights, list the same triangulation
    rng = random.Random(7800 + seed)
    k = rng.choice([4, 5, 6, 7])
    n = rng.randint(k + 6, 18)
    P = np.array([[rng.randint(-3, 3) for _ in range(k)] for _ in range(n)])
    W = oracle_lifts(n, seed)
    piv = bd.host_volume_pivot(P, W, cells=True)
    if piv["status"] != 0 or piv["flags"] & bd.BD_FLAG_DEGENERATE:
        return
    enum = bd.host_cells(P, W, capacity=1 << 14)
    assert set(piv["cell_list"]) == {tuple(sorted(c["cell"])) for c in enum}


def wide_system(n, d, rng):
    """A system in n variables whose solution set has dimension d and whose kernel lattice is
    spanned by the columns of [I_d; R]: A = [-R^T; I_{n-d}], so the points of Eq. 6 are e_1..e_d,
    the rows of R and the origin (up to a unimodular change of basis)."""
    R = np.array([[rng.randint(-2, 2) for _ in range(d)] for _ in range(n - d)], dtype=np.int64)
    A = np.vstack([-R.T, np.eye(n - d, dtype=np.int64)])
    pts = [tuple(int(v) for v in row) for row in np.vstack([np.eye(d, dtype=np.int64), R])] + [(0,) * d]
    return A, pts


@pytest.mark.parametrize("seed", range(5))
def test_host_pivot_two_word_masks_match_placing(seed):
    # 65..127 points: cells are two-word masks; cells and volume as for one-word masks
    rng = random.Random(8100 + seed)
    k = rng.choice([3, 4, 5])
    n = [65, 90, 127, rng.randint(66, 126), rng.randint(66, 126)][seed]
    pts = [tuple(rng.randint(-3, 3) for _ in range(k)) for _ in range(n)]
    W = oracle_lifts(n, seed)
    for width, budget in [(1, 0), (7, 64)]:
        r = bd.host_volume_pivot(np.array(pts), W, team_width=width, walk_budget=budget)
        assert r["status"] == 0
        assert r["nvol"] == nvol_placing(pts)
        assert r["subsets"] == (k + 1) * r["cells"]


def test_reduce_beyond_64_variables():
    rng = random.Random(8200)
    A, pts = wide_system(90, 4, rng)
    red = bd.reduce(A)
    assert red["dim"] == 4 and red["torsion"] == 1 and red["points"].shape == (91, 4)
    # the reduced points are the kernel basis up to a unimodular map: same normalized volume
    W = oracle_lifts(91, 1)
    r = bd.host_volume_pivot(red["points"], W)
    assert r["status"] == 0 and r["nvol"] == nvol_placing(pts)
    with pytest.raises(bd.BinodegError):
        bd.reduce(np.zeros((127, 3), dtype=np.int64))  # above 126 variables


def test_two_word_mask_errors():
    rng = random.Random(8300)
    pts = np.array([[rng.randint(-3, 3) for _ in range(3)] for _ in range(80)])
    with pytest.raises(bd.BinodegError):
        bd.host_volume_pivot(pts, oracle_lifts(80, 0), cells=True)  # cell lists: 64 points at most
    big = np.array([[rng.randint(-3, 3) for _ in range(3)] for _ in range(128)])
    with pytest.raises(bd.BinodegError):
        bd.host_volume_pivot(big, oracle_lifts(128, 0))  # above 127 points


def big_coordinate_set(rng, n, k, bits):
    """n random points in Z^k with coordinates below 2^bits in magnitude (distinct points)."""
    pts = set()
    while len(pts) < n:
        pts.add(tuple(rng.randint(-(1 << bits) + 1, (1 << bits) - 1) for _ in range(k)))
    return sorted(pts)


def hadamard_bits(pts):
    """log2 of the pivoting path's bound on the cell minors: the product of the k largest norms
    ||a_x - a_s|| over one base point s, maximised over s (as the library computes it)."""
    import math
    k, best = len(pts[0]), 0.0
    for s in pts:
        lg = sorted((0.5 * math.log2(max(sum((a - b) ** 2 for a, b in zip(x, s)), 1))) for x in pts)[::-1]
        best = max(best, sum(lg[:k]))
    return best


@pytest.mark.parametrize("seed", range(5))
def test_host_pivot_wide_tableau_matches_placing(seed):
    # cell-minor bounds past 2^62: random points with coordinates in [-6, 6] multiplied by
    # 2^12..2^16.  The tableau takes 128-bit entries (BD_FLAG_INT128);
    # the volume equals the oracle's placing volume of the given points and, for the smallest
    # sets, the cells equal the oracle's lower facets of the same lifting; one lane and a 7-lane
    # lockstep team, every cell eliminated or walked into in place
    rng = random.Random(8600 + seed)
    k = [4, 4, 5, 4, 5][seed]
    n = [12, 24, 14, 40, 30][seed]
    sh = [14, 12, 10, 16, 11][seed]
    pts = sorted({tuple(rng.randint(-6, 6) << sh for _ in range(k)) for _ in range(n)})
    n = len(pts)
    assert hadamard_bits(pts) > 62
    W = oracle_lifts(n, seed)
    ref_vol = nvol_placing(pts)
    ref = lower_cells(pts, W) if n <= 14 else None
    for width, budget in [(1, 0), (7, 64)]:
        r = bd.host_volume_pivot(np.array(pts), W, team_width=width, walk_budget=budget, cells=ref is not None)
        assert r["status"] == 0
        assert r["flags"] & bd.BD_FLAG_INT128 and r["bound_bits"] > 62
        assert r["nvol"] == ref_vol
        assert r["subsets"] == (k + 1) * r["cells"]
        if ref is not None:
            assert set(r["cell_list"]) == {tuple(sorted(c[0])) for c in ref}


@pytest.mark.parametrize("seed", range(6))
def test_host_pivot_random_large_coordinates(seed):
    # random coordinates up to 2^17 in Z^4, 2^14 in Z^5, 2^11 in Z^6: bounds past 2^62, and
    # start cells whose extension steps pass 2^128 before their gcd reduction (formed in 256
    # bits); exact against the oracle's placing volume
    rng = random.Random(8660 + seed)
    k, bits = [(4, 16), (4, 17), (5, 13), (5, 14), (6, 11), (4, 16)][seed]
    n = [20, 30, 16, 24, 14, 64][seed]
    pts = big_coordinate_set(rng, n, k, bits)
    assert hadamard_bits(pts) > 62
    r = bd.host_volume_pivot(np.array(pts), oracle_lifts(n, seed), team_width=1 if n > 30 else 7)
    assert r["status"] == 0 and r["flags"] & bd.BD_FLAG_INT128
    assert r["nvol"] == nvol_placing(pts)


@pytest.mark.parametrize("seed", range(4))
def test_host_pivot_forced_wide_tableau_matches_oracle(seed):
    # the 128-bit tableau forced (test hook) on small sets: the cells equal the oracle's lower
    # facets, the volume its placing volume
    rng = random.Random(8620 + seed)
    k = [2, 3, 4, 5][seed]
    n = [9, 11, 12, 12][seed]
    pts = [tuple(rng.randint(-3, 3) for _ in range(k)) for _ in range(n)]
    W = oracle_lifts(n, seed)
    ref = lower_cells(pts, W)
    prev = bd.pivot_force_wide(True)
    try:
        for width, budget in [(1, 0), (1, 64), (7, 64)]:
            r = bd.host_volume_pivot(np.array(pts), W, team_width=width, walk_budget=budget, cells=True)
            if r["flags"] & bd.BD_FLAG_DEGENERATE:
                assert nvol_placing(pts) == 0
                continue
            assert r["status"] == 0 and r["flags"] & bd.BD_FLAG_INT128
            assert set(r["cell_list"]) == {tuple(sorted(c[0])) for c in ref}
            assert r["nvol"] == sum(c[1] for c in ref) == nvol_placing(pts)
    finally:
        bd.pivot_force_wide(prev)


@pytest.mark.parametrize("seed", range(3))
def test_host_pivot_wide_tableau_two_word_masks(seed):
    # 128-bit tableau entries (forced by the test hook) with two-word masks (65..127 points):
    # the same volume as the oracle's placing volume and as the 64-bit tableau
    rng = random.Random(8650 + seed)
    k = [3, 4, 5][seed]
    n = [70, 100, 127][seed]
    pts = [tuple(rng.randint(-3, 3) for _ in range(k)) for _ in range(n)]
    W = oracle_lifts(n, seed)
    narrow = bd.host_volume_pivot(np.array(pts), W)
    prev = bd.pivot_force_wide(True)
    try:
        for width, budget in [(1, 0), (7, 64)]:
            r = bd.host_volume_pivot(np.array(pts), W, team_width=width, walk_budget=budget)
            assert r["status"] == 0 and r["flags"] & bd.BD_FLAG_INT128
            assert (r["nvol"], r["cells"]) == (narrow["nvol"], narrow["cells"])
    finally:
        bd.pivot_force_wide(prev)
    assert not narrow["flags"] & bd.BD_FLAG_INT128
    assert narrow["nvol"] == nvol_placing(pts)


def test_host_pivot_wide_tableau_agrees_with_narrow():
    # the same points below the 62-bit bound, run with 64-bit entries, and scaled by 2^14 (bound
    # past 62 bits, 128-bit entries): NVol scales by 2^(14k) and the cells stay the same
    rng = random.Random(8700)
    k, n = 4, 30
    pts = [tuple(rng.randint(-6, 6) for _ in range(k)) for _ in range(n)]
    W = oracle_lifts(n, 5)
    a = bd.host_volume_pivot(np.array(pts), W, cells=True)
    big = np.array(pts, dtype=np.int64) << 14
    b = bd.host_volume_pivot(big, W, cells=True)
    assert a["status"] == b["status"] == 0
    assert not (a["flags"] & bd.BD_FLAG_INT128) and b["flags"] & bd.BD_FLAG_INT128
    assert b["nvol"] == a["nvol"] << (14 * k)
    assert b["cell_list"] == a["cell_list"] and b["cells"] == a["cells"]


def test_pivot_refuses_heights_past_the_bound():
    # W_{4,6}: 73 points in dimension 26, Hadamard bound of the cell minors 84 bits: the heights
    # (a minor times a 41-bit lift difference, 27 terms) may leave 127 bits; the refusal comes from
    # the host before any device work.  W_{3,8} (65 bits) takes the 128-bit tableau instead.
    A = master_space_system(4, 6).A
    with pytest.raises(bd.BinodegError, match="127 bits"):
        bd.degree_pivot(A)
    rng = random.Random(8800)
    pts = big_coordinate_set(rng, 12, 6, 19)  # 6 x ~20 bits + 41 > 126
    with pytest.raises(bd.BinodegError, match="127 bits"):
        bd.host_volume_pivot(np.array(pts), oracle_lifts(12, 0))


def test_device_paths_fail_loudly_without_a_gpu():
    # no host fallback: without a CUDA device the GPU entry points return BD_ERR_CUDA
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    rng = random.Random(8600)
    small = np.array([[0, 0], [1, 0], [0, 1], [1, 1], [2, 1]])
    A, _ = wide_system(80, 3, rng)  # 81 points: bd_degree routes it to the walk
    supports = [np.array([[0, 0], [1, 0], [0, 1]]), np.array([[0, 0], [2, 0], [0, 1], [1, 1]])]
    for call in (lambda: bd.volume(small), lambda: bd.volume_pivot(small), lambda: bd.degree(A),
                 lambda: bd.degree_pivot(A), lambda: bd.mixed_volume(supports),
                 lambda: bd.start_solutions(small), lambda: bd.cells(small)):
        with pytest.raises(bd.BinodegError) as err:
            call()
        assert err.value.code == BD_ERR_CUDA
