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


def test_pivot_refuses_minors_past_the_bound():
    # W_{3,8}: 73 points in dimension 26, Hadamard bound of the cell minors 65 bits > 62; the
    # refusal comes from the host before any device work
    A = master_space_system(3, 8).A
    with pytest.raises(bd.BinodegError, match="62 bits"):
        bd.degree_pivot(A)


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
