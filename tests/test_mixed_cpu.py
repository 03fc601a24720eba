"""The mixed-cell walker (bd_mixed.cuh) through its host emulation against the oracle
(oracle/mixed.py): the same fine mixed cells, |det M|, singular and tie counts under the same
heights, one-lane teams and lockstep teams of 7 and 32 lanes, the 64- and 128-bit paths, and
MV against the polarization formula; plus the argument checks of the C ABI."""

import random

import numpy as np
import pytest

import paper_1501_02237_gb300 as bd
from oracle.lifts import lifts as oracle_lifts
from oracle.mixed import mixed_cells, mixed_volume_polarization


def random_supports(rng, k, lo=2, hi=5, span=2):
    return [[tuple(rng.randint(0, span) for _ in range(k)) for _ in range(rng.randint(lo, hi))] for _ in range(k)]


def oracle_result(S, W):
    cells, sing, ties = mixed_cells(S, W)
    return cells, sing, ties


@pytest.mark.parametrize("seed", range(16))
def test_host_mixed_cells_match_oracle(seed):
    rng = random.Random(8100 + seed)
    k = rng.choice([1, 2, 2, 3, 3, 4])
    S = random_supports(rng, k, hi=5 if k < 4 else 4)
    W = oracle_lifts(sum(len(A) for A in S), seed)
    cells, sing, ties = oracle_result(S, W)
    # work items fixing every possible number of levels, one-lane teams and a 7-lane team, the
    # two-level leaf stage and the 3-D one (k >= 3)
    runs = [(1, 0, 0), (7, 0, 0)] + [(1, L, 0) for L in range(1, k)]
    if k >= 3:
        runs += [(1, 0, 1), (7, 0, 1)] + [(1, L, 1) for L in range(1, k - 1)]
    for width, levels, leaf3 in runs:
        r = bd.host_mixed_volume_lifted(S, W, team_width=width, cells=True, prefix_levels=levels, leaf3=leaf3)
        if ties:
            assert r["status"] == 3 and r["ties"] == ties
            continue
        assert r["status"] == 0
        assert r["cell_list"] == [c for c, _ in cells] and r["absdet"] == [v for _, v in cells]
        assert r["mv"] == sum(v for _, v in cells) and r["singular"] == sing
        assert r["tuples"] == np.prod([len(A) * (len(A) - 1) // 2 for A in S])


@pytest.mark.parametrize("seed", range(6))
def test_host_mixed_volume_equals_polarization(seed):
    rng = random.Random(8200 + seed)
    k = rng.choice([2, 3, 4])
    S = random_supports(rng, k, lo=3, hi=4 if k == 4 else 6)
    mv = mixed_volume_polarization(S)
    W = oracle_lifts(sum(len(A) for A in S), 100 + seed)
    r = bd.host_mixed_volume_lifted(S, W)
    if r["status"] == 0:
        assert r["mv"] == mv
    r32 = bd.host_mixed_volume_lifted(S, W, team_width=32, force_int128=True)
    assert (r32["status"], r32["mv"]) == (r["status"], r["mv"])
    r3 = bd.host_mixed_volume_lifted(S, W, team_width=32, leaf3=1)
    assert (r3["status"], r3["mv"], r3["singular"]) == (r["status"], r["mv"], r["singular"])


@pytest.mark.parametrize("k,degs", [(4, (2, 1, 2, 2)), (5, (1, 2, 1, 1, 2))])
def test_host_bezout_larger(k, degs):
    # all lattice points of d_i times the standard simplex: MV = prod d_i (Bezout)
    def simplex_points(d):
        out = []

        def rec(prefix, left):
            if len(prefix) == k:
                out.append(tuple(prefix))
                return
            for v in range(left + 1):
                rec(prefix + [v], left - v)
        rec([], d)
        return out
    S = [simplex_points(d) for d in degs]
    n = sum(len(A) for A in S)
    assert n <= 64
    r = None
    for seed in range(4):
        r = bd.host_mixed_volume_lifted(S, oracle_lifts(n, seed))
        if r["status"] == 0:
            break
    assert r["status"] == 0 and r["mv"] == int(np.prod(degs))


def test_host_unmixed_equals_normalized_volume():
    rng = random.Random(8300)
    k = 3
    P = [tuple(rng.randint(-2, 2) for _ in range(k)) for _ in range(7)]
    from oracle.volume import nvol_pyramid
    v = nvol_pyramid(P)
    W = oracle_lifts(3 * len(P), 5)
    r = bd.host_mixed_volume_lifted([P] * k, W)
    assert r["status"] == 0 and r["mv"] == v


def test_host_mixed_degenerate_and_errors():
    # a one-point set: MV 0, nothing enumerated, flagged
    r = bd.host_mixed_volume_lifted([[(0, 0)], [(0, 0), (1, 0), (0, 1)]], [1, 2, 3, 4])
    assert r["status"] == 0 and r["mv"] == 0 and r["flags"] & bd.BD_FLAG_DEGENERATE
    # coinciding points only
    r = bd.host_mixed_volume_lifted([[(1, 1), (1, 1)], [(0, 0), (1, 0)]], [1, 2, 3, 4])
    assert r["mv"] == 0 and r["flags"] & bd.BD_FLAG_DEGENERATE
    # parallel segments: every tuple singular
    r = bd.host_mixed_volume_lifted([[(0, 0), (1, 1)], [(0, 0), (2, 2)]], [1, 5, 2, 3])
    assert (r["mv"], r["singular"], r["tuples"]) == (0, 1, 1)
    with pytest.raises(ValueError):
        bd.host_mixed_volume_lifted([[(0, 0), (1, 0)]], [1, 2])  # 1 set in Z^2
    with pytest.raises(ValueError):
        bd._supports([[(0, 0), (1, 0)], [(0,), (1,)]])
    with pytest.raises(bd.BinodegError):  # the C ABI's own checks: k out of range
        P, cnt = np.zeros((2, 1), dtype=np.int64), np.array([2], dtype=np.int32)
        out = bd.MixedOut()
        bd.check(bd.lib().bd_host_mixed_volume_lifted(bd.ptr(P), cnt.ctypes.data_as(bd.I32P), 0,
                                                       bd.ptr(np.ones(2, dtype=np.int64)), 1, 0, 0, -1, out, None,
                                                       0, None))
    big = [[(i, 0) for i in range(40)], [(0, i) for i in range(30)]]
    with pytest.raises(bd.BinodegError):
        bd.host_mixed_volume_lifted(big, list(range(1, 71)))  # more than 64 points
    with pytest.raises(bd.BinodegError):
        bd.host_mixed_volume_lifted([[(0, 0), (1 << 41, 0)], [(0, 0), (0, 1)]], [1, 2, 3, 4])


def test_host_mixed_tie_reported():
    # constant heights: the square's two diagonals tie
    S = [[(0, 0), (1, 0), (0, 1), (1, 1)], [(0, 0), (1, 0), (0, 1), (1, 1)]]
    r = bd.host_mixed_volume_lifted(S, [0] * 8)
    assert r["status"] == 3 and r["ties"] > 0
    _, _, ties = oracle_result(S, [0] * 8)
    assert r["ties"] == ties


@pytest.mark.parametrize("seed,big", [(0, 1 << 20), (1, 1 << 20), (2, 1 << 30), (3, 1 << 30), (4, 1 << 24),
                                      (5, 1 << 26)])
def test_host_mixed_near_coplanar_lifts(seed, big):
    # heights big * <l, a> + small noise: every point sits within a few units of one plane, so
    # the single-precision filter cannot decide most tests and the exact route decides them
    rng = random.Random(8400 + seed)
    k = 3
    S = random_supports(rng, k, lo=3, hi=5)
    l = [rng.randint(-3, 3) for _ in range(k)]
    W = [big * sum(x * y for x, y in zip(p, l)) + rng.randint(-2, 2) for A in S for p in A]
    cells, sing, ties = oracle_result(S, W)
    for width, leaf3 in [(1, 0), (7, 0), (1, 1), (7, 1)]:
        r = bd.host_mixed_volume_lifted(S, W, team_width=width, cells=True, leaf3=leaf3)
        if ties:
            assert r["status"] == 3 and r["ties"] == ties
            continue
        assert r["cell_list"] == [c for c, _ in cells] and r["singular"] == sing
