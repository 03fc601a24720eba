"""Pins of oracle/mixed.py against closed forms of the mixed volume and against each other:
Bezout's count for scaled simplices, the permanent for boxes, |det| for segments, the
unmixed case MV(P, .., P) = NVol(P) (the degree case, Appendix A), symmetry, translation and
unimodular invariance, and the lifting route against the polarization route on random
supports under several liftings."""

import random
from itertools import permutations
from math import prod

import pytest

from oracle.lifts import lifts as oracle_lifts
from oracle.mixed import (cell_status, mixed_cells, mixed_volume_lifting, mixed_volume_polarization,
                          REJECTED, SINGULAR)
from oracle.volume import det_int, nvol_pyramid


def simplex(d, k, full=False):
    """d times the standard simplex: its vertices, or all its lattice points."""
    if not full:
        return [tuple(0 for _ in range(k))] + [tuple(d if j == i else 0 for j in range(k)) for i in range(k)]
    pts = []

    def rec(prefix, left):
        if len(prefix) == k:
            pts.append(tuple(prefix))
            return
        for v in range(left + 1):
            rec(prefix + [v], left - v)
    rec([], d)
    return pts


def box(sides):
    k = len(sides)
    return [tuple(sides[j] if (m >> j) & 1 else 0 for j in range(k)) for m in range(1 << k)]


def both(supports, seed=0):
    n = sum(len(A) for A in supports)
    mv_l, _, _, ties = mixed_volume_lifting(supports, oracle_lifts(n, seed))
    assert ties == 0
    return mixed_volume_polarization(supports), mv_l


@pytest.mark.parametrize("degs,full", [((2, 3), False), ((1, 4), True), ((2, 2, 3), False), ((1, 2, 2), True),
                                       ((3, 1, 2), False)])
def test_bezout_scaled_simplices(degs, full):
    k = len(degs)
    S = [simplex(d, k, full) for d in degs]
    assert both(S) == (prod(degs), prod(degs))


@pytest.mark.parametrize("sides", [[[1, 2], [3, 1]], [[2, 1], [1, 1]], [[1, 2, 1], [2, 1, 1], [1, 1, 3]]])
def test_boxes_give_the_permanent(sides):
    k = len(sides)
    perm = sum(prod(sides[i][s[i]] for i in range(k)) for s in permutations(range(k)))
    assert both([box(r) for r in sides]) == (perm, perm)


@pytest.mark.parametrize("seed", range(4))
def test_segments_give_the_determinant(seed):
    rng = random.Random(300 + seed)
    k = rng.choice([2, 3])
    V = [[rng.randint(-3, 3) for _ in range(k)] for _ in range(k)]
    S = [[tuple(0 for _ in range(k)), tuple(v)] for v in V]
    d = abs(det_int(V))
    assert both(S) == (d, d)


@pytest.mark.parametrize("seed", range(4))
def test_unmixed_is_the_normalized_volume(seed):
    rng = random.Random(400 + seed)
    k = rng.choice([2, 3])
    P = [tuple(rng.randint(-2, 2) for _ in range(k)) for _ in range(rng.randint(k + 1, 6))]
    v = nvol_pyramid(P)
    assert both([P] * k) == (v, v)


@pytest.mark.parametrize("seed", range(8))
def test_lifting_route_equals_polarization(seed):
    rng = random.Random(500 + seed)
    k = rng.choice([2, 2, 3, 3])
    S = [[tuple(rng.randint(0, 2) for _ in range(k)) for _ in range(rng.randint(2, 5))] for _ in range(k)]
    pol = mixed_volume_polarization(S)
    n = sum(len(A) for A in S)
    for ls in range(3):
        mv, _, _, ties = mixed_volume_lifting(S, oracle_lifts(n, seed * 10 + ls))
        if ties == 0:
            assert mv == pol


def test_invariances():
    rng = random.Random(77)
    k = 3
    S = [[tuple(rng.randint(0, 2) for _ in range(k)) for _ in range(4)] for _ in range(k)]
    mv = mixed_volume_polarization(S)
    assert mv > 0
    # symmetric in the components
    assert mixed_volume_lifting([S[2], S[0], S[1]], oracle_lifts(12, 3))[0] == mv
    # each component may be translated on its own
    T = [[tuple(x + t for x, t in zip(p, sh)) for p in A] for A, sh in zip(S, [(1, -2, 0), (0, 0, 3), (-1, 1, 1)])]
    assert mixed_volume_lifting(T, oracle_lifts(12, 0))[0] == mv
    # a common unimodular map
    U = [[1, 1, 0], [0, 1, 2], [0, 0, 1]]
    UT = [[tuple(sum(U[r][c] * p[c] for c in range(k)) for r in range(k)) for p in A] for A in S]
    assert mixed_volume_lifting(UT, oracle_lifts(12, 0))[0] == mv
    # multilinear: doubling one component doubles MV
    D = [[tuple(2 * x for x in p) for p in S[0]]] + S[1:]
    assert mixed_volume_lifting(D, oracle_lifts(12, 0))[0] == 2 * mv


def test_degenerate_supports():
    # a one-point component: no pairs, MV 0
    assert both([[(0, 0)], [(0, 0), (1, 1), (2, 0)]]) == (0, 0)
    # two parallel segments in the plane: MV 0, every tuple singular
    S = [[(0, 0), (1, 1)], [(0, 0), (2, 2)]]
    assert both(S) == (0, 0)
    assert cell_status(S, [1, 5, 2, 3], ((0, 1), (0, 1)))[0] == SINGULAR


def test_cell_status_by_hand():
    # A_1 = {0, e1, e2}, A_2 = {0, e1}: MV = 1 (a line x + c = 0 meets a generic line once)
    S = [[(0, 0), (1, 0), (0, 1)], [(0, 0), (1, 0)]]
    # heights 0 at the origin of A_1, large elsewhere; A_2 flat
    w = [0, 10, 10, 0, 0]
    # cell ({0, e2}, {0, e1}): alpha solves alpha_2 = -10, alpha_1 = 0; e1 in A_1 gives 0 + 10 > 0
    st, v = cell_status(S, w, ((0, 2), (0, 1)))
    assert (st, v) == ("accepted", 1)
    # ({0, e1}, {0, e1}) is singular, ({e1, e2}, ..): the origin of A_1 lies below
    assert cell_status(S, w, ((0, 1), (0, 1)))[0] == SINGULAR
    assert cell_status(S, w, ((1, 2), (0, 1)))[0] == REJECTED
    cells, sing, ties = mixed_cells(S, w)
    assert [c for c, _ in cells] == [((0, 2), (0, 1))] and ties == 0
