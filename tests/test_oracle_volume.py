"""Pins for the oracle's normalized volume (Sec. 4, Eq. deg-nvol, Eq. simplex-vol) and
its lower-facet test (Eq. lower-face), against closed forms and invariants."""

import itertools
import math
import random

import numpy as np
import pytest

from oracle.lifts import lifts as oracle_lifts, mix, GOLDEN, MASK
from oracle.lower_facet import (ACCEPTED, REJECTED, SINGULAR, TIE, lower_facet_status,
                                nvol_lifting_bruteforce)
from oracle.volume import det_int, nvol_placing, nvol_pyramid
from oracle.snf import det_fraction


def cube(k):
    return [p for p in itertools.product((0, 1), repeat=k)]


def cross(k):
    pts = []
    for i in range(k):
        for s in (1, -1):
            e = [0] * k
            e[i] = s
            pts.append(tuple(e))
    return pts


def unimodular(rng, k, steps=12):
    U = np.eye(k, dtype=np.int64)
    for _ in range(steps):
        i, j = rng.sample(range(k), 2)
        U[i] += rng.choice((-1, 1)) * U[j]
    if rng.random() < 0.5:
        U[0] *= -1
    return U


@pytest.mark.parametrize("seed", range(30))
def test_det_int_matches_rational_elimination(seed):
    rng = random.Random(seed)
    n = rng.randint(1, 6)
    M = [[rng.randint(-4, 4) for _ in range(n)] for _ in range(n)]
    assert det_int(M) == det_fraction(M)


def test_det_int_leibniz_small():
    rng = random.Random(7)
    for _ in range(50):
        n = rng.randint(1, 4)
        M = [[rng.randint(-5, 5) for _ in range(n)] for _ in range(n)]
        leib = 0
        for perm in itertools.permutations(range(n)):
            inv = sum(1 for a in range(n) for b in range(a + 1, n) if perm[a] > perm[b])
            leib += (-1) ** inv * math.prod(M[i][perm[i]] for i in range(n))
        assert det_int(M) == leib


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_unit_cube(k):
    assert nvol_placing(cube(k)) == math.factorial(k)
    if k <= 4:
        assert nvol_pyramid(cube(k)) == math.factorial(k)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_cross_polytope(k):
    assert nvol_placing(cross(k)) == 2 ** k
    if k <= 4:
        assert nvol_pyramid(cross(k)) == 2 ** k


@pytest.mark.parametrize("seed", range(10))
def test_simplex_is_abs_det(seed):
    rng = random.Random(seed)
    k = rng.randint(1, 5)
    while True:
        pts = [tuple(rng.randint(-4, 4) for _ in range(k)) for _ in range(k + 1)]
        d = det_fraction([[a - b for a, b in zip(p, pts[0])] for p in pts[1:]])
        if d:
            break
    assert nvol_placing(pts) == abs(d)
    assert nvol_pyramid(pts) == abs(d)
    std = [tuple([0] * k)] + [tuple(int(i == j) for j in range(k)) for i in range(k)]
    assert nvol_placing(std) == 1 and nvol_pyramid(std) == 1


@pytest.mark.parametrize("seed", range(8))
def test_zonotope_closed_form(seed):
    # Z = sum of segments [0, g_i]: NVol_k(Z) = k! * sum over k-subsets |det(g_S)|
    rng = random.Random(seed)
    k = rng.randint(2, 3)
    gens = [tuple(rng.randint(-2, 2) for _ in range(k)) for _ in range(k + 2)]
    pts = set()
    for mask in itertools.product((0, 1), repeat=len(gens)):
        pts.add(tuple(sum(b * g[c] for b, g in zip(mask, gens)) for c in range(k)))
    expect = math.factorial(k) * sum(abs(det_fraction(list(S))) for S in itertools.combinations(gens, k))
    assert nvol_placing(sorted(pts)) == expect
    assert nvol_pyramid(sorted(pts)) == expect


@pytest.mark.parametrize("seed", range(12))
def test_invariances_and_dilation(seed):
    rng = random.Random(seed)
    k = rng.randint(2, 4)
    pts = [tuple(rng.randint(-3, 3) for _ in range(k)) for _ in range(rng.randint(k + 2, 10))]
    base = nvol_placing(pts)
    assert base == nvol_pyramid(pts)
    # permutation
    perm = pts[:]
    rng.shuffle(perm)
    assert nvol_placing(perm) == base
    # translation
    t = [rng.randint(-5, 5) for _ in range(k)]
    assert nvol_placing([tuple(a + b for a, b in zip(p, t)) for p in pts]) == base
    # GL_k(Z)
    U = unimodular(rng, k)
    assert nvol_placing([tuple(int(x) for x in U @ np.array(p)) for p in pts]) == base
    # dilation by c multiplies by c^k
    c = rng.randint(2, 3)
    assert nvol_placing([tuple(c * x for x in p) for p in pts]) == c ** k * base
    # duplicates and points of the hull (vertex midpoints of segments scaled by 2) change nothing
    dup = pts + pts[:3]
    assert nvol_placing(dup) == base
    doubled = [tuple(2 * x for x in p) for p in pts]
    mids = [tuple(a + b for a, b in zip(p, q)) for p, q in zip(pts, pts[1:])]
    assert nvol_placing(doubled + mids) == 2 ** k * base


def test_degenerate_is_zero():
    pts = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0), (2, 3, 0)]
    assert nvol_placing(pts) == 0 and nvol_pyramid(pts) == 0


@pytest.mark.parametrize("lifts", [(1, 2, 3, 5), (7, 1, 1, 2), (3, 9, 4, 1), (10, 1, 10, 2)])
def test_unit_square_example(lifts):
    # Sec. 4 example: generic lifts of the unit square give two triangles, NVol 2
    S = [(0, 0), (0, 1), (1, 1), (1, 0)]
    total, acc, sing, ties = nvol_lifting_bruteforce(S, lifts)
    assert (total, acc, ties) == (2, 2, 0)


def test_lower_facet_strictness_and_ties():
    S = [(0, 0), (0, 1), (1, 1), (1, 0)]
    # lifted points coplanar (omega = x + y): every triangle has the 4th point on it
    assert nvol_lifting_bruteforce(S, (0, 1, 2, 1))[3] == 4
    # point (1,1) raised: the square splits along the anti-diagonal (0,1)-(1,0);
    # the two triangles cut by the main diagonal have a lifted point below them
    assert lower_facet_status(S, (0, 0, 5, 0), (0, 1, 3))[0] == ACCEPTED
    assert lower_facet_status(S, (0, 0, 5, 0), (1, 2, 3))[0] == ACCEPTED
    assert lower_facet_status(S, (0, 0, 5, 0), (0, 1, 2))[0] == REJECTED
    assert lower_facet_status(S, (0, 0, 5, 0), (0, 2, 3))[0] == REJECTED
    # three collinear points are singular
    assert lower_facet_status([(0, 0), (1, 1), (2, 2), (0, 1)], (1, 2, 3, 4), (0, 1, 2))[0] == SINGULAR


@pytest.mark.parametrize("seed", range(20))
def test_lifting_bruteforce_equals_hull_volume(seed):
    # a regular triangulation from generic lifts covers conv S (Sec. 4.1)
    rng = random.Random(seed)
    k = rng.randint(1, 3)
    pts = [tuple(rng.randint(-2, 2) for _ in range(k)) for _ in range(rng.randint(k + 1, 8))]
    lf = oracle_lifts(len(pts), seed)
    total, acc, sing, ties = nvol_lifting_bruteforce(pts, lf)
    assert ties == 0
    assert total == nvol_placing(pts) == nvol_pyramid(pts)


def test_splitmix64_published_vector():
    # Steele-Lea-Flood SplitMix64, state 1234567: first outputs of the reference stream
    s, out = 1234567, []
    for _ in range(5):
        s = (s + GOLDEN) & MASK
        out.append(mix(s))
    assert out == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]


def test_lift_range_and_attempts():
    a = oracle_lifts(1000, 42, 0)
    b = oracle_lifts(1000, 42, 1)
    assert all(1 <= x <= 2 ** 20 for x in a)
    assert a != b and a == oracle_lifts(1000, 42, 0)
