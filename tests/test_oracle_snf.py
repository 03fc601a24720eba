"""Pins for the oracle's Smith Normal Form (Sec. 3, Eq. smith, Props. 1-2)."""

import itertools
import math
import random

import numpy as np
import pytest

from oracle.snf import BinomialStructure, _bezout, det_fraction, matmul, smith_normal_form


@pytest.mark.parametrize("a1,a2", [(4, 6), (6, 4), (-3, 5), (7, 0 + 21), (2, -2), (-12, -18), (1, 9)])
def test_bezout_2x1_example(a1, a2):
    # Sec. 3: P = [[s, t], [-a2/d, a1/d]] has det 1 and sends (a1, a2)^T to (d, 0)^T
    s, t, u, v = _bezout(a1, a2)
    assert s * v - t * u == 1
    top, bottom = s * a1 + t * a2, u * a1 + v * a2
    assert bottom == 0
    assert abs(top) == math.gcd(a1, a2)


def _random_int_matrix(rng, n, m, lo=-3, hi=3, rank_drop=0):
    A = [[rng.randint(lo, hi) for _ in range(m)] for _ in range(n)]
    for _ in range(rank_drop):  # make a row a combination of two others
        if n >= 3:
            i, j, k = rng.sample(range(n), 3)
            A[i] = [A[j][c] * 2 - A[k][c] for c in range(m)]
    return A


def _gcd_of_minors(A, r):
    n, m = len(A), len(A[0])
    g = 0
    for rows in itertools.combinations(range(n), r):
        for cols in itertools.combinations(range(m), r):
            g = math.gcd(g, det_fraction([[A[i][j] for j in cols] for i in rows]))
    return g


@pytest.mark.parametrize("seed", range(25))
def test_snf_invariants(seed):
    rng = random.Random(seed)
    n, m = rng.randint(1, 5), rng.randint(1, 5)
    A = _random_int_matrix(rng, n, m, rank_drop=seed % 2)
    P, D, Q, r = smith_normal_form(A)
    # P A Q = D, diagonal with the nonzero entries first
    assert matmul(matmul(P, A), Q) == D
    for i in range(n):
        for j in range(m):
            if i != j or i >= r:
                assert D[i][j] == 0
    assert all(D[i][i] != 0 for i in range(r))
    # unimodular transforms
    assert abs(det_fraction(P)) == 1 and abs(det_fraction(Q)) == 1
    # rank and torsion: |prod d_j| equals the gcd of the r x r minors (Prop. 1)
    assert r == np.linalg.matrix_rank(np.array(A, dtype=float))
    prod = 1
    for i in range(r):
        prod *= D[i][i]
    if r:
        assert abs(prod) == _gcd_of_minors(A, r)


@pytest.mark.parametrize("seed", range(10))
def test_kernel_rows_are_a_saturated_basis(seed):
    rng = random.Random(100 + seed)
    n, m = rng.randint(3, 6), rng.randint(1, 3)
    A = _random_int_matrix(rng, n, m)
    s = BinomialStructure(A)
    d = s.dim
    # P_0 A = 0 (Eq. rank-decomp)
    for row in s.P0:
        assert all(sum(row[i] * A[i][j] for i in range(n)) == 0 for j in range(m))
    # saturated: the d x d minors of P_0 have gcd 1 (it extends to a unimodular matrix)
    if d:
        assert _gcd_of_minors(s.P0, d) == 1


def test_consistency_check():
    # x = 2 and x = 3 : rank 1 < m = 2, inconsistent (Eq. consistency)
    A = [[1, 1]]
    coef_bad = [((1, 1), (-2, 1)), ((1, 1), (-3, 1))]   # x - 2 = 0, x - 3 = 0
    coef_ok = [((1, 1), (-2, 1)), ((1, 2), (-1, 1))]    # x - 2 = 0, x/2 - 1 = 0
    assert not BinomialStructure(A, coef_bad).consistent
    assert BinomialStructure(A, coef_ok).consistent
    # x^2 = 4 and x = -2 : consistent;  x^2 = 4 and x = 3 : not
    A2 = [[2, 1]]
    assert BinomialStructure(A2, [((1, 1), (-4, 1)), ((1, 1), (2, 1))]).consistent
    assert not BinomialStructure(A2, [((1, 1), (-4, 1)), ((1, 1), (-3, 1))]).consistent
