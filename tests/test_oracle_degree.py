"""Pins for the oracle's degree (Props. 1, 2, 4) against closed forms and the paper's
master-space tables (Sec. 6, Tables mspace-dim and mspace-deg)."""

import json
import os

import pytest

from oracle.degree import degree
from oracle.snf import BinomialStructure
from workloads import master_space_system

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "master_space_table.json")))


def test_parabola():
    # y - x^2 = 0 (Sec. 2): column alpha - beta = (0,1) - (2,0); degree 2
    r = degree([[-2], [1]])
    assert (r.degree, r.dim, r.torsion) == (2, 1, 1)


def test_hyperbola_line_and_cubic():
    assert degree([[1], [1]]).degree == 2            # x y = 1
    assert degree([[1], [-1]]).degree == 1           # x = y
    # twisted cubic y = x^2, z = x^3 : degree 3
    assert degree([[-2, -3], [1, 0], [0, 1]]).degree == 3


def test_no_equations_is_the_torus():
    # A with no columns: the whole (C*)^n, degree 1 (standard simplex)
    r = degree([[] for _ in range(3)])
    assert (r.degree, r.dim, r.nvol) == (1, 3, 1)


def test_isolated_points_count_torsion():
    # x^2 = c : rank n, d = 0, |prod d_j| = 2 isolated points (Prop. 1)
    r = degree([[2]])
    assert (r.degree, r.dim, r.torsion) == (2, 0, 2)
    # x^2 y^3 = 1, x y^2 = 1 : det = 1 -> one point
    assert degree([[2, 1], [3, 2]]).degree == 1
    # x^2 = 1, y^3 = 1 : 6 points
    assert degree([[2, 0], [0, 3]]).degree == 6


def test_torsion_times_volume():
    # x^2 y^2 = 1 : d_1 = 2 (two components x y = +-1), each of degree 2
    r = degree([[2], [2]])
    assert (r.torsion, r.nvol, r.degree) == (2, 2, 4)


def test_inconsistent_system_has_degree_zero():
    r = degree([[1, 1]], [((1, 1), (-2, 1)), ((1, 1), (-3, 1))])
    assert (r.degree, r.consistent) == (0, False)


def test_pyramid_and_placing_agree_on_degree():
    for m, k in [(1, 2), (1, 3), (2, 1), (2, 2)]:
        s = master_space_system(m, k)
        assert degree(s.A.tolist(), s.coef.tolist(), method="pyramid").degree == \
            degree(s.A.tolist(), s.coef.tolist()).degree


FAST = ["1,2", "1,3", "1,4", "1,5", "1,6", "1,7", "1,8", "2,1", "2,2", "2,3", "2,4", "3,1", "3,2", "4,1", "4,2"]


@pytest.mark.parametrize("mk", FAST)
def test_master_space_table(mk):
    m, k = map(int, mk.split(","))
    s = master_space_system(m, k)
    r = degree(s.A.tolist(), s.coef.tolist())
    assert r.consistent
    assert r.degree == GOLDEN["degree"][mk]
    if mk in GOLDEN["dimension"]:
        assert r.dim == GOLDEN["dimension"][mk]


@pytest.mark.slow
@pytest.mark.parametrize("mk", ["3,3", "2,5"])
def test_master_space_table_larger(mk):
    m, k = map(int, mk.split(","))
    s = master_space_system(m, k)
    r = degree(s.A.tolist(), s.coef.tolist())
    assert r.degree == GOLDEN["degree"][mk]
    assert r.dim == GOLDEN["dimension"][mk]


def test_master_space_dimension_formula():
    # Table mspace-dim: dim = mk + 2 for every listed (m, k) other than (1, 1)
    for mk, dim in GOLDEN["dimension"].items():
        m, k = map(int, mk.split(","))
        assert dim == m * k + 2
        if m * k <= 6:
            assert BinomialStructure(master_space_system(m, k).A.tolist()).dim == dim
