"""Pins for oracle/cells.py: a worked example by hand, the defining equalities and strict
inequalities of every inner normal, and the cells' volumes summing to the volume."""

import random
from fractions import Fraction

from oracle.cells import cell_normal, lower_cells
from oracle.lifts import lifts as oracle_lifts
from oracle.volume import nvol_placing


def test_unit_square_by_hand():
    # lifts 0, 0, 0, 1 on (0,0), (1,0), (0,1), (1,1): the lower hull is the flat triangle at
    # height 0 (alpha = 0, beta = 0) and the triangle through (1,0,0), (0,1,0), (1,1,1), the
    # plane omega = x + y - 1, so alpha = (-1, -1) and beta = -1
    pts = [(0, 0), (1, 0), (0, 1), (1, 1)]
    cells = lower_cells(pts, [0, 0, 0, 1])
    assert [c[0] for c in cells] == [(0, 1, 2), (1, 2, 3)]
    assert cells[0][2:] == ([0, 0], 0)
    assert cells[1][2:] == ([-1, -1], -1)
    assert all(c[1] == 1 for c in cells)


def test_normals_satisfy_the_facet_conditions():
    rng = random.Random(5)
    for trial in range(12):
        k = rng.choice([2, 3])
        n = rng.randint(k + 2, 8)
        pts = [tuple(rng.randint(-3, 3) for _ in range(k)) for _ in range(n)]
        lf = oracle_lifts(n, trial)
        cells = lower_cells(pts, lf)
        assert sum(c[1] for c in cells) == nvol_placing(pts)
        for sub, vol, alpha, beta in cells:
            for q in range(n):
                h = sum(Fraction(x) * a for x, a in zip(pts[q], alpha)) + lf[q]
                if q in sub:
                    assert h == beta
                else:
                    assert h > beta


def test_cell_normal_rejects_flat_subsets():
    try:
        cell_normal([(0, 0), (1, 1), (2, 2)], [1, 2, 3], (0, 1, 2))
    except ValueError:
        return
    assert False
