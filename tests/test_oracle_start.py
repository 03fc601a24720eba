"""Pins for oracle/start.py: solution counts equal the cell volumes, every solution satisfies
the binomial equations and the start system itself, and a 1-D worked example."""

import cmath
import math
import random

import numpy as np

from oracle.cells import lower_cells
from oracle.lifts import lifts as oracle_lifts
from oracle.start import cell_binomial, coefficient, solve_binomial, start_solutions


def test_one_dimensional_roots_of_unity():
    # y^3 = 1: the three cube roots of unity
    sols = solve_binomial([[3]], [1.0 + 0j])
    angles = sorted((cmath.phase(s[0]) % (2 * math.pi)) for s in sols)
    assert np.allclose(angles, [0, 2 * math.pi / 3, 4 * math.pi / 3])
    assert all(abs(abs(s[0]) - 1) < 1e-12 for s in sols)


def test_two_dimensional_count_and_residual():
    E = [[2, 1], [0, 3]]
    b = [0.5 + 0.25j, -1.5 + 0.1j]
    sols = solve_binomial(E, b)
    assert len(sols) == 6
    for y in sols:
        for j in range(2):
            v = y[0] ** E[j][0] * y[1] ** E[j][1]
            assert abs(v / b[j] - 1) < 1e-12
    # distinct
    assert len({(round(y[0].real, 9), round(y[0].imag, 9), round(y[1].real, 9), round(y[1].imag, 9)) for y in sols}) == 6


def test_start_systems_of_a_triangulation():
    rng = random.Random(4)
    for trial in range(6):
        k = rng.choice([2, 3])
        n = rng.randint(k + 2, 7)
        pts = [tuple(rng.randint(-2, 2) for _ in range(k)) for _ in range(n)]
        cells = lower_cells(pts, oracle_lifts(n, trial))
        sols = start_solutions(pts, [c[0] for c in cells], coef_seed=trial)
        for (cell, vol, _, _), ys in zip(cells, sols):
            assert len(ys) == vol
            C = [[coefficient(trial, n, i, q) for q in cell] for i in range(k)]
            for y in ys:
                z = [np.prod([y[c] ** pts[q][c] for c in range(k)]) for q in cell]
                # the start system itself: C z = 0 (relative to the size of the terms)
                for i in range(k):
                    s = sum(C[i][j] * z[j] for j in range(k + 1))
                    assert abs(s) <= 1e-9 * sum(abs(C[i][j] * z[j]) for j in range(k + 1))
