"""Solutions of the per-cell start systems of the witness-set homotopy (Sec. 6).

Test infrastructure only (see oracle/__init__.py).

For a cell {a_0, .., a_k} of the lifting's triangulation (point indices q_0 < .. < q_k) and the
k x (k+1) coefficient matrix C of the cell's points, the start system (Eq. affine-cut-starting)
is C (y^{a_0}, .., y^{a_k})^T = 0.  For generic C its null space is one line, spanned by kappa
with kappa_j = (-1)^j det(C without column j), so y^{a_j} = lambda kappa_j and the system is the
binomial system y^{a_j - a_k} = kappa_j / kappa_k, j < k (Eq. affine-cut-eliminated).  It is
solved by Sec. 3's method: with the Smith form P E Q = D of the exponent matrix E (rows
a_j - a_k), w = Q^-1 log y satisfies d_i w_i = (P log b)_i + 2 pi i r_i, r_i = 0 .. |d_i| - 1,
and y = exp(Q w): |det E| solutions, the cell's normalized volume.

Generic coefficients (reading: the paper only asks for generic complex coefficients): unit
complex numbers c_{i,q} = exp(2 pi i u) with u from SplitMix64 (the generator of
oracle/lifts.py, on its own stream):
    s = mix(coef_seed XOR 0xC2B2AE3D27D4EB4F),
    u(i, q) = (mix(s + (i N + q + 1) * 0x9E3779B97F4A7C15) >> 11) / 2^53,
for equation i < k and point q < N.  numpy's determinant and complex exp are the library
steps; everything else is written out.
"""

from __future__ import annotations

import cmath
import math
from itertools import product
from typing import List, Sequence

import numpy as np

from .lifts import GOLDEN, MASK, mix
from .snf import smith_normal_form

COEF_XOR = 0xC2B2AE3D27D4EB4F


def coefficient(coef_seed: int, npts: int, i: int, q: int) -> complex:
    s = mix((coef_seed ^ COEF_XOR) & MASK)
    u = (mix((s + (i * npts + q + 1) * GOLDEN) & MASK) >> 11) / float(1 << 53)
    return cmath.exp(2j * math.pi * u)


def cell_binomial(points: Sequence[Sequence[int]], cell: Sequence[int], coef_seed: int):
    """(E, b): the binomial system y^E = b of one cell (rows of E: a_j - a_k)."""
    k = len(points[0])
    n = len(points)
    C = np.array([[coefficient(coef_seed, n, i, q) for q in cell] for i in range(k)], dtype=complex)
    kappa = [(-1) ** j * np.linalg.det(np.delete(C, j, axis=1)) for j in range(k + 1)]
    E = [[int(points[cell[j]][c]) - int(points[cell[k]][c]) for c in range(k)] for j in range(k)]
    b = [kappa[j] / kappa[k] for j in range(k)]
    return E, b


def solve_binomial(E: Sequence[Sequence[int]], b: Sequence[complex]) -> List[List[complex]]:
    """All solutions y in (C*)^k of prod_i y_i^E[j][i] = b_j (Sec. 3, via the Smith form)."""
    k = len(E)
    P, D, Q, r = smith_normal_form(E)
    if r < k:
        raise ValueError("singular exponent matrix")
    logb = [cmath.log(x) for x in b]
    Plogb = [sum(P[i][j] * logb[j] for j in range(k)) for i in range(k)]
    d = [D[i][i] for i in range(k)]
    out = []
    for rr in product(*[range(abs(x)) for x in d]):
        w = [(Plogb[i] + 2j * math.pi * rr[i]) / d[i] for i in range(k)]
        x = [sum(Q[i][j] * w[j] for j in range(k)) for i in range(k)]
        out.append([cmath.exp(v) for v in x])
    return out


def start_solutions(points, cells, coef_seed: int):
    """The start solutions of every cell, cells in the given order."""
    res = []
    for cell in cells:
        E, b = cell_binomial(points, cell, coef_seed)
        res.append(solve_binomial(E, b))
    return res
