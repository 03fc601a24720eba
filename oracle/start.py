"""Solutions of the per-cell start systems of the witness-set homotopy (Sec. 6).

Test infrastructure only (see oracle/__init__.py).

For a cell {a_0, .., a_k} of the lifting's triangulation (point indices q_0 < .. < q_k) and the
k x (k+1) coefficient matrix C of the cell's points, the start system (Eq. affine-cut-starting)
is C (y^{a_0}, .., y^{a_k})^T = 0.  For generic C its null space is one line, spanned by kappa
with kappa_j = (-1)^j det(C without column j), so y^{a_j} = lambda kappa_j and the system is the
binomial system y^{a_j - a_k} = kappa_j / kappa_k, j < k (Eq. affine-cut-eliminated).  It is
solved by Sec. 3's method: with the Smith form P E Q = D of the exponent matrix E (rows
a_j - a_k), w = Q^-1 log y satisfies d_i w_i = (P log b)_i + 2 pi i r_i, r_i = 0 .. |d_i| - 1,
and y = exp(Q w): |det E| solutions, the cell's normalized volume.  Written as
log y = E^-1 log b + 2 pi i Q (r / d), the first term uses the exact rational E^-1 and the
second is an exact fraction of a turn per coordinate (reduced mod 1 before any rounding), so
large transform entries cost no precision.

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
from fractions import Fraction
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


def _inverse(E):
    """Exact inverse over Q (Gauss-Jordan with Fractions)."""
    k = len(E)
    a = [[Fraction(x) for x in row] + [Fraction(int(i == j)) for j in range(k)] for i, row in enumerate(E)]
    for c in range(k):
        p = next(r for r in range(c, k) if a[r][c] != 0)
        a[c], a[p] = a[p], a[c]
        piv = a[c][c]
        a[c] = [x / piv for x in a[c]]
        for r in range(k):
            if r != c and a[r][c] != 0:
                f = a[r][c]
                a[r] = [x - f * y for x, y in zip(a[r], a[c])]
    return [row[k:] for row in a]


def solve_binomial(E: Sequence[Sequence[int]], b: Sequence[complex]) -> List[List[complex]]:
    """All solutions y in (C*)^k of prod_i y_i^E[j][i] = b_j (Sec. 3, via the Smith form)."""
    k = len(E)
    P, D, Q, r = smith_normal_form(E)
    if r < k:
        raise ValueError("singular exponent matrix")
    Einv = _inverse(E)
    logb = [cmath.log(x) for x in b]
    base = [complex(math.fsum(float(Einv[i][j]) * logb[j].real for j in range(k)),
                    math.fsum(float(Einv[i][j]) * logb[j].imag for j in range(k))) for i in range(k)]
    d = [D[i][i] for i in range(k)]
    L = 1
    for x in d:
        L = L * abs(x) // math.gcd(L, abs(x))
    # turns_i = (Q (r / d))_i mod 1 = (sum_j Q_ij r_j L / d_j mod L) / L, in integers
    w = [[Q[i][j] * (L // d[j]) for j in range(k)] for i in range(k)]
    out = []
    for rr in product(*[range(abs(x)) for x in d]):
        turns = [(sum(w[i][j] * rr[j] for j in range(k)) % L) / L for i in range(k)]
        out.append([cmath.exp(base[i] + 2j * math.pi * turns[i]) for i in range(k)])
    return out


def start_solutions(points, cells, coef_seed: int):
    """The start solutions of every cell, cells in the given order."""
    res = []
    for cell in cells:
        E, b = cell_binomial(points, cell, coef_seed)
        res.append(solve_binomial(E, b))
    return res
