"""The cells of the regular triangulation induced by a lifting, each with its inner normal.

Test infrastructure only (see oracle/__init__.py).

Sec. 6 (the witness-set construction, Eq. lower-d-face-again): every cell {a_0, .., a_k} of the
regular subdivision is the projection of a lower facet of the lifted point set, with a unique
inner normal alpha^ = (alpha, 1) such that <a^_j, alpha^> = beta for the cell's points and
<a^, alpha^> > beta for every other point; (alpha, beta) also define the change of variables
t_i = y_i s^alpha_i and the shift s^-beta of the homotopy H^{alpha,beta}.  Here (alpha, beta)
are exact rationals from the k+1 equalities, and the cells are found by testing every
(k+1)-subset (tiny inputs only).
"""

from __future__ import annotations

from fractions import Fraction
from itertools import combinations
from typing import List, Sequence, Tuple

from .lower_facet import ACCEPTED, _solve, lower_facet_status


def cell_normal(points: Sequence[Sequence[int]], lifts: Sequence[int],
                subset: Sequence[int]) -> Tuple[List[Fraction], Fraction]:
    """(alpha, beta) with <a_j, alpha> + omega(a_j) = beta for the cell's points (Sec. 6)."""
    k = len(points[0])
    M = [[int(x) for x in points[i]] + [-1] for i in subset]
    sol = _solve(M, [-int(lifts[i]) for i in subset])
    if sol is None:
        raise ValueError("the subset is not full-dimensional")
    return sol[:k], sol[k]


def lower_cells(points: Sequence[Sequence[int]], lifts: Sequence[int]):
    """Every accepted cell as (subset, |det|, alpha, beta), subsets in lexicographic order."""
    k = len(points[0])
    out = []
    for sub in combinations(range(len(points)), k + 1):
        st, vol = lower_facet_status(points, lifts, sub)
        if st == ACCEPTED:
            alpha, beta = cell_normal(points, lifts, sub)
            out.append((sub, vol, alpha, beta))
    return out
