"""The lower-facet test of one lifted (k+1)-subset, written as Eq. lower-face.

Test infrastructure only (see oracle/__init__.py).

Sec. 4: with lifted points a^ = (a, omega(a)), the subset {a_0..a_k} spans a lower
k-face iff some inner normal alpha^ = (alpha, 1) gives
    <a^_0, alpha^> = <a^_j, alpha^>   (j = 1..k)      and
    <a^_0, alpha^> <= <a^, alpha^>    (all a in S),
and Sec. 5 (Eq. lower-d-face-again) states the cell condition with strict '<' for
the points outside the cell.  Reading used: strict inequality for every point of
S outside the subset; a point with equality (and none below) is a tie, which the
method answers by re-lifting.  With alpha^ = (alpha, 1) the k+1 equalities are the
square linear system  <a_j, alpha> - beta = -omega(a_j)  (j = 0..k)  for the unknowns
(alpha, beta), beta = <a^_0, alpha^>; it is solvable iff the subset is affinely
independent, i.e. the cell is full-dimensional.  The cell's normalized volume is
|det(a_1 - a_0, .., a_k - a_0)| (Eq. simplex-vol).
"""

from __future__ import annotations

from fractions import Fraction
from itertools import combinations
from typing import Sequence, Tuple

from .volume import det_int

SINGULAR, REJECTED, ACCEPTED, TIE = "singular", "rejected", "accepted", "tie"


def _solve(M, rhs):
    """Gaussian elimination over Q; None if singular."""
    n = len(M)
    a = [[Fraction(x) for x in row] + [Fraction(b)] for row, b in zip(M, rhs)]
    for c in range(n):
        p = next((r for r in range(c, n) if a[r][c] != 0), None)
        if p is None:
            return None
        a[c], a[p] = a[p], a[c]
        for r in range(n):
            if r != c and a[r][c] != 0:
                f = a[r][c] / a[c][c]
                a[r] = [x - f * y for x, y in zip(a[r], a[c])]
    return [a[i][n] / a[i][i] for i in range(n)]


def lower_facet_status(points: Sequence[Sequence[int]], lifts: Sequence[int],
                       subset: Sequence[int]) -> Tuple[str, int]:
    """(status, |det|) of the cell `subset` (k+1 indices into `points`)."""
    k = len(points[0])
    sub = list(subset)
    assert len(sub) == k + 1
    M = [[int(x) for x in points[i]] + [-1] for i in sub]
    sol = _solve(M, [-int(lifts[i]) for i in sub])
    if sol is None:
        return SINGULAR, 0
    alpha, beta = sol[:k], sol[k]
    below = on = False
    members = set(sub)
    for q in range(len(points)):
        if q in members:
            continue
        val = sum(Fraction(int(x)) * a for x, a in zip(points[q], alpha)) + int(lifts[q]) - beta
        if val < 0:
            below = True
            break
        if val == 0:
            on = True
    vol = abs(det_int([[int(x) - int(y) for x, y in zip(points[i], points[sub[0]])] for i in sub[1:]]))
    if below:
        return REJECTED, vol
    if on:
        return TIE, vol
    return ACCEPTED, vol


def nvol_lifting_bruteforce(points: Sequence[Sequence[int]], lifts: Sequence[int]):
    """Sum of |det| over all accepted cells (tiny inputs only).
    Returns (nvol, n_accepted, n_singular, n_ties)."""
    k = len(points[0])
    total = acc = sing = ties = 0
    for sub in combinations(range(len(points)), k + 1):
        st, v = lower_facet_status(points, lifts, sub)
        if st == ACCEPTED:
            total += v
            acc += 1
        elif st == SINGULAR:
            sing += 1
        elif st == TIE:
            ties += 1
    return total, acc, sing, ties
