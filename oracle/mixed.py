"""Mixed volume MV(conv A_1, .., conv A_k) of k lattice point sets in Z^k.

Test infrastructure only (see oracle/__init__.py).

Appendix A (Kushnirenko's theorem) notes that the degree computed by the method is the
special case of the BKK bound (Bernstein's theorem) in which every equation has the same
support: the number of isolated C*-solutions of a generic system with supports A_1..A_k
is the mixed volume of their convex hulls, and MV(P, .., P) = k! Vol_k(P) = NVol_k(P).
Sec. 4's remark on earlier work places the degree problem inside mixed cell enumeration
(Huber-Sturmfels 1995), which computes MV from a random lifting.  This module states MV
twice, by two unrelated routes:

* `mixed_volume_polarization`: the definition.  Vol_k(l_1 P_1 + .. + l_k P_k) is a
  homogeneous polynomial of degree k in l_1..l_k >= 0 and MV is the coefficient of
  l_1 l_2 .. l_k; inclusion-exclusion over the subsets S of {1..k} isolates it:
      MV = sum_{S != {}} (-1)^(k - |S|) Vol_k(sum_{i in S} P_i),
  normalised so that MV(P, .., P) = k! Vol_k(P).  With NVol = k! Vol this reads
      MV = sum_S (-1)^(k - |S|) NVol_k(sum_{i in S} P_i) / k!.
  The Minkowski sums are formed point by point and their volumes taken by the
  placing triangulation of `volume.py`.

* `mixed_cells` / `mixed_volume_lifting`: the lifting method step by step.  Every point
  a of A_i gets a height w_i(a).  A tuple of pairs C = ({a_1, a_1'}, .., {a_k, a_k'}),
  C_i a 2-subset of A_i, is a fine mixed cell iff the k x k matrix M with rows
  a_i' - a_i is nonsingular and the unique alpha with
      <a_i' - a_i, alpha> = -(w_i(a_i') - w_i(a_i))          (i = 1..k)
  makes <a, alpha> + w_i(a) minimal over A_i exactly on C_i:
      <b - a_i, alpha> + w_i(b) - w_i(a_i) > 0  for every b in A_i outside C_i.
  Then MV = sum over the fine mixed cells of |det M|.  As in `lower_facet.py`, a tuple
  with no point below and one point on its plane is a tie (the lifting is not generic),
  answered by another lifting.

The lifts of the concatenated points (component 1's points first, then component 2's,
...) are the ones `lifts.py` gives for the total count, so that both sides of a test
see the same heights.
"""

from __future__ import annotations

from fractions import Fraction
from itertools import combinations, product
from math import factorial
from typing import List, Sequence, Tuple

from .lower_facet import _solve
from .volume import affine_rank, det_int, nvol_placing

SINGULAR, REJECTED, ACCEPTED, TIE = "singular", "rejected", "accepted", "tie"


def minkowski_sum(sets: Sequence[Sequence[Sequence[int]]]) -> List[Tuple[int, ...]]:
    """All sums a_1 + .. + a_r (a_i in sets[i]), without repeats."""
    out = {tuple(0 for _ in sets[0][0])}
    for A in sets:
        out = {tuple(x + y for x, y in zip(s, a)) for s in out for a in A}
    return sorted(out)


def nvol_any(points: Sequence[Sequence[int]]) -> int:
    """NVol_k(conv points), 0 when the points do not span Z^k affinely."""
    pts = [tuple(int(x) for x in p) for p in points]
    k = len(pts[0])
    if affine_rank(pts) < k:
        return 0
    return nvol_placing(pts)


def mixed_volume_polarization(supports: Sequence[Sequence[Sequence[int]]]) -> int:
    """MV by the inclusion-exclusion (polarization) formula over Minkowski sums."""
    k = len(supports)
    assert all(len(p) == k for A in supports for p in A), "k point sets in Z^k"
    total = 0
    for r in range(1, k + 1):
        for S in combinations(range(k), r):
            total += (-1) ** (k - r) * nvol_any(minkowski_sum([supports[i] for i in S]))
    assert total % factorial(k) == 0
    return total // factorial(k)


def split_lifts(supports, lifts):
    """The flat list of heights cut into one list per component."""
    out, at = [], 0
    for A in supports:
        out.append([int(w) for w in lifts[at:at + len(A)]])
        at += len(A)
    assert at == len(lifts)
    return out


def cell_status(supports, lifts, pairs) -> Tuple[str, int]:
    """(status, |det M|) of the tuple of pairs `pairs` (pairs[i] = (p, q), indices into
    supports[i]) under the flat heights `lifts`."""
    k = len(supports)
    W = split_lifts(supports, lifts)
    A = [[tuple(int(x) for x in p) for p in S] for S in supports]
    M = [[x - y for x, y in zip(A[i][q], A[i][p])] for i, (p, q) in enumerate(pairs)]
    rhs = [-(W[i][q] - W[i][p]) for i, (p, q) in enumerate(pairs)]
    alpha = _solve(M, rhs)
    if alpha is None:
        return SINGULAR, 0
    below = on = False
    for i, (p, q) in enumerate(pairs):
        for b in range(len(A[i])):
            if b in (p, q):
                continue
            val = sum(Fraction(x - y) * a for x, y, a in zip(A[i][b], A[i][p], alpha)) + W[i][b] - W[i][p]
            if val < 0:
                below = True
                break
            if val == 0:
                on = True
        if below:
            break
    vol = abs(det_int(M))
    if below:
        return REJECTED, vol
    if on:
        return TIE, vol
    return ACCEPTED, vol


def mixed_cells(supports, lifts):
    """Every tuple of pairs, classified.  Returns (cells, n_singular, n_ties) with
    cells = [(pairs, |det M|), ..] in the lexicographic order of the tuples
    (component 1's pair most significant, pairs (p, q) with p < q in lexicographic order)."""
    cells, sing, ties = [], 0, 0
    for pairs in product(*[list(combinations(range(len(A)), 2)) for A in supports]):
        st, v = cell_status(supports, lifts, pairs)
        if st == ACCEPTED:
            cells.append((pairs, v))
        elif st == SINGULAR:
            sing += 1
        elif st == TIE:
            ties += 1
    return cells, sing, ties


def mixed_volume_lifting(supports, lifts):
    """(MV, fine mixed cells, singular tuples, ties) by the lifting method."""
    cells, sing, ties = mixed_cells(supports, lifts)
    return sum(v for _, v in cells), len(cells), sing, ties
