"""Exact normalized volume NVol_k(conv S) = k! * Vol_k(conv S)  (Sec. 4, Eq. deg-nvol).

Test infrastructure only (see oracle/__init__.py).

The degree method reaches NVol through a regular triangulation built by lifting
(Sec. 4.1-4.5).  The oracle does not lift: it computes the volume of the convex hull
by two other exact algorithms, each checkable by eye:

* `nvol_pyramid`: the cone (pyramid) decomposition over the facets of conv S,
      Vol_k(P) = sum_F (1/k) * dist(v, aff F) * Vol_{k-1}(F)        (v a vertex),
  with the facets found by brute force over k-subsets (a facet is a hyperplane
  through k affinely independent points with all of S on one side).  For an
  integer facet normal u with offset c and a coordinate j with u_j != 0, projecting
  F along e_j scales (k-1)-volume by |u_j| / |u|, which gives, in normalized units,
      NVol_k(pyramid(F, v)) = |<u, v> - c| / |u_j| * NVol_{k-1}(proj_j F).
  Exponential in |S|; used for small inputs.

* `nvol_placing`: the placing (beneath-beyond) triangulation: start from k+1
  affinely independent points; each further point p is joined to every boundary
  simplex of the current hull that p sees strictly from outside.  The added simplices
  cover conv(hull + p) minus the hull, so NVol = sum of |det| over all simplices
  (Eq. simplex-vol read as |det(a_1 - a_0, .., a_k - a_0)|).  Fast enough for the
  master-space pins and the mid-size single systems.
"""

from __future__ import annotations

from collections import Counter
from fractions import Fraction
from itertools import combinations
from typing import Dict, FrozenSet, List, Sequence, Tuple

Point = Tuple[int, ...]


def det_int(rows: Sequence[Sequence[int]]) -> int:
    """Exact integer determinant (fraction-free Gaussian elimination with row swaps)."""
    n = len(rows)
    if n == 0:
        return 1
    a = [list(map(int, r)) for r in rows]
    sign = 1
    prev = 1
    for c in range(n - 1):
        p = next((r for r in range(c, n) if a[r][c] != 0), None)
        if p is None:
            return 0
        if p != c:
            a[c], a[p] = a[p], a[c]
            sign = -sign
        for r in range(c + 1, n):
            for j in range(c + 1, n):
                a[r][j] = (a[r][j] * a[c][c] - a[r][c] * a[c][j]) // prev
            a[r][c] = 0
        prev = a[c][c]
    return sign * a[n - 1][n - 1]


def affine_rank(points: Sequence[Point]) -> int:
    """Dimension of the affine hull (rank of the differences over Q)."""
    if not points:
        return -1
    p0 = points[0]
    rows = [[Fraction(x - y) for x, y in zip(p, p0)] for p in points[1:]]
    rank = 0
    ncol = len(p0)
    for c in range(ncol):
        piv = next((r for r in range(rank, len(rows)) if rows[r][c] != 0), None)
        if piv is None:
            continue
        rows[rank], rows[piv] = rows[piv], rows[rank]
        for r in range(len(rows)):
            if r != rank and rows[r][c] != 0:
                f = rows[r][c] / rows[rank][c]
                rows[r] = [x - f * y for x, y in zip(rows[r], rows[rank])]
        rank += 1
    return rank


def hyperplane_normal(pts: Sequence[Point]) -> Tuple[int, ...]:
    """Integer normal u of the hyperplane through k points of Z^k (generalized cross
    product of the k-1 differences: u_i = (-1)^i det(differences without column i)).
    Returns the zero vector when the points are affinely dependent."""
    k = len(pts[0])
    diffs = [[x - y for x, y in zip(p, pts[0])] for p in pts[1:]]
    return tuple((-1) ** i * det_int([row[:i] + row[i + 1:] for row in diffs]) for i in range(k))


def _primitive(u: Sequence[int]) -> Tuple[int, ...]:
    from math import gcd
    g = 0
    for x in u:
        g = gcd(g, x)
    return tuple(x // g for x in u) if g else tuple(u)


def dot(u, v) -> int:
    return sum(int(a) * int(b) for a, b in zip(u, v))


# ----------------------------------------------------------------------------------
# pyramid decomposition
# ----------------------------------------------------------------------------------

def facets_bruteforce(points: Sequence[Point]) -> List[Tuple[Tuple[int, ...], int, Tuple[Point, ...]]]:
    """All facets of conv(points) (full-dimensional in Z^k) as (u, c, points on it):
    u primitive outer normal, u.x <= c on conv(points), equality on the facet."""
    k = len(points[0])
    seen: Dict[Tuple[Tuple[int, ...], int], Tuple[Point, ...]] = {}
    for sub in combinations(points, k):
        u = hyperplane_normal(sub)
        if not any(u):
            continue
        u = _primitive(u)
        c = dot(u, sub[0])
        vals = [dot(u, q) - c for q in points]
        if all(v <= 0 for v in vals):
            pass
        elif all(v >= 0 for v in vals):
            u, c = tuple(-x for x in u), -c
        else:
            continue
        if (u, c) not in seen:
            seen[(u, c)] = tuple(q for q in points if dot(u, q) == c)
    return [(u, c, F) for (u, c), F in seen.items()]


def _nvol_pyramid_rec(points: Tuple[Point, ...]) -> Fraction:
    k = len(points[0])
    if k == 1:
        xs = [p[0] for p in points]
        return Fraction(max(xs) - min(xs))
    v = points[0]
    total = Fraction(0)
    for u, c, F in facets_bruteforce(points):
        h = abs(dot(u, v) - c)
        if h == 0:
            continue  # facets through the apex contribute nothing
        j = next(i for i, x in enumerate(u) if x != 0)
        proj = tuple(sorted(set(p[:j] + p[j + 1:] for p in F)))
        total += Fraction(h, abs(u[j])) * _nvol_pyramid_rec(proj)
    return total


def nvol_pyramid(points: Sequence[Sequence[int]]) -> int:
    """NVol_k(conv points) by facet-enumeration pyramid decomposition; 0 if not full-dimensional."""
    pts = tuple(sorted(set(tuple(int(x) for x in p) for p in points)))
    if not pts:
        return 0
    k = len(pts[0])
    if k == 0:
        return 1
    if affine_rank(pts) < k:
        return 0
    vol = _nvol_pyramid_rec(pts)
    assert vol.denominator == 1, vol
    return int(vol)


# ----------------------------------------------------------------------------------
# placing (beneath-beyond) triangulation
# ----------------------------------------------------------------------------------

def _oriented_facet(face: Tuple[Point, ...], inside: Point):
    """(u, c) of the hyperplane through `face`, oriented so that u.inside < c."""
    u = hyperplane_normal(face)
    c = dot(u, face[0])
    s = dot(u, inside) - c
    assert s != 0, "reference point lies on the facet hyperplane"
    if s > 0:
        u, c = tuple(-x for x in u), -c
    return u, c


def placing_triangulation(points: Sequence[Sequence[int]]):
    """Return the list of full-dimensional simplices (tuples of k+1 points) of the
    placing triangulation of `points` taken in the given order; [] if not full-dimensional."""
    pts = [tuple(int(x) for x in p) for p in points]
    if not pts:
        return []
    k = len(pts[0])
    base: List[Point] = []
    for p in pts:
        if affine_rank(base + [p]) == len(base):
            base.append(p)
            if len(base) == k + 1:
                break
    if len(base) < k + 1:
        return []
    simplices = [tuple(base)]
    boundary: Dict[FrozenSet[Point], Tuple[Tuple[int, ...], int]] = {}
    for i in range(k + 1):
        face = tuple(base[:i] + base[i + 1:])
        boundary[frozenset(face)] = _oriented_facet(face, base[i])
    placed = set(base)
    for p in pts:
        if p in placed:
            continue
        placed.add(p)
        visible = [F for F, (u, c) in boundary.items() if dot(u, p) > c]
        if not visible:
            continue
        ridge_use = Counter()
        ridge_owner = {}
        for F in visible:
            simplices.append(tuple(F) + (p,))
            for w in F:
                R = F - {w}
                ridge_use[R] += 1
                ridge_owner[R] = w
        for F in visible:
            del boundary[F]
        for R, cnt in ridge_use.items():
            if cnt == 1:  # horizon ridge: also on a facet that p does not see
                G = frozenset(R | {p})
                # the far vertex w of the visible facet through R is strictly inside G's side
                boundary[G] = _oriented_facet(tuple(G), ridge_owner[R])
    return simplices


def nvol_placing(points: Sequence[Sequence[int]]) -> int:
    """NVol_k(conv points) as the sum of |det| over a placing triangulation."""
    simplices = placing_triangulation(points)
    total = 0
    for s in simplices:
        total += abs(det_int([[x - y for x, y in zip(q, s[0])] for q in s[1:]]))
    return total
