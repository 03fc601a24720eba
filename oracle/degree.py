"""Degree of the C*-solution set of x^A = b (Props. 1, 2, 4).

Test infrastructure only (see oracle/__init__.py).

* Prop. 2 / Eq. consistency: when rank A < m the system has solutions iff
  b^{Q_0} = 1; otherwise the solution set is empty and the degree is 0.
* Prop. 1: V consists of |prod d_j| components, each of dimension d = n - rank A.
* Prop. 4 (Eq. deg-vol): each component has degree d! Vol_d(conv{p_0^(1)..p_0^(n), 0})
  where p_0^(j) are the columns of P_0.  The origin belongs to the point set.
* Reading used for "degree of the solution set": the components are disjoint and
  share the same monomial parametrization (Prop. 2), so the total degree is
  |prod d_j| * NVol.  When d = 0 every component is a point and the degree is the
  number of points, |prod d_j|.
"""

from __future__ import annotations

from dataclasses import dataclass

from .snf import BinomialStructure
from .volume import nvol_placing, nvol_pyramid


@dataclass
class DegreeResult:
    degree: int
    nvol: int
    torsion: int
    rank: int
    dim: int
    consistent: bool


def degree(A, coef=None, method: str = "placing") -> DegreeResult:
    s = BinomialStructure(A, coef)
    if not s.consistent:
        return DegreeResult(0, 0, s.torsion, s.rank, s.dim, False)
    if s.dim == 0:
        return DegreeResult(s.torsion, 1, s.torsion, s.rank, 0, True)
    pts = s.kernel_points() + [tuple([0] * s.dim)]
    nv = nvol_pyramid(pts) if method == "pyramid" else nvol_placing(pts)
    return DegreeResult(s.torsion * nv, nv, s.torsion, s.rank, s.dim, True)
