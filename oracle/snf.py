"""Smith Normal Form with transforms, by Bezout 2x2 reductions (Sec. 3).

Test infrastructure only (see oracle/__init__.py).

Sec. 3 builds the form from unimodular 2x2 row operations
    [[s, t], [-a2/g, a1/g]]   with  g = gcd(a1, a2) = s*a1 + t*a2,
which send a column (a1, a2) to (g, 0), the same construction transposed for
columns, and row/column permutations.  Repeating them gives P A Q = diag(d_1..d_r, 0..)
(Eq. smith) with P, Q unimodular; the divisibility chain d_1 | d_2 | ... is not
needed (Sec. 3 says so) because only |prod d_j| and the rank are used.
"""

from __future__ import annotations

from fractions import Fraction
from typing import List, Optional, Sequence, Tuple

Matrix = List[List[int]]


def _identity(n: int) -> Matrix:
    return [[int(i == j) for j in range(n)] for i in range(n)]


def _xgcd(a: int, b: int) -> Tuple[int, int, int]:
    """(g, s, t) with g = s*a + t*b = gcd(a, b) >= 0 (extended Euclid)."""
    old_r, r = a, b
    old_s, s = 1, 0
    old_t, t = 0, 1
    while r != 0:
        q = old_r // r
        old_r, r = r, old_r - q * r
        old_s, s = s, old_s - q * s
        old_t, t = t, old_t - q * t
    if old_r < 0:
        old_r, old_s, old_t = -old_r, -old_s, -old_t
    return old_r, old_s, old_t


def _bezout(a1: int, a2: int) -> Tuple[int, int, int, int]:
    """Entries (s, t, u, v) of the unimodular 2x2 [[s, t], [u, v]] = [[s, t], [-a2/g, a1/g]]
    of Sec. 3.  When a1 already divides a2 the plain elimination [[1, 0], [-a2/a1, 1]]
    is used (g = a1), so the pivot is left in place; otherwise |g| < |a1| strictly,
    which makes the alternating row/column clearing terminate."""
    if a2 % a1 == 0:
        return 1, 0, -(a2 // a1), 1
    g, s, t = _xgcd(a1, a2)
    return s, t, -a2 // g, a1 // g


def _row_bezout(M: Matrix, P: Matrix, i: int, j: int, col: int) -> None:
    """Rows (i, j) <- [[s, t], [-a2/g, a1/g]] (rows i, j) so that M[j][col] becomes 0."""
    s, t, u, v = _bezout(M[i][col], M[j][col])
    for X in (M, P):
        ri, rj = X[i], X[j]
        X[i] = [s * x + t * y for x, y in zip(ri, rj)]
        X[j] = [u * x + v * y for x, y in zip(ri, rj)]


def _col_bezout(M: Matrix, Q: Matrix, i: int, j: int, row: int) -> None:
    """Columns (i, j) <- (col i, col j) [[s, -a2/g], [t, a1/g]] so that M[row][j] becomes 0."""
    s, t, u, v = _bezout(M[row][i], M[row][j])
    for X in (M, Q):
        for r in X:
            x, y = r[i], r[j]
            r[i] = s * x + t * y
            r[j] = u * x + v * y


def smith_normal_form(A: Sequence[Sequence[int]]) -> Tuple[Matrix, Matrix, Matrix, int]:
    """Return (P, D, Q, r) with P*A*Q = D diagonal (nonzero d_1..d_r first), P, Q unimodular."""
    n = len(A)
    m = len(A[0]) if n else 0
    M = [[int(x) for x in row] for row in A]
    P = _identity(n)
    Q = _identity(m)
    r = 0
    while r < min(n, m):
        # pivot: an entry of smallest nonzero magnitude in the trailing block
        best = None
        for i in range(r, n):
            for j in range(r, m):
                if M[i][j] != 0 and (best is None or abs(M[i][j]) < abs(M[best[0]][best[1]])):
                    best = (i, j)
        if best is None:
            break
        bi, bj = best
        if bi != r:
            M[r], M[bi] = M[bi], M[r]
            P[r], P[bi] = P[bi], P[r]
        if bj != r:
            for X in (M, Q):
                for row in X:
                    row[r], row[bj] = row[bj], row[r]
        # clear column r below and row r to the right until both are zero
        while True:
            dirty = False
            for i in range(r + 1, n):
                if M[i][r] != 0:
                    _row_bezout(M, P, r, i, r)
                    dirty = True
            for j in range(r + 1, m):
                if M[r][j] != 0:
                    _col_bezout(M, Q, r, j, r)
                    dirty = True
            if not dirty:
                break
        r += 1
    return P, M, Q, r


def matmul(X: Matrix, Y: Matrix) -> Matrix:
    return [[sum(X[i][t] * Y[t][j] for t in range(len(Y))) for j in range(len(Y[0]))]
            for i in range(len(X))]


def det_fraction(M: Sequence[Sequence[int]]) -> int:
    """Determinant by Gaussian elimination over the rationals (textbook, exact)."""
    n = len(M)
    if n == 0:
        return 1
    a = [[Fraction(x) for x in row] for row in M]
    det = Fraction(1)
    for c in range(n):
        p = next((r for r in range(c, n) if a[r][c] != 0), None)
        if p is None:
            return 0
        if p != c:
            a[c], a[p] = a[p], a[c]
            det = -det
        det *= a[c][c]
        for r in range(c + 1, n):
            f = a[r][c] / a[c][c]
            if f:
                a[r] = [x - f * y for x, y in zip(a[r], a[c])]
    assert det.denominator == 1
    return int(det)


class BinomialStructure:
    """Structure of V(x^A - b) from the Smith form (Props. 1, 2, 4)."""

    def __init__(self, A: Sequence[Sequence[int]], coef=None):
        A = [[int(x) for x in row] for row in A]
        self.n = len(A)
        self.m = len(A[0]) if self.n else 0
        if self.m == 0:
            self.P, self.D, self.Q, self.rank = _identity(self.n), [[] for _ in range(self.n)], [], 0
        else:
            self.P, self.D, self.Q, self.rank = smith_normal_form(A)
        r = self.rank
        self.d = [self.D[j][j] for j in range(r)]
        # Prop. 1: number of components |prod d_j|
        t = 1
        for x in self.d:
            t *= x
        self.torsion = abs(t)
        self.dim = self.n - r
        # Eq. rank-decomp: P_0 = rows r..n-1 of P, Q_0 = columns r..m-1 of Q
        self.P0 = [row[:] for row in self.P[r:]]
        self.Q0 = [[row[j] for j in range(r, self.m)] for row in self.Q]
        self.consistent = True if coef is None else self._consistent(coef)

    def _consistent(self, coef) -> bool:
        """Eq. consistency: when r < m the system is solvable iff b^{Q_0} = (1, .., 1),
        with b_i = -c_{i,2}/c_{i,1} (Eq. standard-form)."""
        b = [-Fraction(int(c[1][0]), int(c[1][1])) / Fraction(int(c[0][0]), int(c[0][1]))
             for c in coef]
        for j in range(self.m - self.rank):
            prod = Fraction(1)
            for i in range(self.m):
                e = self.Q0[i][j]
                if e:
                    prod *= b[i] ** e
            if prod != 1:
                return False
        return True

    def kernel_points(self) -> List[Tuple[int, ...]]:
        """Columns of P_0 as points of Z^d, d = n - r (Prop. 4)."""
        return [tuple(self.P0[i][j] for i in range(self.dim)) for j in range(self.n)]
