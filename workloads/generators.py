"""Seeded generators of binomial systems, point sets and request arrivals.

A binomial system  c_{i,1} x^{alpha_i} + c_{i,2} x^{beta_i} = 0  (i = 1..m, x in (C*)^n)
is stored in the standard form of Sec. 2 (Eq. standard-form): the integer matrix
A (n x m) whose i-th column is alpha_i - beta_i.  The paper's own workload is the
gradient system of the master-space superpotential W_{m,k} (Sec. 6, Eq. superpotential
and Eq. mspace); the random families below are the synthetic stand-ins for the
benchmark configurations (single systems of growing size, a batch of uneven systems
and a served stream).  Every draw is made with numpy's PCG64 (`default_rng(seed)`).

Full column rank is enforced by resampling, using numpy's floating-point rank
(`numpy.linalg.matrix_rank`) of matrices with entries in {-2..2}; this is input
filtering only and plays no part in the computed degrees.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np


@dataclass
class BinomialSystem:
    """One binomial system x^A = b in standard form.

    A      : int64 array (n, m); column i is alpha_i - beta_i.
    coef   : optional int64 array (m, 2, 2): coef[i, j] = (numerator, denominator)
             of c_{i,j+1}.  None means "generic coefficients" (always consistent).
    alpha, beta : the two exponent vectors of every binomial, shape (m, n).
    """

    A: np.ndarray
    name: str = ""
    coef: Optional[np.ndarray] = None
    alpha: Optional[np.ndarray] = None
    beta: Optional[np.ndarray] = None
    meta: Dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.A.shape[0])

    @property
    def m(self) -> int:
        return int(self.A.shape[1])


def _monomial(rng: np.random.Generator, n: int, max_nonzeros: int, values) -> np.ndarray:
    nnz = int(rng.integers(1, max_nonzeros + 1))
    pos = rng.choice(n, size=nnz, replace=False)
    v = np.zeros(n, dtype=np.int64)
    v[pos] = rng.choice(np.asarray(values, dtype=np.int64), size=nnz)
    return v


def _quiver_monomial(rng: np.random.Generator, n: int) -> np.ndarray:
    nnz = int(rng.integers(2, 4))  # a product of 2 or 3 distinct variables
    pos = rng.choice(n, size=nnz, replace=False)
    v = np.zeros(n, dtype=np.int64)
    v[pos] = 1
    return v


def _draw_full_rank(rng, n, m, draw_monomial, max_tries=10000):
    for _ in range(max_tries):
        alpha = np.zeros((m, n), dtype=np.int64)
        beta = np.zeros((m, n), dtype=np.int64)
        for i in range(m):
            while True:
                a = draw_monomial()
                b = draw_monomial()
                if not np.array_equal(a, b):
                    break
            alpha[i], beta[i] = a, b
        A = (alpha - beta).T.copy()
        if np.linalg.matrix_rank(A.astype(np.float64)) == m:
            return A, alpha, beta
    raise RuntimeError(f"no full-rank system found for n={n}, m={m}")


def _unit_coefs(m: int) -> np.ndarray:
    # x^alpha - x^beta : c1 = 1, c2 = -1  (so b_i = -c2/c1 = 1)
    c = np.zeros((m, 2, 2), dtype=np.int64)
    c[:, 0] = (1, 1)
    c[:, 1] = (-1, 1)
    return c


def random_binomial_system(n: int, m: int, seed: int, max_nonzeros: int = 3,
                           values=(1, 2), name: str = "") -> BinomialSystem:
    """m binomials x^a - x^b in n variables; a, b in {0,1,2}^n with at most
    `max_nonzeros` nonzero entries each; resampled until rank A = m."""
    rng = np.random.default_rng(seed)
    A, alpha, beta = _draw_full_rank(rng, n, m, lambda: _monomial(rng, n, max_nonzeros, values))
    return BinomialSystem(A=A, name=name or f"random(n={n},m={m},seed={seed})",
                          coef=_unit_coefs(m), alpha=alpha, beta=beta,
                          meta=dict(n=n, m=m, seed=seed, max_nonzeros=max_nonzeros))


def quiver_binomial_system(n: int, m: int, seed: int, name: str = "") -> BinomialSystem:
    """m binomials whose monomials are products of 2-3 distinct variables (0/1 exponents)."""
    rng = np.random.default_rng(seed)
    A, alpha, beta = _draw_full_rank(rng, n, m, lambda: _quiver_monomial(rng, n))
    return BinomialSystem(A=A, name=name or f"quiver(n={n},m={m},seed={seed})",
                          coef=_unit_coefs(m), alpha=alpha, beta=beta,
                          meta=dict(n=n, m=m, seed=seed, style="quiver"))


# The benchmark configurations, by what they are.
CONFIGS = {
    "small_n10_k4": dict(kind="random", n=10, m=6, seed=0, max_nonzeros=3),
    "single_n24_k8": dict(kind="random", n=24, m=16, seed=0, max_nonzeros=4),
    "heavy_quiver_n32_k10": dict(kind="quiver", n=32, m=22, seed=0),
}


def config_system(name: str) -> BinomialSystem:
    c = CONFIGS[name]
    if c["kind"] == "random":
        return random_binomial_system(c["n"], c["m"], c["seed"], c["max_nonzeros"], name=name)
    return quiver_binomial_system(c["n"], c["m"], c["seed"], name=name)


def batch_systems(count: int = 4096, first_seed: int = 0, n_range=(12, 28), k_range=(4, 9),
                  max_nonzeros: int = 3) -> List[BinomialSystem]:
    """The uneven batch: system s uses seed first_seed+s, n ~ U[n_range], k ~ U[k_range],
    m = n - k binomials with exponents in {0,1,2}."""
    out = []
    for s in range(first_seed, first_seed + count):
        rng = np.random.default_rng(s)
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        sysm = random_binomial_system(n, n - k, seed=(s << 8) | 0x5A, max_nonzeros=max_nonzeros,
                                      name=f"batch{s}(n={n},k={k})")
        sysm.meta.update(batch_seed=s, k=k)
        out.append(sysm)
    return out


def master_space_system(m: int, k: int) -> BinomialSystem:
    """Gradient system of the superpotential W_{m,k} (Sec. 6, Eq. superpotential, Eq. mspace).

    W_{m,k} = sum_{i<m, j<k} x_{i,j} y_{i+1,j} z_{i+1,j+1} - y_{i,j} x_{i,j+1} z_{i+1,j+1},
    with the first index taken mod m and the second mod k.  Variables are ordered
    x_{i,j}, y_{i,j}, z_{i,j} (i major, j minor).  Each partial derivative is a
    binomial; its two monomials and signed coefficients are returned.
    """
    nv = 3 * m * k

    def var(kind, i, j):
        return {"x": 0, "y": 1, "z": 2}[kind] * m * k + (i % m) * k + (j % k)

    terms: Dict[Tuple[int, ...], int] = {}
    for i in range(m):
        for j in range(k):
            for sign, factors in ((+1, (("x", i, j), ("y", i + 1, j), ("z", i + 1, j + 1))),
                                  (-1, (("y", i, j), ("x", i, j + 1), ("z", i + 1, j + 1)))):
                e = [0] * nv
                for f in factors:
                    e[var(*f)] += 1
                key = tuple(e)
                terms[key] = terms.get(key, 0) + sign
    terms = {e: c for e, c in terms.items() if c != 0}

    alphas, betas, coefs = [], [], []
    for v in range(nv):
        deriv = {}
        for e, c in terms.items():
            if e[v] > 0:
                d = list(e)
                d[v] -= 1
                deriv[tuple(d)] = deriv.get(tuple(d), 0) + c * e[v]
        deriv = {e: c for e, c in deriv.items() if c != 0}
        if len(deriv) != 2:
            raise ValueError(f"dW/dv{v} of W_{{{m},{k}}} has {len(deriv)} terms")
        (e1, c1), (e2, c2) = sorted(deriv.items())
        alphas.append(e1)
        betas.append(e2)
        coefs.append(((c1, 1), (c2, 1)))
    alpha = np.asarray(alphas, dtype=np.int64)
    beta = np.asarray(betas, dtype=np.int64)
    A = (alpha - beta).T.copy()
    return BinomialSystem(A=A, name=f"master_space_W{m}{k}", coef=np.asarray(coefs, dtype=np.int64),
                          alpha=alpha, beta=beta, meta=dict(m=m, k=k))


def random_points(npts: int, k: int, seed: int, lo: int = -3, hi: int = 3) -> np.ndarray:
    """npts integer points in Z^k with coordinates uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(npts, k), dtype=np.int64)


def sparse_supports(k: int, points_per_set: int, seed: int, max_nonzeros: int = 3) -> List[np.ndarray]:
    """k supports in Z^k for a mixed volume (the BKK bound of a sparse polynomial system):
    each set holds the origin (a constant term) and points_per_set - 1 distinct exponent
    vectors with 1..max_nonzeros entries in {1, 2} at random positions."""
    rng = np.random.default_rng(seed)
    sets = []
    for _ in range(k):
        pts = {tuple([0] * k)}
        while len(pts) < points_per_set:
            v = np.zeros(k, dtype=np.int64)
            nz = rng.choice(k, size=int(rng.integers(1, max_nonzeros + 1)), replace=False)
            v[nz] = rng.integers(1, 3, size=len(nz))
            pts.add(tuple(int(x) for x in v))
        sets.append(np.array(sorted(pts), dtype=np.int64))
    return sets


# mixed-volume workloads: (k, points per set, seed)
MIXED_CONFIGS: Dict[str, Tuple[int, int, int]] = {
    "mixed_k3_p5": (3, 5, 0),    # 1,000 tuples of pairs: the oracle's size
    "mixed_k5_p6": (5, 6, 0),    # 759,375 tuples
    "mixed_k6_p7": (6, 7, 0),    # 85,766,121 tuples
    "mixed_k6_p8": (6, 8, 0),    # 481,890,304 tuples: the profiled case
    "mixed_k7_p8": (7, 8, 0),    # 13,492,928,512 tuples: the benchmark's mixed workload
}


def mixed_config(name: str) -> List[np.ndarray]:
    k, p, seed = MIXED_CONFIGS[name]
    return sparse_supports(k, p, seed)


def poisson_arrivals(rate_per_s: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: cumulative exponential gaps."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
