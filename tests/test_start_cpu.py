"""Start solutions of the witness-set homotopy (Sec. 6) from the host emulation against the
oracle (oracle/start.py, which solves each cell's binomial system through its own Smith form):
the same solution set per cell, |det| solutions per cell, residuals at rounding level."""

import random

import numpy as np
import pytest

import paper_1501_02237_gb300 as bd
from oracle.cells import lower_cells
from oracle.lifts import lifts as oracle_lifts
from oracle.start import start_solutions


def same_sets(mine, ref, tol=1e-9):
    if len(mine) != len(ref):
        return False
    ref = np.array(ref)
    used = np.zeros(len(ref), dtype=bool)
    for y in mine:
        d = np.max(np.abs(ref - y[None, :]), axis=1)
        d[used] = np.inf
        j = int(np.argmin(d))
        if d[j] > tol * max(1.0, float(np.max(np.abs(y)))):
            return False
        used[j] = True
    return True


@pytest.mark.parametrize("seed", range(10))
def test_host_start_solutions_match_oracle(seed):
    rng = random.Random(5100 + seed)
    k = rng.choice([1, 2, 3, 4])
    n = rng.randint(k + 2, 8)
    pts = [tuple(rng.randint(-2, 2) for _ in range(k)) for _ in range(n)]
    lf = oracle_lifts(n, seed)
    ys, res = bd.host_start_solutions(np.array(pts), np.array(lf), coef_seed=seed)
    cells = lower_cells(pts, lf)
    ref = start_solutions(pts, [c[0] for c in cells], seed)
    assert len(ys) == sum(c[1] for c in cells)
    assert res < 1e-10
    i = 0
    for (cell, vol, _, _), rc in zip(cells, ref):
        assert same_sets(ys[i:i + vol], rc)
        i += vol


@pytest.mark.parametrize("seed", range(2))
def test_host_start_solutions_larger_cells(seed):
    # k = 5 cells with volumes in the hundreds: Hermite forms whose entries would grow without
    # the modular reduction, and Smith transforms large enough to test the oracle's exact phases
    rng = random.Random(7800 + seed)
    k = 5
    n = k + 3
    pts = [tuple(rng.randint(-3, 3) for _ in range(k)) for _ in range(n)]
    lf = oracle_lifts(n, seed)
    ys, res = bd.host_start_solutions(np.array(pts), np.array(lf), coef_seed=seed)
    cells = lower_cells(pts, lf)
    assert max(c[1] for c in cells) <= 4000, "pick a smaller case"
    ref = start_solutions(pts, [c[0] for c in cells], seed)
    assert len(ys) == sum(c[1] for c in cells) and res < 1e-9
    i = 0
    for (cell, vol, _, _), rc in zip(cells, ref):
        assert same_sets(ys[i:i + vol], rc, tol=1e-9)
        i += vol


def test_host_start_residual_far_from_unit_modulus():
    # n=24, k=8 system, coefficient stream 1: solutions range over |y| from 1e-177 to 1e153, so
    # the plain square-and-multiply of y^E under- or overflows; the residual check must not
    from oracle.start import cell_binomial
    from oracle.volume import det_int
    from workloads import config_system
    P = bd.reduce(config_system("single_n24_k8").A)["points"]
    W = np.array(oracle_lifts(P.shape[0], 0))
    ys, res = bd.host_start_solutions(P, W, coef_seed=1)
    mag = np.abs(np.log(np.abs(ys))).max(axis=1)
    assert mag.max() > 300, "the case no longer exercises extreme magnitudes"
    assert res < 1e-10
    # the most extreme solutions, checked in the log domain against the oracle's systems
    cells = bd.host_cells(P, W, capacity=1 << 14)
    pts = P.tolist()
    vols = [abs(det_int([[a - b for a, b in zip(pts[i], pts[c["cell"][-1]])] for i in c["cell"][:-1]]))
            for c in cells]
    first = np.cumsum([0] + vols)
    for t in np.argsort(mag)[-40:]:
        ci = int(np.searchsorted(first, t, side="right")) - 1
        E, b = cell_binomial(pts, cells[ci]["cell"], 1)
        lv = np.log(ys[t]) @ np.array(E).T
        assert np.max(np.abs(np.exp(lv - np.log(np.array(b, dtype=complex))) - 1)) < 1e-9
