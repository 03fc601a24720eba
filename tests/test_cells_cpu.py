"""Cells of the lifting's triangulation with their inner normals, from the host emulation of
the enumeration, against the oracle (oracle/cells.py): same cells, same exact alpha and beta."""

import random

import numpy as np
import pytest

import paper_1501_02237_gb300 as bd
from oracle.cells import lower_cells
from oracle.lifts import lifts as oracle_lifts


@pytest.mark.parametrize("seed", range(14))
def test_host_cells_match_oracle(seed):
    rng = random.Random(2100 + seed)
    k = rng.choice([1, 2, 3, 4])
    n = rng.randint(k + 2, 9)
    scale = 64 if seed % 3 == 2 else 1
    pts = [tuple(scale * rng.randint(-2, 2) for _ in range(k)) for _ in range(n)]
    lf = oracle_lifts(n, seed)
    got = bd.host_cells(np.array(pts), np.array(lf), capacity=2)  # small capacity: exercises the retry
    ref = lower_cells(pts, lf)
    assert [g["cell"] for g in got] == [tuple(c[0]) for c in ref]
    for g, (sub, vol, alpha, beta) in zip(got, ref):
        assert g["alpha"] == alpha and g["beta"] == beta


def test_host_cells_count_only_and_ties():
    pts = np.array([(0, 0), (1, 0), (0, 1), (1, 1)])
    with pytest.raises(bd.BinodegError):
        bd.host_cells(pts, np.zeros(4, dtype=np.int64))  # constant lifts: ties


def test_host_cells_segment_and_mid_path():
    # k = 1: cells are consecutive distinct points; coordinates of 2^20 take the 64-bit path
    pts = np.array([[0], [3], [-2], [5], [3]])
    got = bd.host_cells(pts, np.array(oracle_lifts(5, 1)))
    assert sum(1 for _ in got) == len(lower_cells(pts.tolist(), oracle_lifts(5, 1)))
    pts2 = [(a, b) for a in (0, 1 << 20) for b in (0, 3 << 19)] + [(1 << 19, 1 << 18)]
    lf = oracle_lifts(len(pts2), 2)
    got2 = bd.host_cells(np.array(pts2), np.array(lf))
    ref2 = lower_cells(pts2, lf)
    assert [g["cell"] for g in got2] == [tuple(c[0]) for c in ref2]
    assert all(g["alpha"] == c[2] and g["beta"] == c[3] for g, c in zip(got2, ref2))
