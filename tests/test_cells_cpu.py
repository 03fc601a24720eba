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
