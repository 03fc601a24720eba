"""GPU cells with inner normals (bd_cells) against the oracle: small sets compared cell by cell
with exact alpha and beta; the full-size system checked through the facet conditions on
sampled cells and the volume identity for all of them."""

import random
from fractions import Fraction

import numpy as np
import pytest

import paper_1501_02237_gb300 as bd
from oracle.cells import cell_normal, lower_cells
from oracle.lifts import lifts as oracle_lifts
from workloads import config_system

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", range(10))
def test_gpu_cells_match_oracle(seed):
    rng = random.Random(3100 + seed)
    k = rng.choice([1, 2, 3, 4, 5])
    n = rng.randint(k + 2, 10)
    pts = [tuple(rng.randint(-2, 2) for _ in range(k)) for _ in range(n)]
    got, vol = bd.cells(np.array(pts), seed=seed, capacity=3)
    if vol["relifts"]:
        pytest.skip("the first lifting had a tie")
    ref = lower_cells(pts, oracle_lifts(n, seed))
    assert [g["cell"] for g in got] == [tuple(c[0]) for c in ref]
    for g, (sub, v, alpha, beta) in zip(got, ref):
        assert g["alpha"] == alpha and g["beta"] == beta
    assert vol["cells"] == len(ref)


def test_gpu_cells_full_size():
    P = bd.reduce(config_system("single_n24_k8").A)["points"]
    got, vol = bd.cells(P, seed=0, capacity=1 << 14)
    assert len(got) == vol["cells"] and vol["relifts"] == 0
    pts = P.tolist()
    lf = oracle_lifts(len(pts), 0)
    from oracle.volume import det_int
    total = 0
    for g in got:
        s = g["cell"]
        total += abs(det_int([[a - b for a, b in zip(pts[i], pts[s[0]])] for i in s[1:]]))
    assert total == vol["nvol"]
    rng = random.Random(0)
    for g in rng.sample(got, 40):
        alpha, beta = cell_normal(pts, lf, g["cell"])
        assert g["alpha"] == alpha and g["beta"] == beta
        for q in range(len(pts)):
            h = sum(Fraction(x) * a for x, a in zip(pts[q], alpha)) + lf[q]
            assert (h == beta) if q in g["cell"] else (h > beta)
