"""GPU start solutions (bd_start_solutions) against the oracle: small sets solution by solution,
and the n=24 system (8.27 million solutions) by count, device residual and sampled solutions
checked against the oracle's own binomial systems."""

import random

import numpy as np
import pytest

import paper_1501_02237_gb300 as bd
from oracle.cells import lower_cells
from oracle.lifts import lifts as oracle_lifts
from oracle.start import cell_binomial, start_solutions
from workloads import config_system

from test_start_cpu import same_sets

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", range(8))
def test_gpu_start_solutions_match_oracle(seed):
    rng = random.Random(6100 + seed)
    k = rng.choice([1, 2, 3, 4])
    n = rng.randint(k + 2, 9)
    pts = [tuple(rng.randint(-2, 2) for _ in range(k)) for _ in range(n)]
    _, vol = bd.cells(np.array(pts), seed=seed)
    if vol["relifts"]:
        pytest.skip("the first lifting had a tie")
    ys, res = bd.start_solutions(np.array(pts), seed=seed, coef_seed=seed)
    cells = lower_cells(pts, oracle_lifts(n, seed))
    ref = start_solutions(pts, [c[0] for c in cells], seed)
    assert len(ys) == vol["nvol"] and res < 1e-10
    i = 0
    for (cell, v, _, _), rc in zip(cells, ref):
        assert same_sets(ys[i:i + v], rc)
        i += v


@pytest.mark.parametrize("coef_seed", [1, 3])
def test_gpu_start_solutions_full_size(coef_seed):
    # coefficient stream 1 gives solutions with |y| from 1e-177 to 1e153
    import torch
    P = bd.reduce(config_system("single_n24_k8").A)["points"]
    N, k = P.shape
    cells, vol = bd.cells(P, seed=0, capacity=1 << 14)
    out = torch.empty((vol["nvol"], k), dtype=torch.complex128, device="cuda")
    count, res = bd.start_solutions(P, seed=0, coef_seed=coef_seed, device_out=out)
    assert count == vol["nvol"] and res < 1e-8
    pts = P.tolist()
    from oracle.volume import det_int
    vols = [abs(det_int([[a - b for a, b in zip(pts[i], pts[c["cell"][-1]])] for i in c["cell"][:-1]])) for c in cells]
    first = np.cumsum([0] + vols)
    rng = random.Random(1)
    for ci in rng.sample(range(len(cells)), 12):
        E, b = cell_binomial(pts, cells[ci]["cell"], coef_seed)
        for t in rng.sample(range(vols[ci]), min(3, vols[ci])):
            y = out[first[ci] + t].cpu().numpy()
            lv = np.log(y) @ np.array(E).T  # in the log domain: y^E may leave double range
            assert np.max(np.abs(np.exp(lv - np.log(np.array(b, dtype=complex))) - 1)) < 1e-7
