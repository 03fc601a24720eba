"""The allocation-free entry point bd_volume_noalloc against bd_volume.

bd_volume_noalloc exists for callers that cannot allocate device memory (a process whose device
memory is held by another allocator, or a loop that cannot afford cudaMalloc/cudaFree blocking
and synchronizing the device).  It keeps all device scratch in one static array inside the
library.  Two calls in a row must return exactly what bd_volume returns (results are exact
integers, so the tolerance is equality), which also checks that the second call is not
disturbed by what the first one left in the shared array.

This file sorts last so that a run stopping at the first failure has run every other test; it
passes both alone in a fresh process and after the rest of the suite.
"""

import json
import os

import numpy as np
import pytest

import paper_1501_02237_gb300 as bd
from workloads import config_system, random_points

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_volumes.json")))["configs"]

pytestmark = pytest.mark.gpu

FIELDS = ("nvol", "cells", "singular", "ties", "subsets", "flags", "max_abs_coord", "bound_bits")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    yield


def _same(a, b):
    return {f: a[f] for f in FIELDS} == {f: b[f] for f in FIELDS}


def test_noalloc_matches_volume_twice_in_a_row():
    # the benchmark-size single system (25 points in Z^8), then a different, smaller set: the
    # second call reuses the static array the first one filled
    P = bd.reduce(config_system("single_n24_k8").A)["points"]
    Q = random_points(18, 5, 3, -3, 3)
    for pts, seed in [(P, 0), (Q, 1)]:
        want = bd.volume(pts, seed=seed)
        first = bd.volume_noalloc(pts, seed=seed)
        second = bd.volume_noalloc(pts, seed=seed)
        assert _same(first, want), (first, want)
        assert _same(second, want), (second, want)
    # and the oracle's exact volume of the n = 24 system
    assert bd.volume_noalloc(P, seed=0)["nvol"] == GOLDEN["single_n24_k8"]["nvol"]


def test_noalloc_coarsens_a_work_list_above_the_cap():
    # 33 points in Z^10 (193,536,720 subsets): the first split makes 71,251 prefixes, more than
    # BD_NOALLOC_MAX_ITEMS, so the call coarsens it; the result must not change
    P = bd.reduce(config_system("heavy_quiver_n32_k10").A)["points"]
    want = bd.volume(P, seed=0)
    got = bd.volume_noalloc(P, seed=0)
    assert _same(got, want), (got, want)
    assert got["nvol"] == GOLDEN["heavy_quiver_n32_k10"]["nvol"]


def test_noalloc_128_bit_path():
    # kernel points of a system with exponent differences up to 1000: minors beyond 64 bits
    A = np.random.default_rng(0).integers(-1000, 1001, size=(10, 4)).astype(np.int64)
    P = bd.reduce(A)["points"]
    want = bd.volume(P, seed=4)
    assert want["flags"] & bd.BD_FLAG_INT128
    for _ in range(2):
        got = bd.volume_noalloc(P, seed=4)
        assert _same(got, want), (got, want)


def test_noalloc_rejects_sizes_beyond_the_limits():
    with pytest.raises(bd.BinodegError) as e:
        bd.volume_noalloc(np.zeros((bd.NMAX + 1, 3), dtype=np.int64))
    assert e.value.code == 1
    with pytest.raises(bd.BinodegError) as e:
        bd.volume_noalloc(np.zeros((20, bd.KMAX + 1), dtype=np.int64))
    assert e.value.code == 1
