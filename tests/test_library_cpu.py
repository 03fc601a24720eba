"""CPU checks of the native library: it loads, exports every symbol the public header declares,
and its host emulation of the GPU enumeration (same source as the kernel's walker, run by one
CPU thread per team) agrees with the oracle.  No GPU needed."""

import os
import random
import re

import numpy as np
import pytest

import paper_1501_02237_gb300 as bd
from paper_1501_02237_gb300._lib import SIGNATURES, lib
from oracle.lifts import lifts as oracle_lifts
from oracle.lower_facet import nvol_lifting_bruteforce
from oracle.snf import BinomialStructure
from oracle.volume import nvol_placing
from workloads import config_system, master_space_system

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = __import__("json").load(open(os.path.join(ROOT, "tests", "golden", "oracle_volumes.json")))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "binodeg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bd_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 14
    L = lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(SIGNATURES)


@pytest.mark.parametrize("seed", range(60))
def test_host_walker_matches_oracle_random(seed):
    rng = random.Random(seed)
    k = rng.randint(1, 5)
    npts = rng.randint(k + 1, 14)
    pts = [tuple(rng.randint(-3, 3) for _ in range(k)) for _ in range(npts)]
    lf = oracle_lifts(npts, seed)
    r = bd.host_volume_lifted(np.array(pts), np.array(lf))
    assert r["status"] == 0
    assert r["nvol"] == nvol_placing(pts)
    assert r["subsets"] == __import__("math").comb(npts, k + 1)


@pytest.mark.parametrize("seed", range(15))
def test_host_walker_counts_match_bruteforce(seed):
    # the number of accepted cells and singular subsets are fixed by the lifting
    rng = random.Random(1000 + seed)
    k = rng.randint(1, 3)
    npts = rng.randint(k + 1, 8)
    pts = [tuple(rng.randint(-2, 2) for _ in range(k)) for _ in range(npts)]
    lf = oracle_lifts(npts, seed)
    total, acc, sing, ties = nvol_lifting_bruteforce(pts, lf)
    r = bd.host_volume_lifted(np.array(pts), np.array(lf))
    assert (r["nvol"], r["cells"], r["singular"], r["ties"]) == (total, acc, sing, ties)


def test_host_walker_reports_ties():
    S = np.array([(0, 0), (0, 1), (1, 1), (1, 0)])
    r = bd.host_volume_lifted(S, np.array([0, 1, 2, 1]))
    assert r["status"] == 3 and r["ties"] == 4


def test_reduce_matches_oracle_structure():
    for name in ["small_n10_k4", "single_n24_k8"]:
        s = config_system(name)
        red = bd.reduce(s.A)
        ref = BinomialStructure(s.A.tolist())
        assert (red["rank"], red["dim"], red["torsion"]) == (ref.rank, ref.dim, ref.torsion)
        # the reduced points span the same lattice: volumes agree (GL_k(Z) invariance)
        assert nvol_placing([tuple(p) for p in red["points"]]) == GOLD["configs"][name]["nvol"]


def test_host_walker_config_small():
    s = config_system("small_n10_k4")
    P = bd.reduce(s.A)["points"]
    r = bd.host_volume_lifted(P, np.array(oracle_lifts(len(P), 0)))
    assert r["nvol"] == GOLD["configs"]["small_n10_k4"]["nvol"]


@pytest.mark.parametrize("mk,deg", [((2, 2), 14), ((2, 3), 92), ((1, 6), 32), ((2, 4), 584)])
def test_host_walker_master_space(mk, deg):
    s = master_space_system(*mk)
    red = bd.reduce(s.A, s.coef.reshape(-1, 4))
    assert red["consistent"] and red["torsion"] == 1
    r = bd.host_volume_lifted(red["points"], np.array(oracle_lifts(len(red["points"]), 3)), threads=4)
    assert r["nvol"] == deg


def test_reduce_consistency_matches_oracle():
    A = np.array([[1, 1]])
    assert not bd.reduce(A, [[1, 1, -2, 1], [1, 1, -3, 1]])["consistent"]
    assert bd.reduce(A, [[1, 1, -2, 1], [1, 2, -1, 1]])["consistent"]
    A2 = np.array([[2, 1]])
    assert bd.reduce(A2, [[1, 1, -4, 1], [1, 1, 2, 1]])["consistent"]
    assert not bd.reduce(A2, [[1, 1, -4, 1], [1, 1, -3, 1]])["consistent"]


def test_argument_errors_raise():
    with pytest.raises(bd.BinodegError):
        bd.host_volume_lifted(np.zeros((3, 15), dtype=np.int64), np.zeros(3, dtype=np.int64))
    with pytest.raises(bd.BinodegError):
        bd.host_volume_lifted(np.array([[1 << 41, 0], [0, 1], [1, 1]]), np.array([1, 2, 3]))


def _rand_matrix(rng, n, m, lo=-3, hi=3):
    A = [[rng.randint(lo, hi) for _ in range(m)] for _ in range(n)]
    if n >= 3 and rng.random() < 0.4:  # rank deficiency
        A[0] = [2 * a - b for a, b in zip(A[1], A[2])]
    if rng.random() < 0.3:  # torsion: scale a row-combination
        A[-1] = [3 * x for x in A[-1]]
    return A


@pytest.mark.parametrize("seed", range(80))
def test_reduce_invariants_random_matrices(seed):
    rng = random.Random(seed)
    n, m = rng.randint(1, 7), rng.randint(0, 6)
    A = _rand_matrix(rng, n, m) if m else [[] for _ in range(n)]
    ref = BinomialStructure(A)
    red = bd.reduce(np.array(A, dtype=np.int64).reshape(n, m))
    assert (red["rank"], red["dim"], red["torsion"]) == (ref.rank, ref.dim, ref.torsion)
    if ref.dim:
        P = red["points"][:n]
        # points are a kernel basis: P^T A = 0, and they give the oracle's volume
        assert not (P.T @ np.array(A, dtype=np.int64).reshape(n, m)).any()
        want = nvol_placing(ref.kernel_points() + [tuple([0] * ref.dim)])
        assert nvol_placing([tuple(p) for p in red["points"]]) == want


def test_reduce_batch_systems_match_oracle():
    from workloads import batch_systems
    gold = GOLD["batch_first_256"]
    for s, g in zip(batch_systems(96), gold):
        red = bd.reduce(s.A)
        ref = BinomialStructure(s.A.tolist())
        assert (red["rank"], red["torsion"]) == (ref.rank, ref.torsion), s.name
        P = red["points"][:-1]
        assert not (P.T @ s.A).any()


@pytest.mark.parametrize("idx", [0, 2, 25, 39])
def test_reduce_batch_volume_equals_oracle(idx):
    from workloads import batch_systems
    s = batch_systems(idx + 1)[idx]
    P = bd.reduce(s.A)["points"]
    assert nvol_placing([tuple(p) for p in P]) == GOLD["batch_first_256"][idx]["nvol"]


@pytest.mark.parametrize("seed", range(12))
def test_host_walker_all_integer_paths(seed):
    # small coordinates: int32 coordinate minors; |x| ~ 2^10 in k = 3: int64 minors;
    # forced: int128 minors.  All three must give the oracle's volume.
    rng = random.Random(300 + seed)
    k = 3
    for span, force in [(3, False), (1 << 10, False), (3, True), (1 << 10, True)]:
        pts = [tuple(rng.randint(-span, span) for _ in range(k)) for _ in range(rng.randint(5, 11))]
        lf = oracle_lifts(len(pts), seed)
        r = bd.host_volume_lifted(np.array(pts), np.array(lf), force_int128=force)
        assert r["status"] == 0
        assert r["nvol"] == nvol_placing(pts)
        if force:
            assert r["flags"] & bd.BD_FLAG_INT128


@pytest.mark.parametrize("seed", range(16))
def test_host_walker_deepest_items_and_exact_routes(seed):
    # item_subsets=1 splits every prefix down to the deepest item level, where the bottom stage
    # starts right away; coordinates scaled by 2^8 push the single-precision filters of the
    # bottom stage onto their exact routes (singular triples with large terms).  Every path
    # and split must give the oracle's volume.
    rng = random.Random(900 + seed)
    k = rng.choice([3, 4, 5])
    n = rng.randint(k + 2, 11)
    base = [tuple(rng.randint(-2, 2) for _ in range(k)) for _ in range(n)]
    for scale in (1, 256):
        pts = [tuple(scale * x for x in p) for p in base]
        ref = nvol_placing(pts)
        lf = oracle_lifts(n, seed)
        for items in (1, 0):
            for force in (False, True):
                r = bd.host_volume_lifted(np.array(pts), np.array(lf), force_int128=force, item_subsets=items)
                assert r["status"] == 0
                assert r["nvol"] == ref, (scale, items, force)


def test_host_walker_zero_lifts_are_ties():
    # constant lifts put every point on every lifted hyperplane: the filtered tests cannot
    # decide a sign and the exact route must report the ties
    rng = random.Random(5)
    pts = np.array([[rng.randint(-3, 3) for _ in range(4)] for _ in range(9)] + [[0] * 4])
    r = bd.host_volume_lifted(pts, np.zeros(len(pts), dtype=np.int64))
    assert r["status"] == 3 and r["ties"] > 0


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("width", [32, 7])
def test_lockstep_team_matches_oracle(seed, width):
    # one team of `width` lanes as CPU threads in lockstep runs the walker's multi-lane logic
    # (rows and triples dealt to lanes, ragged tails, votes); 32 is the GPU's team width
    rng = random.Random(1200 + seed)
    k = rng.choice([2, 3, 4, 5])
    n = rng.randint(k + 2, 10)
    pts = [tuple(rng.randint(-2, 2) for _ in range(k)) for _ in range(n)]
    pts = [tuple(16 * x for x in p) for p in pts] if seed % 3 == 2 else pts
    lf = oracle_lifts(n, seed)
    ref = nvol_placing(pts)
    for force in (False, True):
        r = bd.host_volume_lifted(np.array(pts), np.array(lf), force_int128=force, item_subsets=1 + seed % 2 * 40,
                                  team_width=width)
        assert r["status"] == 0
        assert r["nvol"] == ref, (k, n, force)


@pytest.mark.parametrize("seed,n,m", [(198, 46, 45), (234, 42, 41), (711, 39, 38), (5, 6, 5), (13, 12, 11), (44, 20, 19)])
def test_degree_of_curves_matches_oracle(seed, n, m):
    # one-dimensional solution sets: the degree is torsion x the length of the segment spanned
    # by the kernel points and 0 (taken directly, no enumeration), also for kernel vectors far
    # beyond the enumeration's coordinate range; the oracle runs its own Smith form and volume
    from oracle.degree import degree as oracle_degree
    from workloads import random_binomial_system
    s = random_binomial_system(n, m, seed, max_nonzeros=3 + seed % 4)
    o = oracle_degree(np.asarray(s.A).tolist())
    r = bd.degree(s.A)
    assert r["dim"] == 1 == o.dim
    assert r["degree"] == o.degree


@pytest.mark.parametrize("seed", [38, 39, 75, 118])
def test_reduce_large_systems_converges(seed):
    # n ~ 45 variables: the kernel elimination must not cycle between growth and LLL
    from workloads import random_binomial_system
    n = 8 + seed % 40
    m = max(1, n - 1 - seed % 9)
    s = random_binomial_system(n, m, seed, max_nonzeros=3 + seed % 4)
    red = bd.reduce(s.A)
    ref = BinomialStructure(np.asarray(s.A).tolist())
    assert (red["rank"], red["dim"], red["torsion"]) == (ref.rank, ref.dim, ref.torsion)


@pytest.mark.parametrize("seed,width", [(0, 8), (1, 8), (2, 16), (3, 16)])
def test_lockstep_team_narrower_than_the_point_set(seed, width):
    # more points than lanes (the GPU runs 33 points on 32 lanes): the levels whose remaining
    # points fit one pass build them compacted (lane l takes the l-th point outside the prefix),
    # the others deal the ragged tail across lanes; both integer paths against the oracle
    rng = random.Random(5100 + seed)
    n, k = width + 1 + seed % 2 * 2, 4
    pts = [tuple(rng.randint(-3, 3) for _ in range(k)) for _ in range(n)]
    lf = oracle_lifts(n, seed)
    ref = nvol_placing(pts)
    for force in (False, True):
        r = bd.host_volume_lifted(np.array(pts), np.array(lf), force_int128=force, team_width=width)
        assert r["status"] == 0
        assert r["nvol"] == ref, (n, force)


@pytest.mark.parametrize("seed", range(8))
def test_host_walker_5d_exact_routes(seed):
    # degenerate point sets (coordinates 0 and +-63 in dimensions 4 and 5): the 5-D stage's
    # coordinate det4 has terms near 2^24 and sums that round, so singular quadruples land inside
    # the error bound and take the exact route; deepest items and default items, both against
    # the oracle's volume
    rng = random.Random(7700 + seed)
    k = 4 + seed % 2
    n = rng.randint(k + 4, 12)
    pts = [tuple(63 * rng.choice([-1, 0, 0, 1]) for _ in range(k)) for _ in range(n)]
    pts = list(dict.fromkeys(pts))  # distinct points
    if len(pts) < k + 1:
        pytest.skip("degenerate draw")
    ref = nvol_placing(pts)
    lf = oracle_lifts(len(pts), seed)
    for items in (1, 0):
        r = bd.host_volume_lifted(np.array(pts), np.array(lf), item_subsets=items)
        assert r["status"] == 0
        assert r["nvol"] == ref, (k, len(pts), items)
        assert not r["flags"] & bd.BD_FLAG_INT128


@pytest.mark.parametrize("seed", range(6))
def test_host_walker_5d_exact_sides(seed):
    # lifts nearly affine in the coordinates (10^6 times their sum plus a small perturbation) put
    # every point close to every cell's hyperplane at a large scale: the 5-D stage's single-
    # precision side test cannot decide and takes the exact route; an affine part does not change
    # the triangulation, so the volume is the oracle's whatever the perturbation (redrawn when it
    # happens to give a tie)
    rng = random.Random(8800 + seed)
    k = 4 + seed % 2
    n = rng.randint(k + 4, 11)
    pts = list(dict.fromkeys(tuple(31 * rng.choice([-1, 0, 1]) for _ in range(k)) for _ in range(n)))
    if len(pts) < k + 1:
        pytest.skip("degenerate draw")
    ref = nvol_placing(pts)
    for _ in range(8):
        lf = [10**6 * sum(p) + rng.randint(-20, 20) for p in pts]
        r = bd.host_volume_lifted(np.array(pts), np.array(lf))
        if r["status"] == 0:
            break
    assert r["status"] == 0
    assert r["nvol"] == ref


@pytest.mark.parametrize("seed", range(6))
def test_host_walker_64_bit_coordinates_high_dimension(seed):
    # coordinates up to 64 (k = 4) and 40 (k = 5): coordinate minors past 31 bits and lifted
    # minors below 63, so the walk takes the int64 path and its 4-D stage (the 5-D stage runs on
    # 32-bit coordinate minors)
    rng = random.Random(9100 + seed)
    k = 4 + seed % 2
    span = 64 if k == 4 else 40
    pts = [tuple(rng.randint(-span, span) for _ in range(k)) for _ in range(rng.randint(k + 3, 10))]
    lf = oracle_lifts(len(pts), seed)
    for items in (1, 0):
        r = bd.host_volume_lifted(np.array(pts), np.array(lf), item_subsets=items)
        assert r["status"] == 0
        assert r["nvol"] == nvol_placing(pts), (k, items)
        assert r["bound_bits"] > 31 and not r["flags"] & bd.BD_FLAG_INT128


@pytest.mark.parametrize("seed", range(12))
def test_host_walker_both_bottom_stages(seed):
    # the 32-bit coordinate path ends in the 5-D test or the 4-D test (chosen per point set, or
    # fixed by the caller): both give the oracle's volume, with the deepest items, the default
    # items and a lockstep team of four lanes; k = 3 and the int64 path ignore the choice
    rng = random.Random(9900 + seed)
    k = 3 + seed % 4
    n = rng.randint(k + 3, 13)
    span = 3 if seed % 3 else 1
    pts = [tuple(rng.randint(-span, span) for _ in range(k)) for _ in range(n)]
    ref = nvol_placing(pts)
    lf = oracle_lifts(n, seed)
    for stage in (4, 5, 0):
        for items, width in ((1, 1), (0, 1), (0, 4)):
            r = bd.host_volume_lifted(np.array(pts), np.array(lf), item_subsets=items, team_width=width,
                                      bottom_stage=stage)
            if r["status"] == 3:
                continue  # a tie under this lifting: the same for every stage and work list
            assert r["status"] == 0
            assert r["nvol"] == ref, (k, stage, items, width)


def test_bottom_stage_argument_is_checked():
    pts = np.array([(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1), (1, 1, 1, 1)])
    with pytest.raises(bd.BinodegError):
        bd.host_volume_lifted(pts, np.arange(1, 7), bottom_stage=3)


@pytest.mark.parametrize("k", [4, 6])
def test_host_walker_both_stages_at_the_point_limit(k):
    # 64 distinct points (every mask word full) and the deepest work items (5-D nodes split by the
    # first point of their quadruples): both bottom stages give the oracle's volume
    rng = random.Random(64 + k)
    pts = []
    while len(pts) < 64:
        p = tuple(rng.randint(-3, 3) for _ in range(k))
        if p not in pts:
            pts.append(p)
    ref = nvol_placing(pts)
    lf = oracle_lifts(64, k)
    for stage in (4, 5):
        r = bd.host_volume_lifted(np.array(pts), np.array(lf), threads=4, item_subsets=1, bottom_stage=stage)
        assert r["status"] == 0
        assert r["nvol"] == ref, stage
