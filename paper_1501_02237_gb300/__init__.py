"""Exact degree of binomial-system solution sets on GB300 (Chen & Mehta, arXiv 1501.02237).

Python face of libbinodeg.so, with the same names as the C ABI (include/binodeg.h).
Every computation runs in the library: the host front end (Smith form, kernel basis)
in C++ and the lower-facet enumeration in CUDA.  If the library is missing, calls raise.
"""

from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from ._lib import (BD_FEATURES, BD_MLP_PARAMS, BD_FLAG_DEGENERATE, BD_FLAG_INCONSISTENT, BD_FLAG_INT128, BD_FLAG_PIVOT, KMAX,  # noqa: F401
                   NMAX, BatchOpts, BatchStats, BinodegError, DegreeOut, HostOpts, MixedOut, PeakOut, PlanOpts, ServerOpts,
                   ServerStats, VolumeOut, check, i64, lib, ptr)
from ._lib import BD_OK, F32P, I32P, U8P

__all__ = ["CostModel", "Server", "degree", "volume", "volume_noalloc", "volume_lifted", "classify", "reduce", "Plan", "Batch", "set_stream",
           "host_volume_lifted", "cells", "host_cells", "start_solutions", "host_start_solutions", "mixed_volume",
           "mixed_volume_lifted", "host_mixed_volume_lifted", "volume_pivot", "host_volume_pivot", "degree_pivot",
           "issue_peak", "inject_alloc_failure", "pivot_force_wide", "BinodegError", "lib"]


def set_stream(stream) -> None:
    """Stream for the synchronous calls on this thread: a torch.cuda.Stream, a raw handle or None."""
    handle = getattr(stream, "cuda_stream", stream)
    check(lib().bd_set_stream(C.c_void_p(handle or 0)))


def inject_alloc_failure(after: int = 0) -> None:
    """bd_inject_alloc_failure: the after-th device allocation from now fails as out of memory
    (once; after < 0 disarms).  For tests of the error paths."""
    check(lib().bd_inject_alloc_failure(after))


ISSUE_KINDS = {"lop3": 0, "imad": 1, "lop3_imad": 2, "ffma": 3, "lop3_ffma": 4}


def issue_peak(kind: str = "lop3_imad", blocks_per_sm: int = 0, iters: int = 4096) -> dict:
    """bd_issue_peak: lane operations per second of one 32-bit instruction stream at full occupancy
    (kinds: lop3, imad, lop3_imad, ffma, lop3_ffma)."""
    out = PeakOut()
    check(lib().bd_issue_peak(ISSUE_KINDS[kind], blocks_per_sm, iters, C.byref(out)))
    return out.as_dict()


def _coef_array(coef, m: int) -> Optional[np.ndarray]:
    if coef is None:
        return None
    c = i64(coef).reshape(m, 4)
    return np.ascontiguousarray(c)


def degree(A, coef=None, seed: int = 0) -> dict:
    """bd_degree: degree of V(x^A - b); A is n x m (column i = alpha_i - beta_i).
    coef: None or m x 2 x 2 / m x 4 integers (num, den) of c_{i,1}, c_{i,2}."""
    A = i64(A)
    n, m = A.shape
    c = _coef_array(coef, m)
    out = DegreeOut()
    check(lib().bd_degree(ptr(A), n, m, ptr(c) if c is not None else None, C.c_uint64(seed), C.byref(out)))
    return out.as_dict()



def _cells_result(n, k, cells, den, alpha, beta):
    from fractions import Fraction
    out = []
    for r in range(n):
        b = (int(beta[2 * r + 1]) << 64) | (int(beta[2 * r]) & ((1 << 64) - 1))
        d = int(den[r])
        out.append(dict(cell=tuple(int(x) for x in cells[r * (k + 1):(r + 1) * (k + 1)]),
                        alpha=[Fraction(int(a), d) for a in alpha[r * k:(r + 1) * k]], beta=Fraction(b, d)))
    return out


def _cells_call(fn, k, capacity):
    """Call fn(capacity, cells, den, alpha, beta, count) twice if the first capacity is too small."""
    for _ in range(2):
        cap = max(1, capacity)
        cells = np.zeros(cap * (k + 1), dtype=np.uint8)
        den = np.zeros(cap, dtype=np.int64)
        alpha = np.zeros(cap * k, dtype=np.int64)
        beta = np.zeros(2 * cap, dtype=np.int64)
        count = C.c_int64(0)
        rc = fn(capacity, cells.ctypes.data_as(U8P), ptr(den), ptr(alpha), ptr(beta), C.byref(count))
        if rc == 1 and count.value > capacity:  # BD_ERR_ARG with the true count: retry once
            capacity = int(count.value)
            continue
        check(rc)
        return _cells_result(int(count.value), k, cells, den, alpha, beta)
    check(rc)


def cells(points, seed: int = 0, capacity: int = 4096):
    """bd_cells: the cells of the lifting's triangulation with their exact inner normals
    (alpha, beta as Fractions) and the volume result: (cells, volume dict)."""
    P = i64(points)
    npts, k = P.shape
    out = VolumeOut()
    res = _cells_call(lambda cap, c, d, a, b, n: lib().bd_cells(ptr(P), npts, k, C.c_uint64(seed), cap, c, d, a, b, n,
                                                             C.byref(out)), k, capacity)
    return res, out.as_dict()


def host_cells(points, lifts, capacity: int = 4096):
    """bd_host_cells: the same with the given lifts on the host (CPU tests)."""
    P, W = i64(points), i64(lifts)
    npts, k = P.shape
    return _cells_call(lambda cap, c, d, a, b, n: lib().bd_host_cells(ptr(P), ptr(W), npts, k, cap, c, d, a, b, n),
                       k, capacity)


def _start_call(fn, k):
    count = C.c_int64(0)
    res = C.c_double(0)
    rc = fn(0, None, C.byref(count), C.byref(res))  # the count first
    if rc not in (0, 1):
        check(rc)
    n = int(count.value)
    out = np.zeros((max(n, 1), k), dtype=np.complex128)
    check(fn(n, out.ctypes.data_as(C.c_void_p), C.byref(count), C.byref(res)))
    return out[:n], float(res.value)


def start_solutions(points, seed: int = 0, coef_seed: int = 0, device_out=None):
    """bd_start_solutions: (solutions as an (nvol, k) complex array, cell by cell in the order
    of cells(), and the largest equation residual checked on the device).  With device_out (a
    contiguous complex128 CUDA tensor of at least nvol x k elements) the solutions stay in it
    and (count, residual) is returned instead."""
    P = i64(points)
    npts, k = P.shape
    if device_out is not None:
        count, res = C.c_int64(0), C.c_double(0)
        check(lib().bd_start_solutions(ptr(P), npts, k, C.c_uint64(seed), C.c_uint64(coef_seed),
                                       device_out.numel() // k, C.c_void_p(device_out.data_ptr()), 1,
                                       C.byref(count), C.byref(res)))
        return int(count.value), float(res.value)
    return _start_call(lambda cap, buf, cnt, res: lib().bd_start_solutions(ptr(P), npts, k, C.c_uint64(seed),
                                                                          C.c_uint64(coef_seed), cap, buf, 0, cnt, res), k)


def host_start_solutions(points, lifts, coef_seed: int = 0):
    """bd_host_start_solutions: the same with the given lifts on the host (CPU tests)."""
    P, W = i64(points), i64(lifts)
    npts, k = P.shape
    return _start_call(lambda cap, buf, cnt, res: lib().bd_host_start_solutions(ptr(P), ptr(W), npts, k,
                                                                               C.c_uint64(coef_seed), cap, buf, cnt,
                                                                               res), k)

def reduce(A, coef=None) -> dict:
    """bd_reduce: host front end only -> kernel points (n+1 x d, origin last), rank, torsion."""
    A = i64(A)
    n, m = A.shape
    c = _coef_array(coef, m)
    pts = np.zeros((n + 1) * n, dtype=np.int64)
    info = np.zeros(8, dtype=np.int64)
    check(lib().bd_reduce(ptr(A), n, m, ptr(c) if c is not None else None, ptr(pts), ptr(info)))
    d = int(info[1])
    return dict(points=pts[: (n + 1) * d].reshape(n + 1, d), rank=int(info[0]), dim=d, torsion=int(info[2]),
                consistent=bool(info[3]), max_abs_coord=int(info[4]))


def volume(points, seed: int = 0) -> dict:
    """bd_volume: exact NVol_k(conv points), points npts x k (the origin is not added)."""
    P = i64(points)
    npts, k = P.shape
    out = VolumeOut()
    check(lib().bd_volume(ptr(P), npts, k, C.c_uint64(seed), C.byref(out)))
    return out.as_dict()


def volume_noalloc(points, seed: int = 0) -> dict:
    """bd_volume_noalloc: bd_volume without any device allocation (static scratch in the library)."""
    P = i64(points)
    npts, k = P.shape
    out = VolumeOut()
    check(lib().bd_volume_noalloc(ptr(P), npts, k, C.c_uint64(seed), C.byref(out)))
    return out.as_dict()


def volume_lifted(points, lifts) -> dict:
    """bd_volume_lifted: the same with caller-given lift heights and no re-lift."""
    P, W = i64(points), i64(lifts)
    npts, k = P.shape
    out = VolumeOut()
    rc = lib().bd_volume_lifted(ptr(P), ptr(W), npts, k, C.byref(out))
    res = out.as_dict()
    res["status"] = rc
    if rc not in (0, 3):
        check(rc)
    return res


def classify(points, lifts, subsets) -> tuple:
    """bd_classify: (status, absdet) arrays for the given (k+1)-subsets (rows of indices)."""
    P, W = i64(points), i64(lifts)
    npts, k = P.shape
    S = np.ascontiguousarray(np.asarray(subsets, dtype=np.uint8).reshape(-1, k + 1))
    cnt = S.shape[0]
    status = np.zeros(cnt, dtype=np.int32)
    absdet = np.zeros(cnt, dtype=np.int64)
    check(lib().bd_classify(ptr(P), ptr(W), npts, k, S.ctypes.data_as(U8P), cnt, status.ctypes.data_as(I32P),
                            ptr(absdet)))
    return status, absdet


def host_volume_lifted(points, lifts, threads: int = 1, force_int128: bool = False, item_subsets: int = 0,
                       team_width: int = 1, shard: int = 0, shards: int = 1, bottom_stage: int = 0) -> dict:
    """bd_host_volume_lifted: CPU emulation of the enumeration (CPU tests and the native baseline).
    force_int128 runs the 128-bit walker; item_subsets is the work-item split threshold (0: the
    library's default); team_width > 1 runs one team of that many lanes as threads in lockstep;
    shards > 1 runs only shard `shard` of the work list (partial sums); bottom_stage 4 or 5 fixes
    the walk's last stage on the 32-bit coordinate path (0: chosen from the point set)."""
    P, W = i64(points), i64(lifts)
    npts, k = P.shape
    out = VolumeOut()
    opts = HostOpts(threads, int(force_int128), item_subsets, team_width, shard, shards, bottom_stage)
    rc = lib().bd_host_volume_lifted(ptr(P), ptr(W), npts, k, C.byref(opts), C.byref(out))
    res = out.as_dict()
    res["status"] = rc
    if rc not in (0, 3):
        check(rc)
    return res


def volume_pivot(points, seed: int = 0) -> dict:
    """bd_volume_pivot: exact NVol_k(conv points) by simplicial pivoting over the cells on the GPU
    (output-sensitive; k <= 30, up to 127 points); adds the traversal's GPU time as device_ms."""
    P = i64(points)
    npts, k = P.shape
    out, ms = VolumeOut(), C.c_double(0)
    check(lib().bd_volume_pivot(ptr(P), npts, k, C.c_uint64(seed), C.byref(out), C.byref(ms)))
    res = out.as_dict()
    res["device_ms"] = float(ms.value)
    return res


def host_volume_pivot(points, lifts, team_width: int = 1, cells: bool = False, capacity: int = 1 << 16,
                      walk_budget: int = 64) -> dict:
    """bd_host_volume_pivot: the same traversal on the host with the given heights (CPU tests);
    walk_budget cells entered in place below each eliminated cell (0: eliminate every cell);
    cells=True adds the cells as sorted tuples of point indices."""
    P, W = i64(points), i64(lifts)
    npts, k = P.shape
    out = VolumeOut()
    buf = np.zeros(max(capacity, 1), dtype=np.uint64)
    rc = lib().bd_host_volume_pivot(ptr(P), ptr(W), npts, k, team_width, walk_budget, C.byref(out),
                                    buf.ctypes.data_as(C.POINTER(C.c_uint64)) if cells else None, capacity)
    res = out.as_dict()
    res["status"] = rc
    if rc not in (0, 3):
        check(rc)
    if cells and rc == 0:
        res["cell_list"] = [tuple(i for i in range(64) if (int(m) >> i) & 1) for m in buf[: int(out.cells)]]
    return res


def pivot_force_wide(on: bool = True) -> bool:
    """bd_pivot_force_wide (test hook): the pivoting walk takes 128-bit tableau entries whatever
    the bound while on; returns the previous setting."""
    return bool(lib().bd_pivot_force_wide(1 if on else 0))


def degree_pivot(A, coef=None, seed: int = 0) -> dict:
    """bd_degree_pivot: bd_degree with the volume by simplicial pivoting (solution sets of
    dimension up to 30)."""
    A = i64(A)
    n, m = A.shape
    c = _coef_array(coef, m)
    out = DegreeOut()
    check(lib().bd_degree_pivot(ptr(A), n, m, ptr(c) if c is not None else None, C.c_uint64(seed), C.byref(out)))
    return out.as_dict()


def _supports(supports):
    """Point sets -> (flat points, counts, k)."""
    sets = [i64(A).reshape(len(A), -1) for A in supports]
    k = len(sets)
    if any(A.shape[1] != k for A in sets):
        raise ValueError("k point sets in Z^k")
    return i64(np.concatenate(sets, axis=0)), np.array([len(A) for A in sets], dtype=np.int32), k


def mixed_volume(supports, seed: int = 0) -> dict:
    """bd_mixed_volume: MV(conv A_1, .., conv A_k) of k point sets in Z^k on the GPU (the BKK
    bound; MV(P, .., P) = NVol(P))."""
    P, cnt, k = _supports(supports)
    out = MixedOut()
    check(lib().bd_mixed_volume(ptr(P), cnt.ctypes.data_as(I32P), k, C.c_uint64(seed), C.byref(out)))
    return out.as_dict()


def _mixed_lifted(fn, supports, lifts, with_cells, capacity):
    P, cnt, k = _supports(supports)
    W = i64(lifts)
    out = MixedOut()
    while True:
        cap = capacity if with_cells else 0
        cells = np.zeros((max(cap, 1), 2 * k), dtype=np.int32)
        dets = np.zeros(max(cap, 1), dtype=np.int64)
        rc = fn(ptr(P), cnt.ctypes.data_as(I32P), k, ptr(W), out, cells.ctypes.data_as(I32P) if with_cells else None,
                cap, ptr(dets) if with_cells else None)
        if with_cells and rc == 1 and out.cells > cap:
            capacity = int(out.cells)
            continue
        break
    res = out.as_dict()
    res["status"] = rc
    if rc not in (0, 3):
        check(rc)
    if with_cells and rc == 0:
        n = int(out.cells)
        res["cell_list"] = [tuple((int(c[2 * i]), int(c[2 * i + 1])) for i in range(k)) for c in cells[:n]]
        res["absdet"] = [int(d) for d in dets[:n]]
    return res


def mixed_volume_lifted(supports, lifts, cells: bool = False, force_int128: bool = False, capacity: int = 4096) -> dict:
    """bd_mixed_volume_lifted: the same on the GPU with the given flat heights and no re-lift
    (status 3 on a tie); cells=True also lists the fine mixed cells in "cell_list" (pairs of
    local indices per set, lexicographic) with their |det M| in "absdet"."""
    f = lambda *a: lib().bd_mixed_volume_lifted(a[0], a[1], a[2], a[3], int(force_int128), C.byref(a[4]), *a[5:])
    return _mixed_lifted(f, supports, lifts, cells, capacity)


def host_mixed_volume_lifted(supports, lifts, team_width: int = 1, cells: bool = False, force_int128: bool = False,
                             capacity: int = 4096, prefix_levels: int = 0, leaf3: int = -1) -> dict:
    """bd_host_mixed_volume_lifted: the mixed-cell walker on CPU threads (CPU tests);
    prefix_levels > 0 fixes that many levels per work item; leaf3 1/0 forces the 3-D leaf
    stage on/off (-1: the library's choice)."""
    f = lambda *a: lib().bd_host_mixed_volume_lifted(a[0], a[1], a[2], a[3], team_width, int(force_int128),
                                                     prefix_levels, leaf3, C.byref(a[4]), *a[5:])
    return _mixed_lifted(f, supports, lifts, cells, capacity)


class Plan:
    """bd_plan_*: device-resident enumeration of one point set."""

    def __init__(self, points, warps_per_block: int = 0, blocks_per_sm: int = 0, item_subsets: int = 0,
                 force_int128: bool = False, bottom_stage: int = 0):
        P = i64(points)
        self.npts, self.k = P.shape
        opts = PlanOpts(warps_per_block, blocks_per_sm, item_subsets, int(force_int128), bottom_stage)
        h = C.c_void_p()
        check(lib().bd_plan_create(ptr(P), self.npts, self.k, C.byref(opts), C.byref(h)))
        self.handle = h

    def launch(self, seed: int = 0, attempt: int = 0, stream=None, shard: int = 0, shards: int = 1) -> None:
        s = getattr(stream, "cuda_stream", stream)
        if shards > 1:
            check(lib().bd_plan_launch_shard(self.handle, C.c_uint64(seed), attempt, shard, shards, C.c_void_p(s or 0)))
        else:
            check(lib().bd_plan_launch(self.handle, C.c_uint64(seed), attempt, C.c_void_p(s or 0)))

    def read(self) -> dict:
        out = VolumeOut()
        check(lib().bd_plan_read(self.handle, C.byref(out)))
        return out.as_dict()

    def volume(self, seed: int = 0) -> dict:
        out = VolumeOut()
        check(lib().bd_plan_volume(self.handle, C.c_uint64(seed), C.byref(out)))
        return out.as_dict()

    def info(self) -> dict:
        a = np.zeros(8, dtype=np.int64)
        check(lib().bd_plan_info(self.handle, ptr(a)))
        return dict(items=int(a[0]), blocks=int(a[1]), warps_per_block=int(a[2]), smem=int(a[3]),
                    path=("int32/int64", "int64", "int128")[int(a[4])], int128=int(a[4]) == 2, slots=int(a[5]), ranges=int(a[6]),
                    bottom_stage=int(a[7]))

    def close(self) -> None:
        if getattr(self, "handle", None):
            lib().bd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """bd_batch_*: many systems reduced on host threads and enumerated in persistent launches."""

    def __init__(self):
        h = C.c_void_p()
        check(lib().bd_batch_create(C.byref(h)))
        self.handle = h
        self.count = 0

    def add(self, A, coef=None, seed: int = 0) -> int:
        A = i64(A)
        n, m = A.shape
        c = _coef_array(coef, m)
        idx = C.c_int32()
        check(lib().bd_batch_add(self.handle, ptr(A), n, m, ptr(c) if c is not None else None, C.c_uint64(seed),
                                 C.byref(idx)))
        self.count += 1
        return idx.value

    def add_points(self, points, seed: int = 0) -> int:
        P = i64(points)
        npts, k = P.shape
        idx = C.c_int32()
        check(lib().bd_batch_add_points(self.handle, ptr(P), npts, k, C.c_uint64(seed), C.byref(idx)))
        self.count += 1
        return idx.value

    def prepare(self, threads: int = 0) -> None:
        check(lib().bd_batch_prepare(self.handle, threads))

    def features(self) -> np.ndarray:
        f = np.zeros((self.count, BD_FEATURES), dtype=np.float32)
        check(lib().bd_batch_features(self.handle, f.ctypes.data_as(F32P)))
        return f

    def run(self, mode: int = 0, warps_per_block: int = 0, item_factor: int = 0, use_graph: bool = False,
            autotune: bool = False, cost=None, bottom_stage: int = 0) -> dict:
        self._cost = None if cost is None else np.ascontiguousarray(np.asarray(cost, dtype=np.float32))
        o = BatchOpts(mode, warps_per_block, item_factor, int(use_graph), int(autotune), bottom_stage,
                      self._cost.ctypes.data_as(F32P) if self._cost is not None else None)
        st = BatchStats()
        check(lib().bd_batch_run(self.handle, C.byref(o), C.byref(st)))
        return st.as_dict()

    def result(self, index: int) -> dict:
        out = DegreeOut()
        cyc = C.c_uint64()
        check(lib().bd_batch_result(self.handle, index, C.byref(out), C.byref(cyc)))
        d = out.as_dict()
        d["cycles"] = int(cyc.value)
        return d

    def results(self) -> list:
        return [self.result(i) for i in range(self.count)]

    def close(self) -> None:
        if getattr(self, "handle", None):
            lib().bd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


class CostModel:
    """bd_mlp_*: the learned cost model (16 -> 64 -> 64 -> 1, FP32) trained by the library's kernels."""

    def __init__(self, seed: int = 0):
        h = C.c_void_p()
        check(lib().bd_mlp_create(C.c_uint64(seed), C.byref(h)))
        self.handle = h

    def params(self):
        p = np.zeros(BD_MLP_PARAMS, dtype=np.float32)
        nrm = np.zeros(2 * BD_FEATURES, dtype=np.float32)
        check(lib().bd_mlp_get_params(self.handle, p.ctypes.data_as(F32P), nrm.ctypes.data_as(F32P)))
        return p, nrm

    def set_params(self, params, norm=None) -> None:
        p = _f32(params)
        n = None if norm is None else _f32(norm)
        check(lib().bd_mlp_set_params(self.handle, p.ctypes.data_as(F32P), None if n is None else n.ctypes.data_as(F32P)))

    def predict(self, X) -> np.ndarray:
        X = _f32(X)
        y = np.zeros(X.shape[0], dtype=np.float32)
        check(lib().bd_mlp_predict(self.handle, X.ctypes.data_as(F32P), X.shape[0], y.ctypes.data_as(F32P)))
        return y

    def gradient(self, X, y):
        X, y = _f32(X), _f32(y)
        g = np.zeros(BD_MLP_PARAMS, dtype=np.float32)
        loss = C.c_float()
        check(lib().bd_mlp_gradient(self.handle, X.ctypes.data_as(F32P), y.ctypes.data_as(F32P), X.shape[0],
                                    g.ctypes.data_as(F32P), C.byref(loss)))
        return g, float(loss.value)

    def train(self, X, y, epochs: int = 60, batch: int = 256, lr: float = 2e-3, seed: int = 0) -> float:
        X, y = _f32(X), _f32(y)
        loss = C.c_float()
        check(lib().bd_mlp_train(self.handle, X.ctypes.data_as(F32P), y.ctypes.data_as(F32P), X.shape[0], epochs,
                                 batch, C.c_float(lr), C.c_uint64(seed), C.byref(loss)))
        return float(loss.value)

    def close(self) -> None:
        if getattr(self, "handle", None):
            lib().bd_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """bd_server_*: continuous-batching service (persistent kernel fed while it runs)."""

    def __init__(self, slots: int = 0, ring_items: int = 0, memory_budget: int = 0, warps_per_block: int = 0,
                 blocks_per_sm: int = 0, item_subsets: int = 0, max_inflight_items: int = 0, order: int = 0,
                 publish_wait_ms: int = 0, test_withhold: int = 0, bottom_stage: int = 0):
        o = ServerOpts(slots, ring_items, memory_budget, warps_per_block, blocks_per_sm, item_subsets,
                       max_inflight_items, order, publish_wait_ms, test_withhold, bottom_stage)
        h = C.c_void_p()
        check(lib().bd_server_start(C.byref(o), C.byref(h)))
        self.handle = h

    def submit(self, A, coef=None, seed: int = 0, predicted_cost: float = 0.0) -> int:
        A = i64(A)
        n, m = A.shape
        c = _coef_array(coef, m)
        t = C.c_int64()
        check(lib().bd_server_submit(self.handle, ptr(A), n, m, ptr(c) if c is not None else None,
                                     C.c_uint64(seed), C.c_double(predicted_cost), C.byref(t)))
        return t.value

    def poll(self, wait_ms: int = 0):
        """(ticket, result dict, latency ms) of one finished request, or None."""
        out = DegreeOut()
        t = C.c_int64()
        lat = C.c_double()
        rc = lib().bd_server_poll(self.handle, wait_ms, C.byref(t), C.byref(out), C.byref(lat))
        if rc == 7:  # BD_ERR_STATE: nothing finished yet
            return None
        if rc != BD_OK:  # a failed request: the error carries its ticket
            err = BinodegError(rc, lib().bd_last_error().decode())
            err.ticket = t.value
            raise err
        return t.value, out.as_dict(), lat.value

    def stats(self) -> dict:
        s = ServerStats()
        check(lib().bd_server_stats_get(self.handle, C.byref(s)))
        return s.as_dict()

    def stop(self) -> None:
        if getattr(self, "handle", None):
            check(lib().bd_server_stop(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
