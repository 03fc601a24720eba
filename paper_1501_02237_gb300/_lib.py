"""ctypes binding of libbinodeg.so: argument marshalling only (every step runs in the library)."""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbinodeg.so")

BD_OK, BD_ERR_ARG, BD_ERR_OVERFLOW, BD_ERR_TIES, BD_ERR_CUDA, BD_ERR_TIMEOUT, BD_ERR_NOMEM, BD_ERR_STATE = range(8)
BD_FLAG_DEGENERATE, BD_FLAG_INT128, BD_FLAG_INCONSISTENT, BD_FLAG_PIVOT = 1, 2, 4, 8
KMAX, NMAX = 14, 64

ERROR_NAMES = {0: "BD_OK", 1: "BD_ERR_ARG", 2: "BD_ERR_OVERFLOW", 3: "BD_ERR_TIES", 4: "BD_ERR_CUDA",
               5: "BD_ERR_TIMEOUT", 6: "BD_ERR_NOMEM", 7: "BD_ERR_STATE"}


class BinodegError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class VolumeOut(C.Structure):
    _fields_ = [("nvol_lo", C.c_uint64), ("nvol_hi", C.c_uint64), ("cells", C.c_uint64),
                ("singular", C.c_uint64), ("ties", C.c_uint64), ("subsets", C.c_uint64),
                ("relifts", C.c_int32), ("flags", C.c_int32), ("max_abs_coord", C.c_int32),
                ("bound_bits", C.c_int32)]

    @property
    def nvol(self) -> int:
        return (int(self.nvol_hi) << 64) | int(self.nvol_lo)

    def as_dict(self):
        return dict(nvol=self.nvol, cells=int(self.cells), singular=int(self.singular), ties=int(self.ties),
                    subsets=int(self.subsets), relifts=int(self.relifts), flags=int(self.flags),
                    max_abs_coord=int(self.max_abs_coord), bound_bits=int(self.bound_bits))


class MixedOut(C.Structure):
    _fields_ = [("mv_lo", C.c_uint64), ("mv_hi", C.c_uint64), ("cells", C.c_uint64), ("singular", C.c_uint64),
                ("ties", C.c_uint64), ("tuples", C.c_uint64), ("relifts", C.c_int32), ("flags", C.c_int32),
                ("bound_bits", C.c_int32), ("reserved", C.c_int32), ("device_ms", C.c_double)]

    def as_dict(self):
        return dict(mv=(int(self.mv_hi) << 64) | int(self.mv_lo), cells=int(self.cells),
                    singular=int(self.singular), ties=int(self.ties), tuples=int(self.tuples),
                    relifts=int(self.relifts), flags=int(self.flags), bound_bits=int(self.bound_bits),
                    device_ms=float(self.device_ms))


class DegreeOut(C.Structure):
    _fields_ = [("degree_lo", C.c_uint64), ("degree_hi", C.c_uint64), ("nvol_lo", C.c_uint64),
                ("nvol_hi", C.c_uint64), ("torsion", C.c_uint64), ("rank", C.c_int32), ("dim", C.c_int32),
                ("consistent", C.c_int32), ("relifts", C.c_int32), ("subsets", C.c_uint64),
                ("cells", C.c_uint64), ("flags", C.c_int32), ("max_abs_coord", C.c_int32)]

    def as_dict(self):
        return dict(degree=(int(self.degree_hi) << 64) | int(self.degree_lo),
                    nvol=(int(self.nvol_hi) << 64) | int(self.nvol_lo), torsion=int(self.torsion),
                    rank=int(self.rank), dim=int(self.dim), consistent=bool(self.consistent),
                    relifts=int(self.relifts), subsets=int(self.subsets), cells=int(self.cells),
                    flags=int(self.flags), max_abs_coord=int(self.max_abs_coord))


class PlanOpts(C.Structure):
    _fields_ = [("warps_per_block", C.c_int32), ("blocks_per_sm", C.c_int32), ("item_subsets", C.c_int64),
                ("force_int128", C.c_int32), ("bottom_stage", C.c_int32), ("reserved", C.c_int32 * 2)]


class HostOpts(C.Structure):
    _fields_ = [("threads", C.c_int32), ("force_int128", C.c_int32), ("item_subsets", C.c_uint64),
                ("team_width", C.c_int32), ("shard", C.c_int32), ("shards", C.c_int32), ("bottom_stage", C.c_int32)]


class BatchOpts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("warps_per_block", C.c_int32), ("item_factor", C.c_int32),
                ("use_graph", C.c_int32), ("autotune", C.c_int32), ("bottom_stage", C.c_int32),
                ("cost", C.POINTER(C.c_float)), ("reserved", C.c_int32 * 4)]


class BatchStats(C.Structure):
    _fields_ = [("host_ms", C.c_double), ("gpu_ms", C.c_double), ("wall_ms", C.c_double), ("tune_ms", C.c_double),
                ("subsets", C.c_int64), ("items", C.c_int64), ("launches", C.c_int32),
                ("warps_per_block", C.c_int32), ("item_factor", C.c_int32), ("relifted", C.c_int32)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class ServerOpts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("ring_items", C.c_int32), ("memory_budget", C.c_int64),
                ("warps_per_block", C.c_int32), ("blocks_per_sm", C.c_int32), ("item_subsets", C.c_int64),
                ("max_inflight_items", C.c_int64), ("order", C.c_int32), ("publish_wait_ms", C.c_int32),
                ("test_withhold", C.c_int32), ("bottom_stage", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("relifted", C.c_int64), ("launches", C.c_int64),
                ("ring_items", C.c_int64), ("slots", C.c_int32), ("blocks", C.c_int32),
                ("warps_per_block", C.c_int32), ("waiting", C.c_int32), ("routed", C.c_int64),
                ("peak_resident", C.c_int32), ("faults", C.c_int32)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class PeakOut(C.Structure):
    _fields_ = [("lane_ops", C.c_double), ("ms", C.c_double), ("lane_ops_per_s", C.c_double),
                ("sm_cycles", C.c_double), ("sm_mhz", C.c_double), ("lane_ops_per_sm_clk", C.c_double),
                ("sms", C.c_int32), ("blocks", C.c_int32), ("threads_per_block", C.c_int32), ("kind", C.c_int32)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


BD_FEATURES = 16
BD_MLP_PARAMS = 5313
I64P = C.POINTER(C.c_int64)
I32P = C.POINTER(C.c_int32)
F32P = C.POINTER(C.c_float)
U8P = C.POINTER(C.c_uint8)

# name -> (restype, argtypes); every symbol include/binodeg.h declares
SIGNATURES = {
    "bd_last_error": (C.c_char_p, []),
    "bd_set_stream": (C.c_int, [C.c_void_p]),
    "bd_inject_alloc_failure": (C.c_int, [C.c_int32]),
    "bd_degree": (C.c_int, [I64P, C.c_int32, C.c_int32, I64P, C.c_uint64, C.POINTER(DegreeOut)]),
    "bd_reduce": (C.c_int, [I64P, C.c_int32, C.c_int32, I64P, I64P, I64P]),
    "bd_volume": (C.c_int, [I64P, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(VolumeOut)]),
    "bd_volume_lifted": (C.c_int, [I64P, I64P, C.c_int32, C.c_int32, C.POINTER(VolumeOut)]),
    "bd_classify": (C.c_int, [I64P, I64P, C.c_int32, C.c_int32, U8P, C.c_int32, I32P, I64P]),
    "bd_plan_create": (C.c_int, [I64P, C.c_int32, C.c_int32, C.POINTER(PlanOpts), C.POINTER(C.c_void_p)]),
    "bd_plan_launch": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int32, C.c_void_p]),
    "bd_plan_launch_shard": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]),
    "bd_plan_read": (C.c_int, [C.c_void_p, C.POINTER(VolumeOut)]),
    "bd_plan_volume": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(VolumeOut)]),
    "bd_plan_info": (C.c_int, [C.c_void_p, I64P]),
    "bd_plan_destroy": (C.c_int, [C.c_void_p]),
    "bd_host_volume_lifted": (C.c_int, [I64P, I64P, C.c_int32, C.c_int32, C.POINTER(HostOpts), C.POINTER(VolumeOut)]),
    "bd_cells": (C.c_int, [I64P, C.c_int32, C.c_int32, C.c_uint64, C.c_int64, U8P, I64P, I64P, I64P,
                           C.POINTER(C.c_int64), C.POINTER(VolumeOut)]),
    "bd_host_cells": (C.c_int, [I64P, I64P, C.c_int32, C.c_int32, C.c_int64, U8P, I64P, I64P, I64P,
                                C.POINTER(C.c_int64)]),
    "bd_start_solutions": (C.c_int, [I64P, C.c_int32, C.c_int32, C.c_uint64, C.c_uint64, C.c_int64, C.c_void_p,
                                     C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "bd_host_start_solutions": (C.c_int, [I64P, I64P, C.c_int32, C.c_int32, C.c_uint64, C.c_int64, C.c_void_p,
                                          C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "bd_volume_noalloc": (C.c_int, [I64P, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(VolumeOut)]),
    "bd_mixed_volume": (C.c_int, [I64P, I32P, C.c_int32, C.c_uint64, C.POINTER(MixedOut)]),
    "bd_volume_pivot": (C.c_int, [I64P, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(VolumeOut),
                                  C.POINTER(C.c_double)]),
    "bd_pivot_force_wide": (C.c_int, [C.c_int32]),
    "bd_host_volume_pivot": (C.c_int, [I64P, I64P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(VolumeOut),
                                       C.POINTER(C.c_uint64), C.c_int64]),
    "bd_degree_pivot": (C.c_int, [I64P, C.c_int32, C.c_int32, I64P, C.c_uint64, C.POINTER(DegreeOut)]),
    "bd_mixed_volume_lifted": (C.c_int, [I64P, I32P, C.c_int32, I64P, C.c_int32, C.POINTER(MixedOut), I32P,
                                         C.c_int64, I64P]),
    "bd_host_mixed_volume_lifted": (C.c_int, [I64P, I32P, C.c_int32, I64P, C.c_int32, C.c_int32, C.c_int32,
                                              C.c_int32, C.POINTER(MixedOut), I32P, C.c_int64, I64P]),
    "bd_issue_peak": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.POINTER(PeakOut)]),
    "bd_batch_create": (C.c_int, [C.POINTER(C.c_void_p)]),
    "bd_batch_add": (C.c_int, [C.c_void_p, I64P, C.c_int32, C.c_int32, I64P, C.c_uint64, I32P]),
    "bd_batch_add_points": (C.c_int, [C.c_void_p, I64P, C.c_int32, C.c_int32, C.c_uint64, I32P]),
    "bd_batch_size": (C.c_int, [C.c_void_p, I32P]),
    "bd_batch_prepare": (C.c_int, [C.c_void_p, C.c_int32]),
    "bd_batch_features": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "bd_batch_run": (C.c_int, [C.c_void_p, C.POINTER(BatchOpts), C.POINTER(BatchStats)]),
    "bd_batch_result": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(DegreeOut), C.POINTER(C.c_uint64)]),
    "bd_batch_destroy": (C.c_int, [C.c_void_p]),
    "bd_server_start": (C.c_int, [C.POINTER(ServerOpts), C.POINTER(C.c_void_p)]),
    "bd_server_submit": (C.c_int, [C.c_void_p, I64P, C.c_int32, C.c_int32, I64P, C.c_uint64, C.c_double,
                                   C.POINTER(C.c_int64)]),
    "bd_server_poll": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64), C.POINTER(DegreeOut),
                                 C.POINTER(C.c_double)]),
    "bd_server_stats_get": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "bd_server_stop": (C.c_int, [C.c_void_p]),
    "bd_mlp_create": (C.c_int, [C.c_uint64, C.POINTER(C.c_void_p)]),
    "bd_mlp_destroy": (C.c_int, [C.c_void_p]),
    "bd_mlp_get_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "bd_mlp_set_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "bd_mlp_predict": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_int32, C.POINTER(C.c_float)]),
    "bd_mlp_gradient": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int32,
                                  C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "bd_mlp_train": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int32, C.c_int32,
                               C.c_int32, C.c_float, C.c_uint64, C.POINTER(C.c_float)]),
}

_lib = None


def lib() -> C.CDLL:
    """The loaded library.  Raises if it has not been built: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1501_02237_gb300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != BD_OK:
        raise BinodegError(rc, lib().bd_last_error().decode())


def i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def ptr(a: np.ndarray, t=I64P):
    return a.ctypes.data_as(t)
