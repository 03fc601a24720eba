"""ctypes binding of libbinodeg.so: argument marshalling only (every step runs in the library)."""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbinodeg.so")

BD_OK, BD_ERR_ARG, BD_ERR_OVERFLOW, BD_ERR_TIES, BD_ERR_CUDA, BD_ERR_TIMEOUT, BD_ERR_NOMEM, BD_ERR_STATE = range(8)
BD_FLAG_DEGENERATE, BD_FLAG_INT128, BD_FLAG_INCONSISTENT = 1, 2, 4
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
                ("force_int128", C.c_int32), ("reserved", C.c_int32 * 3)]


I64P = C.POINTER(C.c_int64)
I32P = C.POINTER(C.c_int32)
U8P = C.POINTER(C.c_uint8)

# name -> (restype, argtypes); every symbol include/binodeg.h declares
SIGNATURES = {
    "bd_last_error": (C.c_char_p, []),
    "bd_set_stream": (C.c_int, [C.c_void_p]),
    "bd_degree": (C.c_int, [I64P, C.c_int32, C.c_int32, I64P, C.c_uint64, C.POINTER(DegreeOut)]),
    "bd_reduce": (C.c_int, [I64P, C.c_int32, C.c_int32, I64P, I64P, I64P]),
    "bd_volume": (C.c_int, [I64P, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(VolumeOut)]),
    "bd_volume_lifted": (C.c_int, [I64P, I64P, C.c_int32, C.c_int32, C.POINTER(VolumeOut)]),
    "bd_classify": (C.c_int, [I64P, I64P, C.c_int32, C.c_int32, U8P, C.c_int32, I32P, I64P]),
    "bd_plan_create": (C.c_int, [I64P, C.c_int32, C.c_int32, C.POINTER(PlanOpts), C.POINTER(C.c_void_p)]),
    "bd_plan_launch": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int32, C.c_void_p]),
    "bd_plan_read": (C.c_int, [C.c_void_p, C.POINTER(VolumeOut)]),
    "bd_plan_volume": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(VolumeOut)]),
    "bd_plan_info": (C.c_int, [C.c_void_p, I64P]),
    "bd_plan_destroy": (C.c_int, [C.c_void_p]),
    "bd_host_volume_lifted": (C.c_int, [I64P, I64P, C.c_int32, C.c_int32, C.c_int32, C.POINTER(VolumeOut)]),
    "bd_volume_noalloc": (C.c_int, [I64P, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(VolumeOut)]),
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
