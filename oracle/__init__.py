"""CPU oracle for the SVT track-fitting chain (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
CPU-baseline leg are the only users; the product path (the CUDA library and
its binding) never imports this package.  The C source (svt_oracle.c) states
what is computed and which passage of the paper (arXiv:1312.0917, Sec. II and
II-A) or which reading each step follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "svt_oracle.c"), os.path.join(_HERE, "svt_oracle_mt.c")]
_LIB = os.path.join(_HERE, "libsvt_oracle.so")

OK, E_BADWORD, E_TRUNCATED, E_LIMIT, E_NOMEM = 0, -2, -3, -4, -8

ROAD_DTYPE = np.dtype([
    ("event", np.uint32), ("road", np.uint32), ("wedge", np.int32),
    ("barrel", np.int32), ("excl", np.int32), ("curv", np.int32),
    ("phi", np.int32), ("n", np.int32, (5,)), ("coord", np.uint16, (5, 8)),
], align=True)
assert ROAD_DTYPE.itemsize == 128

FIT_DTYPE = np.dtype([
    ("event", np.uint32), ("road", np.uint32), ("comb", np.uint32),
    ("p", np.int32, (3,)), ("chi2", np.int64), ("coord", np.uint16, (5,)),
    ("pad", np.uint16), ("pass", np.int32),
], align=True)
assert FIT_DTYPE.itemsize == 48


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP for the event-parallel driver)
    into oracle/libsvt_oracle.so."""
    deps = _SRCS + [os.path.join(_HERE, "svt_oracle.h")]
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(map(os.path.getmtime, deps)):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fopenmp",
                               "-fPIC", "-shared", "-o", tmp] + _SRCS)
        os.replace(tmp, _LIB)
    return _LIB


class _Times(C.Structure):
    _fields_ = [("unpack", C.c_double), ("fit", C.c_double), ("warrior", C.c_double),
                ("wall", C.c_double), ("threads", C.c_int32), ("pad", C.c_int32)]


class _Consts(C.Structure):
    _fields_ = [("F", C.c_void_p), ("q", C.c_void_p), ("C", C.c_void_p),
                ("k", C.c_void_p), ("n_sets", C.c_uint32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        sz = C.c_size_t
        _lib.orc_unpack.argtypes = [C.c_void_p, sz, C.c_void_p, sz, C.POINTER(sz),
                                    C.POINTER(sz), C.POINTER(sz)]
        _lib.orc_fit_all.argtypes = [C.c_void_p, sz, C.POINTER(_Consts), C.c_int64,
                                     C.POINTER(C.c_void_p), C.POINTER(sz)]
        _lib.orc_chi2_all.argtypes = [C.c_void_p, sz, C.POINTER(_Consts),
                                      C.POINTER(C.c_void_p), C.POINTER(sz)]
        _lib.orc_run.argtypes = [C.c_void_p, sz, C.POINTER(_Consts), C.c_int64, C.c_int,
                                 C.POINTER(C.c_void_p), C.POINTER(sz)]
        _lib.orc_run_mt.argtypes = [C.c_void_p, sz, C.POINTER(_Consts), C.c_int64, C.c_int, C.c_int,
                                    C.POINTER(C.c_void_p), C.POINTER(sz), C.POINTER(_Times)]
        _lib.orc_free.argtypes = [C.c_void_p]
        for f in ("orc_unpack", "orc_fit_all", "orc_chi2_all", "orc_run", "orc_run_mt"):
            getattr(_lib, f).restype = C.c_int
    return _lib


class _Held:
    """Keeps the numpy constant arrays alive while C holds their pointers."""

    def __init__(self, consts: dict):
        self.F = np.ascontiguousarray(consts["F"], dtype=np.int16)
        self.q = np.ascontiguousarray(consts["q"], dtype=np.int32)
        self.C = np.ascontiguousarray(consts["C"], dtype=np.int16)
        self.k = np.ascontiguousarray(consts["k"], dtype=np.int32)
        assert self.F.shape[1:] == (3, 6) and self.C.shape[1:] == (3, 6)
        n = self.F.shape[0]
        assert self.q.shape == (n, 3) and self.k.shape == (n, 3) and self.C.shape[0] == n
        self.s = _Consts(self.F.ctypes.data, self.q.ctypes.data, self.C.ctypes.data,
                         self.k.ctypes.data, n)


def _words(words) -> np.ndarray:
    return np.ascontiguousarray(words, dtype=np.uint32)


def unpack(words):
    """-> (status, roads structured array, n_events, err_pos)"""
    w = _words(words)
    nr, ne, ep = C.c_size_t(), C.c_size_t(), C.c_size_t()
    cap = len(w) // 3 + 1
    roads = np.zeros(cap, dtype=ROAD_DTYPE)
    rc = lib().orc_unpack(w.ctypes.data, len(w), roads.ctypes.data, cap,
                          C.byref(nr), C.byref(ne), C.byref(ep))
    return rc, roads[:min(nr.value, cap)], ne.value, ep.value


def _take(ptr: C.c_void_p, n: int, dtype) -> np.ndarray:
    if not ptr.value or n == 0:
        if ptr.value:
            lib().orc_free(ptr)
        return np.zeros(0, dtype=dtype)
    buf = (C.c_char * (n * np.dtype(dtype).itemsize)).from_address(ptr.value)
    arr = np.frombuffer(buf, dtype=dtype).copy()
    lib().orc_free(ptr)
    return arr


def fit_all(words, consts: dict, cut: int = 0):
    """Every combination before the cut -> (status, FIT_DTYPE array)."""
    w, h = _words(words), _Held(consts)
    p, n = C.c_void_p(), C.c_size_t()
    rc = lib().orc_fit_all(w.ctypes.data, len(w), C.byref(h.s), int(cut), C.byref(p), C.byref(n))
    return rc, _take(p, n.value, FIT_DTYPE)


def chi2_all(words, consts: dict):
    """chi2 of every combination -> (status, int64 array)."""
    w, h = _words(words), _Held(consts)
    p, n = C.c_void_p(), C.c_size_t()
    rc = lib().orc_chi2_all(w.ctypes.data, len(w), C.byref(h.s), C.byref(p), C.byref(n))
    return rc, _take(p, n.value, np.int64)


def run(words, consts: dict, cut: int, warrior: int = 1):
    """The whole chain -> (status, FIT_DTYPE array of survivors).

    warrior: 0 pairwise definition, 1 triple projections, -1 none."""
    w, h = _words(words), _Held(consts)
    p, n = C.c_void_p(), C.c_size_t()
    rc = lib().orc_run(w.ctypes.data, len(w), C.byref(h.s), int(cut), int(warrior),
                       C.byref(p), C.byref(n))
    return rc, _take(p, n.value, FIT_DTYPE)


def run_mt(words, consts: dict, cut: int, warrior: int = 1, threads: int = 0):
    """The whole chain with the events spread over host threads (OpenMP, one
    event per thread at a time): -> (status, survivors, times) where times =
    {"threads", "unpack_s", "fit_s", "warrior_s", "wall_s"} (fit and warrior
    summed over the threads).  Output identical to run()."""
    w, h = _words(words), _Held(consts)
    p, n, t = C.c_void_p(), C.c_size_t(), _Times()
    rc = lib().orc_run_mt(w.ctypes.data, len(w), C.byref(h.s), int(cut), int(warrior), int(threads),
                          C.byref(p), C.byref(n), C.byref(t))
    times = {"threads": t.threads, "unpack_s": t.unpack, "fit_s": t.fit, "warrior_s": t.warrior,
             "wall_s": t.wall}
    return rc, _take(p, n.value, FIT_DTYPE), times
