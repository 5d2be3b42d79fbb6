"""ctypes binding of libsvt.so: the C ABI of include/svt.h, argument
marshalling only.  Every step of the track-fitting chain runs in the
library's CUDA kernels; there is no CPU fallback, and a missing library is
an error.

Device buffers are passed as raw pointers (an int, or any object with
``data_ptr()`` such as a torch tensor); streams as a ``cudaStream_t`` value
(an int, or an object with ``cuda_stream``); None is the legacy default
stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsvt.so")

OK, E_INVAL, E_BADWORD, E_TRUNCATED, E_LIMIT = 0, -1, -2, -3, -4
E_CAPACITY, E_CUDA, E_TIMEOUT, E_STATE = -5, -6, -7, -9
PLAIN, PERSISTENT = 0, 1

CONST_DTYPE = np.dtype([("F", np.int16, (3, 6)), ("q", np.int32, (3,)),
                        ("C", np.int16, (3, 6)), ("k", np.int32, (3,))])
TRACK_DTYPE = np.dtype([("event", np.uint32), ("road", np.uint16), ("comb", np.uint16),
                        ("p", np.int32, (3,)), ("pad", np.uint32), ("chi2", np.int64),
                        ("hits", np.uint64)], align=True)
ROAD_DTYPE = np.dtype([("event", np.uint32), ("road", np.uint16), ("curv", np.int16),
                       ("phi", np.int16), ("wedge", np.uint8), ("barrel", np.uint8),
                       ("excl", np.uint8), ("n", np.uint8, (5,)), ("pad", np.uint8, (2,)),
                       ("coord", np.uint16, (5, 8))], align=True)
assert CONST_DTYPE.itemsize == 96 and TRACK_DTYPE.itemsize == 40 and ROAD_DTYPE.itemsize == 100


class Limits(C.Structure):
    _fields_ = [("max_words", C.c_uint64), ("max_events", C.c_uint32),
                ("max_roads", C.c_uint32), ("max_tracks", C.c_uint64),
                ("hash_slots", C.c_uint32), ("pad", C.c_uint32),
                ("max_combinations", C.c_uint64)]


class Stats(C.Structure):
    _fields_ = [("n_events", C.c_uint64), ("n_roads", C.c_uint64),
                ("n_combinations", C.c_uint64), ("n_passing", C.c_uint64),
                ("n_tracks", C.c_uint64), ("status", C.c_int32), ("n_groups", C.c_uint32),
                ("error_word", C.c_uint64), ("phase_ns", C.c_uint64 * 6)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "phase_ns"}
        d["phase_ns"] = list(self.phase_ns)
        return d


class Launch(C.Structure):
    _fields_ = [("block", C.c_int32), ("blocks_per_sm", C.c_int32), ("small_n4", C.c_int32),
                ("run_roads", C.c_int32), ("max_ctas", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class TunePoint(C.Structure):
    _fields_ = [("cfg", Launch), ("ms", C.c_float)]


class ServerConfig(C.Structure):
    _fields_ = [("n_slots", C.c_uint32), ("ctas_per_sm", C.c_uint32), ("max_ctas", C.c_uint32),
                ("mode", C.c_int32), ("max_words", C.c_uint64), ("max_events", C.c_uint32),
                ("max_roads", C.c_uint32), ("max_tracks", C.c_uint64), ("hash_slots", C.c_uint32),
                ("pad", C.c_uint32), ("max_combinations", C.c_uint64)]


class ServerResult(C.Structure):
    _fields_ = [("request_id", C.c_uint64), ("status", C.c_int32), ("pad", C.c_uint32),
                ("n_tracks", C.c_uint64), ("n_events", C.c_uint64), ("n_combinations", C.c_uint64),
                ("latency_ns", C.c_uint64)]


# every entry point of include/svt.h with its argument types
SIGNATURES = {
    "svt_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(Limits)]),
    "svt_destroy": (None, [C.c_void_p]),
    "svt_load_constants": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32, C.c_int64, C.c_void_p]),
    "svt_unpack": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "svt_fit_events": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "svt_get_tracks": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t),
                                 C.c_void_p]),
    "svt_get_roads": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t),
                                C.c_void_p]),
    "svt_get_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats), C.c_void_p]),
    "svt_set_launch": (C.c_int, [C.c_void_p, C.POINTER(Launch)]),
    "svt_set_track_output": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "svt_get_launch": (C.c_int, [C.c_void_p, C.POINTER(Launch)]),
    "svt_use_graph": (C.c_int, [C.c_void_p, C.c_int]),
    "svt_debug_wait": (C.c_int, [C.c_void_p, C.c_uint32, C.c_int]),
    "svt_last_launch_count": (C.c_int, [C.c_void_p]),
    "svt_strerror": (C.c_char_p, [C.c_int]),
    "svt_measure_int_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double)]),
    "svt_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_uint32, C.POINTER(C.c_uint32),
                                C.c_void_p]),
    "svt_run_static": (C.c_int, [C.c_void_p, C.c_size_t, C.c_void_p, C.c_uint32, C.c_int64, C.c_void_p,
                                  C.c_size_t, C.POINTER(C.c_size_t), C.c_void_p]),
    "svt_server_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(ServerConfig), C.c_void_p,
                                    C.c_uint32, C.c_int64]),
    "svt_server_destroy": (None, [C.c_void_p]),
    "svt_server_get_config": (C.c_int, [C.c_void_p, C.POINTER(ServerConfig)]),
    "svt_server_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_uint64)]),
    "svt_server_wait": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(ServerResult)]),
    "svt_server_take": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]),
}

_lib = None


class SvtError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = lib().svt_strerror(code).decode() if _lib is not None else str(code)
        super().__init__("%s: %s (%d)" % (what, msg, code))


def lib() -> C.CDLL:
    """Load libsvt.so (built by paper_1312_0917_gb300.build); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libsvt.so is not built: run "
                              "`python -m paper_1312_0917_gb300.build` (or __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def ptr(x) -> int | None:
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x)


def stream_ptr(s) -> int | None:
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def check(code: int, what: str) -> int:
    if code != OK:
        raise SvtError(code, what)
    return code


def pack_constants(consts: dict) -> np.ndarray:
    """dict(F, q, C, k) with shapes (360,3,6), (360,3), (360,3,6), (360,3)
    -> array of svt_const_set records."""
    n = consts["F"].shape[0]
    out = np.zeros(n, dtype=CONST_DTYPE)
    out["F"], out["q"] = consts["F"], consts["q"]
    out["C"], out["k"] = consts["C"], consts["k"]
    return out


class Context:
    """One svt_ctx (one stream at a time)."""

    def __init__(self, device: int = 0, **limits):
        self._h = C.c_void_p()
        lim = Limits(**limits)
        check(lib().svt_create(C.byref(self._h), device, C.byref(lim)), "svt_create")

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().svt_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_constants(self, consts: dict, cut: int, stream=None):
        sets = pack_constants(consts)
        check(lib().svt_load_constants(self._h, sets.ctypes.data, len(sets), int(cut),
                                       stream_ptr(stream)), "svt_load_constants")

    def unpack(self, d_words, n_words: int, stream=None) -> int:
        return lib().svt_unpack(self._h, ptr(d_words), n_words, stream_ptr(stream))

    def fit_events(self, mode: int = PERSISTENT, stream=None) -> int:
        return lib().svt_fit_events(self._h, mode, stream_ptr(stream))

    def get_tracks(self, out=None, cap: int | None = None, stream=None):
        """Returns (status, tracks).  Without `out`, copies to a new host array."""
        n = C.c_size_t()
        if out is None:
            st = lib().svt_get_tracks(self._h, None, 0, C.byref(n), stream_ptr(stream))
            if st not in (OK, E_CAPACITY) or (st == E_CAPACITY and n.value == 0):
                return st, np.zeros(0, dtype=TRACK_DTYPE)
            host = np.zeros(n.value, dtype=TRACK_DTYPE)
            st = lib().svt_get_tracks(self._h, host.ctypes.data, n.value, C.byref(n),
                                      stream_ptr(stream))
            return st, host
        st = lib().svt_get_tracks(self._h, ptr(out), cap, C.byref(n), stream_ptr(stream))
        return st, n.value

    def set_track_output(self, host=None, cap: int = 0):
        """Tracks written straight into `host` (page-locked memory: a pinned
        torch tensor or its data pointer), or back to the device buffer (None)."""
        check(lib().svt_set_track_output(self._h, ptr(host) if host is not None else None, cap),
              "svt_set_track_output")

    def get_roads(self, stream=None):
        n = C.c_size_t()
        st = lib().svt_get_roads(self._h, None, 0, C.byref(n), stream_ptr(stream))
        if st not in (OK, E_CAPACITY) or (st == E_CAPACITY and n.value == 0):
            return st, np.zeros(0, dtype=ROAD_DTYPE)
        host = np.zeros(n.value, dtype=ROAD_DTYPE)
        st = lib().svt_get_roads(self._h, host.ctypes.data, n.value, C.byref(n),
                                 stream_ptr(stream))
        return st, host

    def get_stats(self, stream=None) -> dict:
        s = Stats()
        check(lib().svt_get_stats(self._h, C.byref(s), stream_ptr(stream)), "svt_get_stats")
        return s.as_dict()

    def set_launch(self, block: int = 0, blocks_per_sm: int = 0, small_n4: int = 0, run_roads: int = 0,
                   max_ctas: int = 0):
        cfg = Launch(block, blocks_per_sm, small_n4, run_roads, max_ctas)
        check(lib().svt_set_launch(self._h, C.byref(cfg)), "svt_set_launch")

    def get_launch(self) -> dict:
        cfg = Launch()
        check(lib().svt_get_launch(self._h, C.byref(cfg)), "svt_get_launch")
        return cfg.as_dict()

    def autotune(self, reps: int = 5, stream=None) -> list:
        """Measure every launch configuration on the bound batch and keep the
        fastest; returns [({block, blocks_per_sm, small_n4, run_roads, max_ctas}, ms), ...]."""
        pts = (TunePoint * 512)()
        n = C.c_uint32()
        check(lib().svt_autotune(self._h, reps, pts, 512, C.byref(n), stream_ptr(stream)), "svt_autotune")
        return [(p.cfg.as_dict(), p.ms) for p in pts[:n.value]]

    def use_graph(self, enable: bool = True):
        check(lib().svt_use_graph(self._h, int(enable)), "svt_use_graph")

    def debug_wait(self, wait_limit_us: int = 0, skip_arrival: int = 0):
        """skip_arrival: 0 none, 1 block 0 leaves before the first grid
        barrier, 2 after the fit stage (next persistent launch only)."""
        check(lib().svt_debug_wait(self._h, wait_limit_us, int(skip_arrival)), "svt_debug_wait")

    def last_launch_count(self) -> int:
        return lib().svt_last_launch_count(self._h)


class Server:
    """A serving runtime (svt_server): continuous batching of independent
    requests over device slots.  Words and results are host numpy arrays."""

    def __init__(self, consts: dict, cut: int, device: int = 0, mode: int = PERSISTENT, **config):
        self._h = C.c_void_p()
        cfg = ServerConfig(mode=mode, **config)
        sets = pack_constants(consts)
        check(lib().svt_server_create(C.byref(self._h), device, C.byref(cfg), sets.ctypes.data,
                                      len(sets), int(cut)), "svt_server_create")

    def config(self) -> dict:
        cfg = ServerConfig()
        check(lib().svt_server_get_config(self._h, C.byref(cfg)), "svt_server_get_config")
        return {f: getattr(cfg, f) for f, _ in cfg._fields_ if f != "pad"}

    def submit(self, words) -> int:
        w = np.ascontiguousarray(words, dtype=np.uint32)
        rid = C.c_uint64()
        check(lib().svt_server_submit(self._h, w.ctypes.data, len(w), C.byref(rid)), "svt_server_submit")
        return rid.value

    def wait(self, timeout_us: int = -1):
        """Next completed request as a dict, or None on timeout."""
        r = ServerResult()
        st = lib().svt_server_wait(self._h, int(timeout_us), C.byref(r))
        if st == E_TIMEOUT:
            return None
        check(st, "svt_server_wait")
        return {f: getattr(r, f) for f, _ in r._fields_ if f != "pad"}

    def take(self, request_id: int, n_tracks: int) -> np.ndarray:
        out = np.zeros(n_tracks, dtype=TRACK_DTYPE)
        n = C.c_size_t()
        check(lib().svt_server_take(self._h, request_id, out.ctypes.data, n_tracks, C.byref(n)),
              "svt_server_take")
        return out[:n.value]

    def close(self):
        if self._h:
            lib().svt_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_int_peak(device: int = 0) -> dict:
    """svt_measure_int_peak: integer operations per second of the device
    -> {"imad": ..., "iadd": ..., "mixed": ...}."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    check(lib().svt_measure_int_peak(device, C.byref(a), C.byref(b), C.byref(c)), "svt_measure_int_peak")
    return {"imad": a.value, "iadd": b.value, "mixed": c.value}
