"""ctypes wrapper of the CPU oracle (cufz_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg.  The engine (paper_2601_01048_gb300) never
imports it.

The oracle runs every thread of every block serially (the paper's collapsing
transform, Sec. 4.1, Listings 1-2), checks every access exactly and counts
AFL-style edges (Sec. 2.1); see the header of cufz_oracle.c for the full
definition it computes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cufz_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "libcufz_oracle.so")

RESULT_DTYPE = np.dtype([
    ("status", "<i4"), ("flags", "<u4"), ("n_accesses", "<u8"), ("n_violations", "<u8"),
    ("first_key", "<u8"), ("digest", "<u8"), ("n_branch", "<u8"), ("n_threads", "<u8"),
    ("n_records", "<u4"), ("n_edges", "<u4"), ("n_ops", "<u8"),
])
assert RESULT_DTYPE.itemsize == 72

RECORD_DTYPE = np.dtype([
    ("block_lin", "<u4"), ("thread_lin", "<u4"), ("ordinal", "<u4"), ("site", "<u2"),
    ("buf", "u1"), ("kind", "u1"), ("width", "u1"), ("space", "u1"), ("cls", "u1"),
    ("pad0", "u1"), ("pad1", "<u4"), ("byte_off", "<i8"),
])
assert RECORD_DTYPE.itemsize == 32

ST_OK, ST_VIOLATION, ST_INVALID_CONFIG, ST_LIMIT = 0, 1, 2, 3
FL_BUDGET, FL_OVERFLOW, FL_NEW_COV = 1, 2, 4
(CLS_NONE, CLS_UNDERFLOW_RZ, CLS_OVERFLOW_RZ, CLS_OTHER_ALLOC, CLS_WILD, CLS_DIV_ZERO,
 CLS_USE_AFTER_FREE, CLS_DOUBLE_FREE, CLS_INVALID_FREE) = range(9)


class Opts(ctypes.Structure):
    _fields_ = [("redzone", ctypes.c_uint32), ("iter_budget", ctypes.c_uint32),
                ("max_threads", ctypes.c_uint64)]


DEFAULT_REDZONE = 256
DEFAULT_BUDGET = 4096
DEFAULT_MAX_THREADS = 1 << 31

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle with the host C compiler (plain -O2)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            vp, sz, u64, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int
            L.orc_load.restype = vp
            L.orc_load.argtypes = [ctypes.c_char_p, sz, ctypes.POINTER(i32)]
            L.orc_free.argtypes = [vp]
            L.orc_n_access_sites.argtypes = [vp]
            L.orc_run.argtypes = [vp, vp, ctypes.POINTER(Opts), vp, vp, u64, vp, vp]
            L.orc_run.restype = i32
            L.orc_run_batch.argtypes = [vp, u64, vp, u64, ctypes.POINTER(Opts), vp, vp, u64, vp,
                                        vp, i32]
            L.orc_run_batch.restype = i32
            L.orc_fmix32.argtypes = [ctypes.c_uint32]
            L.orc_fmix32.restype = ctypes.c_uint32
            L.orc_bucket.argtypes = [u64]
            L.orc_bucket.restype = ctypes.c_uint8
            _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


class Program:
    """A decoded program held by the oracle."""

    def __init__(self, data: bytes):
        err = ctypes.c_int(0)
        self.data = bytes(data)
        self.h = lib().orc_load(self.data, len(self.data), ctypes.byref(err))
        self.err = err.value
        if not self.h:
            raise OracleError(f"invalid program ({self.err})")

    @property
    def n_access_sites(self) -> int:
        return lib().orc_n_access_sites(self.h)

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.orc_free(h)
            self.h = None


def validate(data: bytes) -> int:
    """0 if the oracle accepts the program, else its negative error code."""
    err = ctypes.c_int(0)
    h = lib().orc_load(bytes(data), len(data), ctypes.byref(err))
    if h:
        lib().orc_free(h)
    return err.value


def opts(redzone: int = DEFAULT_REDZONE, iter_budget: int = DEFAULT_BUDGET,
         max_threads: int = DEFAULT_MAX_THREADS) -> Opts:
    return Opts(redzone, iter_budget, max_threads)


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def run(program: Program | bytes, inp, o: Opts | None = None, rec_cap: int = 1 << 16,
        bitmap: bool = True, snapshot: np.ndarray | None = None):
    """Runs one input record; returns (result, records, bitmap-or-None)."""
    if not isinstance(program, Program):
        program = Program(program)
    o = o or opts()
    inp = np.ascontiguousarray(np.asarray(inp).reshape(1))
    res = np.zeros(1, RESULT_DTYPE)
    recs = np.zeros(max(rec_cap, 1), RECORD_DTYPE)
    bm = np.zeros(65536, np.uint8) if bitmap else None
    snap = None if snapshot is None else np.ascontiguousarray(snapshot, dtype=np.uint8)
    e = lib().orc_run(program.h, _ptr(inp), ctypes.byref(o), _ptr(res), _ptr(recs), rec_cap,
                      _ptr(bm), _ptr(snap))
    if e:
        raise OracleError(f"orc_run failed ({e})")
    r = res[0]
    return r, recs[: int(r["n_records"])].copy(), bm


def run_batch(programs: list, inputs: np.ndarray, o: Opts | None = None, rec_cap: int = 0,
              bitmaps: bool = False, snapshot: np.ndarray | None = None,
              threads: int | None = None):
    """Runs every input (inputs[i].program_id indexes `programs`) over a pool
    of host threads; returns (results, records[n, rec_cap] or None,
    bitmaps[n, 65536] or None)."""
    progs = [p if isinstance(p, Program) else Program(p) for p in programs]
    handles = (ctypes.c_void_p * len(progs))(*[p.h for p in progs])
    o = o or opts()
    inputs = np.ascontiguousarray(inputs)
    n = len(inputs)
    res = np.zeros(n, RESULT_DTYPE)
    recs = np.zeros((n, rec_cap), RECORD_DTYPE) if rec_cap else None
    bms = np.zeros((n, 65536), np.uint8) if bitmaps else None
    snap = None if snapshot is None else np.ascontiguousarray(snapshot, dtype=np.uint8)
    threads = threads or os.cpu_count() or 1
    e = lib().orc_run_batch(ctypes.cast(handles, ctypes.c_void_p), len(progs), _ptr(inputs), n,
                            ctypes.byref(o), _ptr(res), _ptr(recs), rec_cap, _ptr(bms),
                            _ptr(snap), threads)
    if e:
        raise OracleError(f"orc_run_batch failed ({e})")
    return res, recs, bms


def fmix32(x: int) -> int:
    return lib().orc_fmix32(x & 0xFFFFFFFF)


def bucket(n: int) -> int:
    return lib().orc_bucket(n)
