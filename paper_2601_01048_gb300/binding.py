"""Thin ctypes binding of the cufz C ABI (include/cufz.h).

The functions named cufz_* marshal arguments to the entry points of the same
name; every step of the checked execution runs in libcufz.so.  PyTorch only
supplies the device arena (a uint8 tensor) and the stream.  There is no CPU
path: if the library cannot be built or loaded, this module raises.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build_ext
from .gen import INPUT_DTYPE

# ---------------------------------------------------------------- constants
OK = 0
E_INVALID_ARG, E_INVALID_PROGRAM, E_NOMEM, E_BUSY, E_TIMEOUT, E_CUDA, E_NOT_FOUND, \
    E_NO_DEVICE, E_DEVICE_FAULT, E_IO, E_UNSUPPORTED = range(-1, -12, -1)
ST_OK, ST_VIOLATION, ST_INVALID_CONFIG, ST_LIMIT, ST_BAD_PROGRAM = range(5)
FL_BUDGET, FL_OVERFLOW, FL_NEW_COV, FL_PARTIAL = 1, 2, 4, 8
CF_KEEP_BITMAPS, CF_PLAIN_LAUNCH, CF_NO_PRUNE, CF_AUTO_RELEASE, CF_NO_GRAPH, CF_NO_DIGEST, \
    CF_JIT, CF_JIT_FAST_COMPILE, CF_PREX = 1, 2, 4, 8, 16, 32, 64, 128, 256
PREX_MAX_PLAN = 4096

RESULT_DTYPE = np.dtype([
    ("ticket", "<u8"), ("user_tag", "<u8"), ("status", "<i4"), ("flags", "<u4"),
    ("n_accesses", "<u8"), ("n_violations", "<u8"), ("first_key", "<u8"), ("digest", "<u8"),
    ("n_branch", "<u8"), ("n_threads", "<u8"), ("n_ops", "<u8"), ("n_records", "<u4"),
    ("n_edges", "<u4"), ("n_branch_folded", "<u8"),
])
assert RESULT_DTYPE.itemsize == 96

VIOLATION_DTYPE = np.dtype([
    ("block_lin", "<u4"), ("thread_lin", "<u4"), ("ordinal", "<u4"), ("site", "<u2"),
    ("buf", "u1"), ("kind", "u1"), ("width", "u1"), ("space", "u1"), ("cls", "u1"),
    ("pad0", "u1"), ("pad1", "<u4"), ("byte_off", "<i8"),
])
assert VIOLATION_DTYPE.itemsize == 32


class cufz_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("stream", ctypes.c_void_p), ("arena", ctypes.c_void_p),
                ("arena_bytes", ctypes.c_uint64), ("max_slots", ctypes.c_uint32),
                ("record_cap", ctypes.c_uint32), ("redzone", ctypes.c_uint32),
                ("iter_budget", ctypes.c_uint32), ("max_threads", ctypes.c_uint64),
                ("item_threads", ctypes.c_uint32), ("cta_threads", ctypes.c_uint32),
                ("n_lanes", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("jit_min_ctas", ctypes.c_uint32), ("lane_items", ctypes.c_uint32),
                ("autotune_cache", ctypes.c_char_p)]


class cufz_stats(ctypes.Structure):
    _fields_ = [("inputs_submitted", ctypes.c_uint64), ("inputs_completed", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("graph_launches", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("kernel_ms", ctypes.c_double),
                ("cta_threads", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("item_threads", ctypes.c_uint32), ("n_sms", ctypes.c_uint32),
                ("max_slots", ctypes.c_uint32), ("smem_bytes", ctypes.c_uint32),
                ("graph_failures", ctypes.c_uint32), ("last_cuda_error", ctypes.c_int32),
                ("overlapping_batch_pairs", ctypes.c_uint64),
                ("max_concurrent_batches", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class cufz_prog_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in (
        "n_ops_in", "n_ops_kept", "n_regs_in", "n_regs_alloc", "n_access_sites",
        "n_branch_sites", "n_loads_value_dead", "reserved")]


class cufz_campaign_config(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_uint32), ("corpus_cap", ctypes.c_uint32),
                ("bucket_cap", ctypes.c_uint32), ("hang_cap", ctypes.c_uint32),
                ("item_threads", ctypes.c_uint32), ("max_items", ctypes.c_uint32),
                ("seed", ctypes.c_uint64)]


class cufz_campaign_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint64), ("executed", ctypes.c_uint64),
                ("violating", ctypes.c_uint64), ("hang_execs", ctypes.c_uint64),
                ("new_coverage", ctypes.c_uint64)] + [
        (n, ctypes.c_uint32) for n in ("corpus", "buckets", "hangs", "corpus_dropped",
                                       "buckets_dropped", "hangs_dropped", "limit_children",
                                       "cycles_done")]


BUCKET_DTYPE = np.dtype([("key", "<u8"), ("first", "<u8"), ("hits", "<u4"), ("pad", "<u4"),
                         ("input", INPUT_DTYPE)])
assert BUCKET_DTYPE.itemsize == 152


class CufzError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {cufz_status_str(status)} ({status})")


_lib = None
_lock = threading.Lock()

EXPORTS = [
    "cufz_config_default", "cufz_arena_bytes", "cufz_validate_program", "cufz_prune_program",
    "cufz_status_str", "cufz_create", "cufz_destroy", "cufz_load_program", "cufz_submit_inputs",
    "cufz_poll_results", "cufz_get_records", "cufz_get_bitmap", "cufz_get_union",
    "cufz_new_epoch", "cufz_release", "cufz_sync", "cufz_get_stats", "cufz_reset_stats",
    "cufz_int32_peak", "cufz_compile_programs", "cufz_program_cuda", "cufz_compile_check",
    "cufz_run_noalloc", "cufz_set_program_path", "cufz_get_program_path", "cufz_autotune",
    "cufz_set_program_lanes", "cufz_get_program_lanes",
    "cufz_unload_program", "cufz_verify_prune", "cufz_prex_check",
    "cufz_prex_plan", "cufz_mutate_inputs", "cufz_mutate_children", "cufz_campaign_bytes",
    "cufz_campaign_create", "cufz_campaign_run", "cufz_campaign_sync", "cufz_campaign_get_stats",
    "cufz_campaign_corpus", "cufz_campaign_buckets", "cufz_campaign_hangs",
    "cufz_campaign_restore", "cufz_campaign_destroy",
]


def lib():
    """Loads libcufz.so, building it first if the sources are newer."""
    global _lib
    with _lock:
        if _lib is None:
            path = build_ext.build()
            L = ctypes.CDLL(path)
            vp, sz, u32, u64, i32 = (ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32,
                                     ctypes.c_uint64, ctypes.c_int32)
            P = ctypes.POINTER
            sig = {
                "cufz_config_default": (None, [P(cufz_config)]),
                "cufz_arena_bytes": (u64, [P(cufz_config), u32]),
                "cufz_validate_program": (i32, [vp, sz]),
                "cufz_prune_program": (i32, [vp, sz, vp, sz, P(sz), P(cufz_prog_stats)]),
                "cufz_status_str": (ctypes.c_char_p, [i32]),
                "cufz_create": (i32, [P(cufz_config), P(vp)]),
                "cufz_destroy": (i32, [vp]),
                "cufz_load_program": (i32, [vp, vp, sz, P(u32), P(cufz_prog_stats)]),
                "cufz_submit_inputs": (i32, [vp, vp, u32, P(u32), P(u64)]),
                "cufz_poll_results": (i32, [vp, vp, u32, P(u32), i32]),
                "cufz_get_records": (i32, [vp, u64, vp, u32, P(u32)]),
                "cufz_get_bitmap": (i32, [vp, u64, vp]),
                "cufz_get_union": (i32, [vp, vp]),
                "cufz_new_epoch": (i32, [vp]),
                "cufz_release": (i32, [vp, u64]),
                "cufz_sync": (i32, [vp, i32]),
                "cufz_get_stats": (i32, [vp, P(cufz_stats)]),
                "cufz_reset_stats": (i32, [vp]),
                "cufz_int32_peak": (i32, [i32, vp, P(ctypes.c_double)]),
                "cufz_compile_programs": (i32, [vp, ctypes.c_char_p, u32]),
                "cufz_program_cuda": (i32, [vp, sz, u32, ctypes.c_char_p, sz, P(sz)]),
                "cufz_compile_check": (i32, [vp, vp, u32, u32, ctypes.c_char_p, u32, P(sz)]),
                "cufz_run_noalloc": (i32, [vp, sz, vp, u32, u32, u32, vp, u32, vp, vp, vp]),
                "cufz_set_program_path": (i32, [vp, u32, u32]),
                "cufz_get_program_path": (i32, [vp, u32, P(u32)]),
                "cufz_set_program_lanes": (i32, [vp, u32, u32]),
                "cufz_get_program_lanes": (i32, [vp, u32, P(u32)]),
                "cufz_autotune": (i32, [vp, vp, u32, P(u32)]),
                "cufz_unload_program": (i32, [vp, u32]),
                "cufz_verify_prune": (i32, [vp, u32, vp, u32, P(u32)]),
                "cufz_prex_check": (i32, [vp, sz, vp, u32, P(u32)]),
                "cufz_prex_plan": (i32, [vp, sz, vp, u32, P(u32), u32, P(u32)]),
                "cufz_mutate_inputs": (i32, [vp, u32, vp, u32, P(u64)]),
                "cufz_mutate_children": (i32, [vp, u32, vp, u32, u64, u64]),
                "cufz_campaign_bytes": (u64, [P(cufz_campaign_config)]),
                "cufz_campaign_create": (i32, [vp, P(cufz_campaign_config), vp, u64, vp, u32, P(vp)]),
                "cufz_campaign_run": (i32, [vp, u32]),
                "cufz_campaign_sync": (i32, [vp, i32]),
                "cufz_campaign_get_stats": (i32, [vp, P(cufz_campaign_stats)]),
                "cufz_campaign_corpus": (i32, [vp, vp, vp, vp, u32, P(u32)]),
                "cufz_campaign_buckets": (i32, [vp, vp, u32, P(u32)]),
                "cufz_campaign_hangs": (i32, [vp, vp, vp, u32, P(u32)]),
                "cufz_campaign_restore": (i32, [vp, vp, vp, u32, vp, u32, vp, vp, u32,
                                                P(cufz_campaign_stats)]),
                "cufz_campaign_destroy": (i32, [vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(st: int, what: str) -> int:
    if st < 0:
        raise CufzError(st, what)
    return st


def _bytes_ptr(b: bytes):
    return ctypes.cast(ctypes.c_char_p(b), ctypes.c_void_p)


# ------------------------------------------------------------ ABI mirrors

def cufz_status_str(st: int) -> str:
    return lib().cufz_status_str(st).decode()


def cufz_config_default() -> cufz_config:
    c = cufz_config()
    lib().cufz_config_default(ctypes.byref(c))
    return c


def cufz_arena_bytes(cfg: cufz_config, n_slots: int) -> int:
    return lib().cufz_arena_bytes(ctypes.byref(cfg), n_slots)


def cufz_validate_program(prog: bytes) -> int:
    return lib().cufz_validate_program(_bytes_ptr(prog), len(prog))


def cufz_prune_program(prog: bytes) -> tuple[bytes, cufz_prog_stats]:
    cap = len(prog) + 64
    out = ctypes.create_string_buffer(cap)
    n = ctypes.c_size_t(0)
    st = cufz_prog_stats()
    _check(lib().cufz_prune_program(_bytes_ptr(prog), len(prog), out, cap, ctypes.byref(n),
                                    ctypes.byref(st)), "cufz_prune_program")
    return out.raw[: n.value], st


def cufz_create(cfg: cufz_config):
    h = ctypes.c_void_p()
    _check(lib().cufz_create(ctypes.byref(cfg), ctypes.byref(h)), "cufz_create")
    return h


def cufz_destroy(ctx) -> None:
    _check(lib().cufz_destroy(ctx), "cufz_destroy")


def cufz_load_program(ctx, prog: bytes) -> tuple[int, cufz_prog_stats]:
    pid = ctypes.c_uint32(0)
    st = cufz_prog_stats()
    _check(lib().cufz_load_program(ctx, _bytes_ptr(prog), len(prog), ctypes.byref(pid),
                                   ctypes.byref(st)), "cufz_load_program")
    return pid.value, st


def cufz_unload_program(ctx, program_id: int) -> None:
    _check(lib().cufz_unload_program(ctx, program_id), "cufz_unload_program")


def cufz_prex_check(prog: bytes, inp: np.ndarray, iter_budget: int = 0) -> bool:
    """Whether the corner threads of the input decide its verdict."""
    inp = np.ascontiguousarray(np.asarray(inp, dtype=INPUT_DTYPE).reshape(1))
    ok = ctypes.c_uint32(0)
    _check(lib().cufz_prex_check(_bytes_ptr(prog), len(prog), inp.ctypes.data, iter_budget,
                                 ctypes.byref(ok)), "cufz_prex_check")
    return bool(ok.value)


def cufz_prex_plan(prog: bytes, inp: np.ndarray, iter_budget: int = 0) -> np.ndarray | None:
    """The linear ids of the threads that decide the input's verdict, or None
    when no PREX rule applies."""
    inp = np.ascontiguousarray(np.asarray(inp, dtype=INPUT_DTYPE).reshape(1))
    n = ctypes.c_uint32(0)
    cap = 256
    while True:
        out = np.zeros(cap, dtype=np.uint32)
        st = lib().cufz_prex_plan(_bytes_ptr(prog), len(prog), inp.ctypes.data, iter_budget,
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), cap,
                                  ctypes.byref(n))
        if st == E_NOMEM:
            cap = int(n.value)
            continue
        _check(st, "cufz_prex_plan")
        return out[: n.value].copy() if n.value else None


def cufz_mutate_inputs(inputs: np.ndarray, n_bufs, rng_state: int) -> int:
    """Mutates the input records in place (they must be a contiguous
    INPUT_DTYPE array); returns the advanced generator state."""
    if inputs.dtype != INPUT_DTYPE or not inputs.flags["C_CONTIGUOUS"]:
        raise CufzError(E_INVALID_ARG, "cufz_mutate_inputs")
    nb = np.ascontiguousarray(n_bufs, dtype=np.uint8)
    st = ctypes.c_uint64(rng_state)
    _check(lib().cufz_mutate_inputs(inputs.ctypes.data, len(inputs), nb.ctypes.data, len(nb),
                                    ctypes.byref(st)), "cufz_mutate_inputs")
    return st.value


def cufz_mutate_children(inputs: np.ndarray, n_bufs, seed: int, round_: int) -> None:
    """Mutates child j of round `round_` in place from its own stream (the
    device campaign's draws)."""
    if inputs.dtype != INPUT_DTYPE or not inputs.flags["C_CONTIGUOUS"]:
        raise CufzError(E_INVALID_ARG, "cufz_mutate_children")
    nb = np.ascontiguousarray(n_bufs, dtype=np.uint8)
    _check(lib().cufz_mutate_children(inputs.ctypes.data, len(inputs), nb.ctypes.data, len(nb),
                                      seed & (2**64 - 1), round_), "cufz_mutate_children")


def cufz_campaign_bytes(cfg: cufz_campaign_config) -> int:
    return int(lib().cufz_campaign_bytes(ctypes.byref(cfg)))


def cufz_campaign_create(ctx, cfg: cufz_campaign_config, dev_mem: int, dev_bytes: int,
                         seeds: np.ndarray):
    seeds = np.ascontiguousarray(seeds, dtype=INPUT_DTYPE)
    out = ctypes.c_void_p()
    _check(lib().cufz_campaign_create(ctx, ctypes.byref(cfg), ctypes.c_void_p(dev_mem), dev_bytes,
                                      seeds.ctypes.data, len(seeds), ctypes.byref(out)),
           "cufz_campaign_create")
    return out


def cufz_campaign_run(camp, rounds: int) -> None:
    _check(lib().cufz_campaign_run(camp, rounds), "cufz_campaign_run")


def cufz_campaign_sync(camp, timeout_us: int = -1) -> None:
    _check(lib().cufz_campaign_sync(camp, timeout_us), "cufz_campaign_sync")


def cufz_campaign_get_stats(camp) -> cufz_campaign_stats:
    s = cufz_campaign_stats()
    _check(lib().cufz_campaign_get_stats(camp, ctypes.byref(s)), "cufz_campaign_get_stats")
    return s


def cufz_campaign_corpus(camp):
    """(inputs, favoured flags, pick counts) of the device corpus."""
    n = ctypes.c_uint32(0)
    _check(lib().cufz_campaign_corpus(camp, None, None, None, 0, ctypes.byref(n)),
           "cufz_campaign_corpus")
    k = int(n.value)
    inp = np.zeros(k, INPUT_DTYPE)
    fav = np.zeros(k, np.uint8)
    picks = np.zeros(k, np.uint32)
    _check(lib().cufz_campaign_corpus(camp, inp.ctypes.data, fav.ctypes.data, picks.ctypes.data, k,
                                      ctypes.byref(n)), "cufz_campaign_corpus")
    return inp, fav.astype(bool), picks


def cufz_campaign_buckets(camp) -> np.ndarray:
    n = ctypes.c_uint32(0)
    _check(lib().cufz_campaign_buckets(camp, None, 0, ctypes.byref(n)), "cufz_campaign_buckets")
    out = np.zeros(int(n.value), BUCKET_DTYPE)
    _check(lib().cufz_campaign_buckets(camp, out.ctypes.data, len(out), ctypes.byref(n)),
           "cufz_campaign_buckets")
    return out


def cufz_campaign_hangs(camp):
    n = ctypes.c_uint32(0)
    _check(lib().cufz_campaign_hangs(camp, None, None, 0, ctypes.byref(n)), "cufz_campaign_hangs")
    k = int(n.value)
    inp = np.zeros(k, INPUT_DTYPE)
    rounds = np.zeros(k, np.uint64)
    _check(lib().cufz_campaign_hangs(camp, inp.ctypes.data, rounds.ctypes.data, k, ctypes.byref(n)),
           "cufz_campaign_hangs")
    return inp, rounds


def cufz_campaign_restore(camp, favoured, picks, buckets: np.ndarray, hangs: np.ndarray,
                          hang_rounds, counters: cufz_campaign_stats) -> None:
    fav = np.ascontiguousarray(favoured, dtype=np.uint8)
    pk = np.ascontiguousarray(picks, dtype=np.uint32)
    bk = np.ascontiguousarray(buckets, dtype=BUCKET_DTYPE)
    hg = np.ascontiguousarray(hangs, dtype=INPUT_DTYPE)
    hr = np.ascontiguousarray(hang_rounds, dtype=np.uint64)
    _check(lib().cufz_campaign_restore(camp, fav.ctypes.data, pk.ctypes.data, len(fav),
                                       bk.ctypes.data, len(bk), hg.ctypes.data, hr.ctypes.data,
                                       len(hg), ctypes.byref(counters)), "cufz_campaign_restore")


def cufz_campaign_destroy(camp) -> None:
    _check(lib().cufz_campaign_destroy(camp), "cufz_campaign_destroy")


def cufz_verify_prune(ctx, program_id: int, inputs: np.ndarray) -> int:
    """Number of inputs whose outcome differs between the pruned and the
    unpruned program."""
    inputs = np.ascontiguousarray(inputs, dtype=INPUT_DTYPE)
    n = ctypes.c_uint32(0)
    _check(lib().cufz_verify_prune(ctx, program_id, inputs.ctypes.data, len(inputs), ctypes.byref(n)),
           "cufz_verify_prune")
    return n.value


def cufz_submit_inputs(ctx, inputs: np.ndarray) -> tuple[int, int, int]:
    """Returns (status, n_accepted, first_ticket); BUSY is not an error."""
    inputs = np.ascontiguousarray(inputs, dtype=INPUT_DTYPE)
    acc = ctypes.c_uint32(0)
    first = ctypes.c_uint64(0)
    st = lib().cufz_submit_inputs(ctx, inputs.ctypes.data, len(inputs), ctypes.byref(acc),
                                  ctypes.byref(first))
    if st < 0 and st != E_BUSY:
        raise CufzError(st, "cufz_submit_inputs")
    return st, acc.value, first.value


def cufz_poll_results(ctx, max_results: int, timeout_us: int = 0) -> np.ndarray:
    out = np.zeros(max_results, RESULT_DTYPE)
    n = ctypes.c_uint32(0)
    st = lib().cufz_poll_results(ctx, out.ctypes.data, max_results, ctypes.byref(n), timeout_us)
    if st < 0:
        raise CufzError(st, "cufz_poll_results")
    return out[: n.value]


def cufz_get_records(ctx, ticket: int, cap: int) -> np.ndarray:
    out = np.zeros(max(cap, 1), VIOLATION_DTYPE)
    n = ctypes.c_uint32(0)
    _check(lib().cufz_get_records(ctx, ticket, out.ctypes.data, cap, ctypes.byref(n)),
           "cufz_get_records")
    return out[: n.value]


def cufz_get_bitmap(ctx, ticket: int) -> np.ndarray:
    out = np.zeros(65536, np.uint8)
    _check(lib().cufz_get_bitmap(ctx, ticket, out.ctypes.data), "cufz_get_bitmap")
    return out


def cufz_get_union(ctx) -> np.ndarray:
    out = np.zeros(65536, np.uint8)
    _check(lib().cufz_get_union(ctx, out.ctypes.data), "cufz_get_union")
    return out


def cufz_new_epoch(ctx) -> None:
    _check(lib().cufz_new_epoch(ctx), "cufz_new_epoch")


def cufz_release(ctx, ticket: int) -> None:
    _check(lib().cufz_release(ctx, ticket), "cufz_release")


def cufz_sync(ctx, timeout_us: int = -1) -> None:
    _check(lib().cufz_sync(ctx, timeout_us), "cufz_sync")


def cufz_get_stats(ctx) -> cufz_stats:
    s = cufz_stats()
    _check(lib().cufz_get_stats(ctx, ctypes.byref(s)), "cufz_get_stats")
    return s


def cufz_reset_stats(ctx) -> None:
    _check(lib().cufz_reset_stats(ctx), "cufz_reset_stats")


def cufz_compile_programs(ctx) -> str:
    """Compiles the loaded programs for the compiled path; returns the log."""
    buf = ctypes.create_string_buffer(1 << 16)
    st = lib().cufz_compile_programs(ctx, buf, len(buf))
    log = buf.value.decode(errors="replace")
    if st < 0:
        raise CufzError(st, "cufz_compile_programs: " + log[-2000:])
    return log


def cufz_program_cuda(prog: bytes, flags: int = 0) -> str:
    n = ctypes.c_size_t(0)
    lib().cufz_program_cuda(_bytes_ptr(prog), len(prog), flags, None, 0, ctypes.byref(n))
    buf = ctypes.create_string_buffer(max(n.value, 1))
    _check(lib().cufz_program_cuda(_bytes_ptr(prog), len(prog), flags, buf, len(buf),
                                   ctypes.byref(n)), "cufz_program_cuda")
    return buf.value.decode()


def cufz_compile_check(progs: list[bytes], flags: int = 0) -> tuple[int, str, int]:
    """Runtime-compiles the module of `progs` without a device; returns
    (status, log, cubin bytes)."""
    bufs = [ctypes.create_string_buffer(p, len(p)) for p in progs]
    ptrs = (ctypes.c_void_p * max(len(progs), 1))(*[ctypes.cast(b, ctypes.c_void_p) for b in bufs])
    sizes = (ctypes.c_size_t * max(len(progs), 1))(*[len(p) for p in progs])
    log = ctypes.create_string_buffer(1 << 16)
    nb = ctypes.c_size_t(0)
    st = lib().cufz_compile_check(ctypes.cast(ptrs, ctypes.c_void_p),
                                  ctypes.cast(sizes, ctypes.c_void_p), len(progs), flags, log,
                                  len(log), ctypes.byref(nb))
    return st, log.value.decode(errors="replace"), nb.value


def cufz_run_noalloc(prog: bytes, inp, records_ptr: int, record_cap: int, bitmap_ptr: int,
                     result_ptr: int, flags: int = 0, redzone: int = 256,
                     iter_budget: int = 4096, stream: int = 0) -> None:
    """One input without device allocation (see include/cufz.h); the output
    pointers are raw addresses (device memory; the result may be host)."""
    rec = np.ascontiguousarray(np.asarray(inp, dtype=INPUT_DTYPE).reshape(1))
    _check(lib().cufz_run_noalloc(_bytes_ptr(prog), len(prog), rec.ctypes.data, flags, redzone,
                                  iter_budget, records_ptr or None, record_cap,
                                  bitmap_ptr or None, result_ptr, stream or None),
           "cufz_run_noalloc")


def cufz_set_program_path(ctx, program_id: int, compiled: bool) -> None:
    _check(lib().cufz_set_program_path(ctx, program_id, int(bool(compiled))),
           "cufz_set_program_path")


def cufz_get_program_path(ctx, program_id: int) -> bool:
    v = ctypes.c_uint32(0)
    _check(lib().cufz_get_program_path(ctx, program_id, ctypes.byref(v)), "cufz_get_program_path")
    return bool(v.value)


def cufz_set_program_lanes(ctx, program_id: int, lanes: int) -> None:
    _check(lib().cufz_set_program_lanes(ctx, program_id, lanes), "cufz_set_program_lanes")


def cufz_get_program_lanes(ctx, program_id: int) -> int:
    v = ctypes.c_uint32(0)
    _check(lib().cufz_get_program_lanes(ctx, program_id, ctypes.byref(v)), "cufz_get_program_lanes")
    return int(v.value)


def cufz_autotune(ctx, sample: np.ndarray) -> int:
    """Times each program of the sample compiled and interpreted, keeps the
    faster; returns how many programs stay compiled."""
    sample = np.ascontiguousarray(sample, dtype=INPUT_DTYPE)
    n = ctypes.c_uint32(0)
    _check(lib().cufz_autotune(ctx, sample.ctypes.data, len(sample), ctypes.byref(n)),
           "cufz_autotune")
    return n.value


def cufz_int32_peak(device: int = 0, stream: int = 0) -> float:
    v = ctypes.c_double(0)
    _check(lib().cufz_int32_peak(device, ctypes.c_void_p(stream), ctypes.byref(v)),
           "cufz_int32_peak")
    return v.value


# ------------------------------------------------------------ convenience

class Engine:
    """One cufz context over a torch-allocated arena on one device."""

    def __init__(self, device: int = 0, arena_bytes: int | None = None, max_slots: int = 0,
                 record_cap: int = 4096, flags: int = CF_KEEP_BITMAPS, redzone: int = 256,
                 iter_budget: int = 4096, max_threads: int = 1 << 31, cta_threads: int = 256,
                 item_threads: int = 0, n_lanes: int = 4, ctas_per_sm: int = 0,
                 jit_min_ctas: int = 0, autotune_cache: str | None = None, lane_items: int = 0):
        import torch

        if not torch.cuda.is_available():
            raise CufzError(E_NO_DEVICE, "Engine")
        self.device = device
        cfg = cufz_config_default()
        cfg.device = device
        cfg.flags = flags
        cfg.record_cap = record_cap
        cfg.redzone = redzone
        cfg.iter_budget = iter_budget
        cfg.max_threads = max_threads
        cfg.cta_threads = cta_threads
        cfg.item_threads = item_threads
        cfg.n_lanes = n_lanes
        cfg.ctas_per_sm = ctas_per_sm
        cfg.jit_min_ctas = jit_min_ctas
        cfg.lane_items = lane_items
        self._tune_path = autotune_cache.encode() if autotune_cache else None
        cfg.autotune_cache = self._tune_path
        cfg.max_slots = max_slots
        if arena_bytes is None:
            arena_bytes = cufz_arena_bytes(cfg, max_slots or 1024)
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=f"cuda:{device}")
        self.stream = torch.cuda.current_stream(device)
        cfg.arena = self.arena.data_ptr()
        cfg.arena_bytes = int(arena_bytes)
        cfg.stream = self.stream.cuda_stream
        self.cfg = cfg
        self.record_cap = record_cap
        self.ctx = cufz_create(cfg)
        self.prog_stats: list[cufz_prog_stats] = []

    def close(self) -> None:
        if getattr(self, "ctx", None):
            cufz_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def load(self, prog: bytes) -> int:
        pid, st = cufz_load_program(self.ctx, prog)
        self.prog_stats.append(st)
        return pid

    def run(self, inputs: np.ndarray, records: bool = True, bitmaps: bool = True,
            release: bool = True, timeout_s: float = 600.0):
        """Submits every input (resubmitting as slots free up), waits for all
        results and returns (results sorted by ticket order of `inputs`,
        list of record arrays or None, bitmaps [n, 65536] or None)."""
        import time

        inputs = np.ascontiguousarray(inputs, dtype=INPUT_DTYPE)
        n = len(inputs)
        res = np.zeros(n, RESULT_DTYPE)
        recs = [None] * n if records else None
        bms = np.zeros((n, 65536), np.uint8) if bitmaps else None
        ticket_to_idx = {}
        pos = 0
        got = 0
        t_end = time.time() + timeout_s
        while got < n:
            if pos < n:
                st, acc, first = cufz_submit_inputs(self.ctx, inputs[pos:])
                for k in range(acc):
                    ticket_to_idx[first + k] = pos + k
                pos += acc
            out = cufz_poll_results(self.ctx, 4096, 200 if pos < n else 20000)
            for r in out:
                i = ticket_to_idx.pop(int(r["ticket"]))
                res[i] = r
                t = int(r["ticket"])
                if records:
                    nr = int(r["n_records"])
                    recs[i] = (cufz_get_records(self.ctx, t, nr) if nr
                               else np.zeros(0, VIOLATION_DTYPE))
                if bitmaps:
                    bms[i] = cufz_get_bitmap(self.ctx, t)
                if release:
                    cufz_release(self.ctx, t)
                got += 1
            if time.time() > t_end:
                raise CufzError(E_TIMEOUT, "Engine.run")
        return res, recs, bms

    def union(self) -> np.ndarray:
        return cufz_get_union(self.ctx)

    def new_epoch(self) -> None:
        cufz_new_epoch(self.ctx)

    def stats(self) -> cufz_stats:
        return cufz_get_stats(self.ctx)
