#!/usr/bin/env python3
"""Benchmark of the cufz checked-execution engine on GB300.

Default workload (the random-program configuration): 32 seeded random access
programs of 20-200 int32 ops, 256 inputs each, 2D grids of up to 256 x 256
blocks of 16 x 16 threads.  A step is one pass of the whole hot path (load
already done; admission, staging, interpretation of every test thread,
bounds checks, record compaction, coverage, finalize) over one batch of
inputs, run as one persistent launch in a CUDA graph.

Prints one JSON line (rank 0): checked thread-accesses per second, timed with
CUDA events on the engine's stream (value) and end to end through the C ABI
with host input records and host result records (e2e), with the roofline of
the dominant kernel (the compiled-program kernel) against the INT32 issue
rate and the CPU oracle's rate on a bounded sample.  `--impl reference` times
the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "checked thread-accesses/sec"
UNIT = "checked accesses/s"
# INT32 issue peak derived from the unit counts: 152 SMs x 4 sub-partitions x
# 32 lanes per clock, at the maximum SM clock (MEASURED_PEAKS sm_max_mhz).
N_SM_GB300 = 152
LANES_PER_SM = 128
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the dominant kernel on a whole workload, from one ncu capture (the command
# is in profiles/), keyed by a hash of that kernel: the device headers of the
# compiled path (code without comments) and the CUDA the loader emits for the
# workload's programs, with the module's launch shape.  Once the kernel
# changes the figure no longer applies and is reported as null.
TRAFFIC_HEADERS = ("jit_kernel.cuh", "jit_launch.cuh", "device_common.cuh", "layout.h")
TRAFFIC_BYTES: dict[str, tuple[str, int, str]] = {
    "c2": ("338961bf148fdf72", 53_855_488 + 1_491_637_248,
           "lane mapping {1: 29, 2: 2, 4: 1}, item_threads 65536"),
}


def _code_only(text: str) -> str:
    """The source without comments, blank lines and runs of whitespace
    (string and character literals kept), so that comment and layout edits
    keep the hash."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c and text[j] != "\n":
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            i = text.find("\n", i)
            i = n if i < 0 else i
        elif text.startswith("/*", i):
            i = text.find("*/", i + 2)
            i = n if i < 0 else i + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(" ".join(l.split()) for l in "".join(out).split("\n") if l.strip())


def kernel_key(programs, cta_threads: int = 256, min_ctas: int = 3, lanes=None) -> str:
    """Hash of the compiled module a workload runs: device headers, the
    emitted code of each program, each program's lane mapping (all 1 when
    not given), the module's launch shape."""
    from paper_2601_01048_gb300 import binding as B

    h = hashlib.sha256()
    for name in TRAFFIC_HEADERS:
        with open(os.path.join(ROOT, "paper_2601_01048_gb300", "csrc", name), encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
    for k, p in enumerate(programs):
        h.update(_code_only(B.cufz_program_cuda(p)).encode())
        if lanes and lanes[k] != 1:
            h.update(f"lanes[{k}]={lanes[k]}".encode())
    h.update(f"cta_threads={cta_threads} min_ctas={min_ctas}".encode())
    return h.hexdigest()[:16]


def measured_traffic(args, wl_key, per_step: int, n_all: int, code_key: str):
    """DRAM bytes per launch if captured for this workload and this code (the
    kernel key without the lane mapping: a mapping and an item size decide
    which lane runs which test thread, while the bytes a launch reads and
    writes are its inputs, bitmaps, records and results), with the settings
    of the capture."""
    entry = TRAFFIC_BYTES.get(wl_key)
    if (entry is None or per_step != n_all or args.plain or args.path != "jit"
            or args.cta_threads not in (0, 256) or args.jit_min_ctas not in (0, 3)):
        return None, None
    return (entry[1], entry[2]) if entry[0] == code_key else (None, None)


# algorithmic integer ops per checked access and per branch evaluation
OPS_PER_ACCESS = 5
OPS_PER_BRANCH = 4


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--workload", default="c2",
                    choices=["c1", "c2", "c3", "c4", "c5", "affine", "guard2d", "div", "heap",
                             "barrier", "barrier_live", "campaign"])
    ap.add_argument("--prex", action="store_true",
                    help="partial representative execution: inputs with a PREX plan run only its threads")
    ap.add_argument("--rate", type=float, default=50000.0, help="c5: offered inputs/s")
    ap.add_argument("--lanes", type=int, default=4, help="c5: batches that may overlap (1-8)")
    ap.add_argument("--duration", type=float, default=2.0, help="c5: seconds of arrivals")
    ap.add_argument("--inputs-per-step", type=int, default=0, help="0: the whole workload")
    ap.add_argument("--plain", action="store_true", help="one kernel launch per input")
    ap.add_argument("--path", default="jit", choices=["jit", "interp"],
                    help="compiled programs (default) or the bytecode interpreter")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cta-threads", type=int, default=256)
    ap.add_argument("--jit-min-ctas", type=int, default=0)
    ap.add_argument("--jit-fast-compile", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the load-time path choice (for profiling a single launch)")
    ap.add_argument("--item-threads", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="persistent CTAs per SM (0: occupancy)")
    ap.add_argument("--tune-file", default="",
                    help="autotune cache file: tuned into when absent, loaded (no tuning) when "
                         "present, so that a later run (a profiler's) gets the same kernels")
    ap.add_argument("--no-sub", action="store_true",
                    help="default run: leave out the other configurations' sub-records")
    return ap.parse_args()


# ------------------------------------------------------------------ workload

def workload(name: str, rank: int = 0):
    from paper_2601_01048_gb300 import gen

    if name == "c1":
        return ("c1: 1 guarded 1D program, 1000 inputs, grid 64 x 128",
                [gen.c1_program()], gen.c1_inputs(1000), 1 << 15)
    if name == "c2":
        progs = gen.c2_programs()
        return ("c2: 32 random access programs (20-200 ops) x 256 inputs, 2D grids up to "
                "256x256 blocks of 16x16", progs, gen.c2_inputs(progs, 256), 4096)
    if name == "c3":
        return ("c3: 4096 inputs over 16 C1-family programs, 1-65536 blocks x 32-1024 threads",
                gen.c3_programs(), gen.c3_inputs(4096), 4096)
    if name == "affine":
        return ("affine: 4096 inputs over 16 unguarded affine-access programs (PREX's class), "
                "1-65536 blocks x 32-1024 threads", gen.affine_programs(), gen.affine_inputs(4096), 4096)
    if name == "guard2d":
        return ("guard2d: 4096 inputs over 16 bounds-guarded 2D matrix programs, grids up to "
                "256 x 256 blocks of 8x8 to 32x32", gen.guard2d_programs(), gen.guard2d_inputs(4096),
                4096)
    if name == "div":
        return ("div: 8192 inputs over 16 programs with signed divisions (zero divisors for some "
                "threads and inputs), blocks of 16x4, grids up to 4096 blocks",
                gen.div_programs(), gen.div_inputs(8192, max_blocks=4096), 4096)
    if name == "heap":
        return ("heap: 8192 inputs over 16 programs on the per-thread device heap (use after "
                "free, double and invalid frees, heap bounds), blocks of 16x2, grids up to 4096 "
                "blocks", gen.heap_programs(), gen.heap_inputs(8192, max_blocks=4096), 4096)
    if name == "barrier_live":
        return ("barrier_live: 8192 inputs over 16 programs whose performed shared stores reach "
                "checks (barriers kept; the block-serial form), blocks of 16-32 threads, grids "
                "up to 4096 blocks", gen.barrier_programs(live=True),
                gen.barrier_inputs(8192, max_blocks=4096), 4096)
    if name == "barrier":
        return ("barrier: 8192 inputs over 16 programs with performed shared stores in 2-4 "
                "barrier phases that BarrierElimination removes, blocks of 16-32 threads, grids "
                "up to 4096 blocks", gen.barrier_programs(),
                gen.barrier_inputs(8192, max_blocks=4096), 4096)
    if name == "c5":
        progs = gen.c5_programs()
        return ("c5: mutated inputs over 64 resident programs", progs,
                gen.c5_stream(progs, gen.c5_corpus(progs), 4096), 1024)
    progs = gen.c4_programs()
    return ("c4: 16 branch-heavy programs (<=64 data-dependent sites), 16384 inputs, "
            "1-1024 blocks x 256", progs, gen.c4_inputs(16384), 1024)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.device), "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = max(mx, float(p[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ dist

def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def allreduce_max(pg, x: float, device) -> float:
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(pg, x: float, device) -> float:
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle

def oracle_rate(progs, inputs, seconds: float, seed: int = 11):
    """Runs the CPU oracle over a seeded random order of the inputs, in chunks
    over all host cores, until `seconds` have passed; returns (accesses/s,
    inputs/s, cores, n_inputs, accesses)."""
    from oracle import oracle

    cores = os.cpu_count() or 1
    P = [oracle.Program(p) for p in progs]
    order = np.random.default_rng(seed).permutation(len(inputs))
    done_acc = 0
    done_in = 0
    t0 = time.perf_counter()
    pos = 0
    chunk = max(cores, 1)
    while pos < len(order) and time.perf_counter() - t0 < seconds:
        sel = inputs[order[pos: pos + chunk]]
        res, _, _ = oracle.run_batch(P, sel, threads=cores)
        done_acc += int(res["n_accesses"].sum())
        done_in += len(sel)
        pos += chunk
    dt = time.perf_counter() - t0
    return done_acc / dt, done_in / dt, cores, done_in, done_acc, dt


# ------------------------------------------------------------------ engine arm

# Per workload, the autotuner's choices of this process (an autotune cache
# file): the first context of a workload tunes, later ones load the choices.
TUNE_FILES: dict[str, str] = {}
TUNED: set[str] = set()


def tune_file(key: str):
    """(cache path, whether it already holds this workload's choices)."""
    import tempfile

    if key not in TUNE_FILES:
        fd, path = tempfile.mkstemp(prefix=f"cufz_tune_{key}_", suffix=".txt")
        os.close(fd)
        os.unlink(path)
        TUNE_FILES[key] = path
        return path, False
    return TUNE_FILES[key], True


def autotune_or_load(B, E, key, sample, n_programs):
    """Runs the autotuner for the workload's first context; later contexts
    got the same choices from the cache at load.  Returns the number of
    programs on the compiled path."""
    if key not in TUNED:
        TUNED.add(key)
        return B.cufz_autotune(E.ctx, sample)
    return sum(int(B.cufz_get_program_path(E.ctx, p)) for p in range(n_programs))


def measure_engine(args, wl_key, plain, steps, warmup, per_step_arg, rank, world, local, pg,
                   prex=False, cta_threads=None):
    """One workload through the engine: warm-up steps, then `steps` timed
    steps (each a whole batch: submit host input records, poll host result
    records).  Returns the JSON line's fields (without the CPU baseline)."""
    import torch

    from paper_2601_01048_gb300 import binding as B

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl_name, progs, inputs, cap = workload(wl_key, rank)
    n_all = len(inputs)
    per_step = per_step_arg or n_all
    cta = args.cta_threads if cta_threads is None else cta_threads
    flags = B.CF_AUTO_RELEASE | B.CF_KEEP_BITMAPS | (B.CF_PLAIN_LAUNCH if plain else 0)
    if prex:
        flags |= B.CF_PREX
    if args.path == "jit":
        flags |= B.CF_JIT | (B.CF_JIT_FAST_COMPILE if args.jit_fast_compile else 0)
    tune_path = None
    if args.path == "jit" and not args.no_autotune:
        tune_path = args.tune_file or tune_file(wl_key)[0]
        if args.tune_file and os.path.exists(args.tune_file):
            TUNED.add(wl_key)                       # its choices load with the programs
    E = B.Engine(device=local, max_slots=per_step, record_cap=cap, flags=flags,
                 cta_threads=cta, item_threads=args.item_threads, n_lanes=2,
                 jit_min_ctas=args.jit_min_ctas, ctas_per_sm=args.ctas_per_sm,
                 autotune_cache=tune_path)
    for p in progs:
        E.load(p)
    tuned = None
    if tune_path:
        # the project's autotuner: per program, compiled vs interpreted on a
        # sample of that program's inputs (up to eight per program)
        sample = np.concatenate([inputs[inputs["program_id"] == p][:8]
                                 for p in np.unique(inputs["program_id"])])
        tuned = autotune_or_load(B, E, wl_key, sample, len(progs))
    lanes = None
    prog_lanes = [B.cufz_get_program_lanes(E.ctx, p) for p in range(len(progs))]
    if tune_path:
        # the autotuner's lane mappings: compiled programs per test threads per lane
        lanes = {}
        for p in range(len(progs)):
            if B.cufz_get_program_path(E.ctx, p):
                k = str(prog_lanes[p])
                lanes[k] = lanes.get(k, 0) + 1
    n_batches = (n_all + per_step - 1) // per_step
    batches = [inputs[(k * per_step) % n_all: (k * per_step) % n_all + per_step]
               for k in range(n_batches)]

    def step(k):
        batch = batches[k % n_batches]
        pos, got = 0, 0
        acc = np.zeros(len(batch), B.RESULT_DTYPE)
        lat = []
        t_sub = time.perf_counter()
        while got < len(batch):
            if pos < len(batch):
                st, n_acc, _ = B.cufz_submit_inputs(E.ctx, batch[pos:])
                pos += n_acc
            out = B.cufz_poll_results(E.ctx, len(batch), 2000)
            now = time.perf_counter()
            if len(out):
                acc[got: got + len(out)] = out
                lat.extend([now - t_sub] * len(out))
                got += len(out)
        return acc, lat

    for k in range(warmup):
        step(k)
    torch.cuda.synchronize(dev)
    barrier(pg)
    B.cufz_reset_stats(E.ctx)
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    tot = dict(acc=0, inputs=0, ops=0, br=0, folded=0, viol=0, threads=0, partial=0,
               bug_inputs=0)
    lats = []
    h2d = d2h = 0
    for k in range(steps):
        res, lat = step(warmup + k)
        lats += lat
        tot["acc"] += int(res["n_accesses"].sum())
        tot["inputs"] += len(res)
        tot["ops"] += int(res["n_ops"].sum())
        tot["br"] += int(res["n_branch"].sum())
        tot["folded"] += int(res["n_branch_folded"].sum())
        tot["viol"] += int(res["n_violations"].sum())
        tot["threads"] += int(res["n_threads"].sum())
        tot["partial"] += int(((res["flags"] & B.FL_PARTIAL) != 0).sum())
        tot["bug_inputs"] += int((res["status"] == B.ST_VIOLATION).sum())
        h2d += len(res) * 128
        d2h += len(res) * 96
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    barrier(pg)
    clk = clocks.stop()
    st = B.cufz_get_stats(E.ctx)
    kernel_s = st.kernel_ms / 1e3
    wall_s = t1 - t0
    kernel_s_max = allreduce_max(pg, kernel_s, dev)
    wall_s_max = allreduce_max(pg, wall_s, dev)
    acc_all = allreduce_sum(pg, tot["acc"], dev)
    inputs_all = allreduce_sum(pg, tot["inputs"], dev)
    launches = int(st.kernel_launches)
    E.close()

    peaks = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = int(st.n_sms) or N_SM_GB300
    peak_ops = n_sm * LANES_PER_SM * sm_max * 1e6
    alg_ops = tot["ops"] + OPS_PER_ACCESS * tot["acc"] + OPS_PER_BRANCH * tot["br"]
    # the same work with each closed-form loop-head evaluation credited as a
    # share of the one edge update it took instead of an update of its own
    alg_ops_folded = alg_ops - OPS_PER_BRANCH * tot["folded"]
    achieved = alg_ops / kernel_s if kernel_s > 0 else 0.0
    s = max(steps, 1)
    key = kernel_key(progs, int(st.cta_threads), args.jit_min_ctas or 3, prog_lanes)
    code_key = kernel_key(progs, int(st.cta_threads), args.jit_min_ctas or 3)
    traffic, traffic_with = ((None, None) if plain else
                             measured_traffic(args, wl_key, per_step, n_all, code_key))
    return {
        "metric": METRIC,
        "value": acc_all / kernel_s_max if kernel_s_max > 0 else 0.0,
        "unit": UNIT,
        "n_gpus": world,
        "steps": steps,
        "warmup": warmup,
        "ms_per_step": kernel_s_max * 1e3 / s,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic (seeded programs and fuzz inputs)",
        "config": {
            "workload": wl_name,
            "inputs_per_step": per_step,
            "path": ("plain one launch per input" if plain else
                     "persistent kernel in a CUDA graph"),
            "engine": ("programs compiled to sm_103a at load or interpreted, chosen per program "
                       "by the autotuner" if args.path == "jit" else "bytecode interpreter"),
            "cta_threads": int(st.cta_threads),
            "jit_min_ctas": args.jit_min_ctas or 3,
            "programs_compiled": tuned,
            "lane_mapping": lanes,
            "ctas_per_sm": int(st.ctas_per_sm),
            "item_threads": int(st.item_threads),
            "record_cap": cap,
            "l2": "no flush: every step writes one 64 KiB bitmap per input (>= 64 MiB per "
                  "step, 512 MiB for the default workload) plus edge counters and records, "
                  "and reads no input twice within a step",
            "parallelism": f"replicas x{world}",
        },
        "inputs_per_s": inputs_all / kernel_s_max if kernel_s_max > 0 else 0.0,
        "violating_inputs_per_step": tot["bug_inputs"] // s,
        "prex": ({"partial_inputs_per_step": tot["partial"] // s,
                  "note": "partial inputs ran only their PREX plan's threads (the corners, or for "
                          "guarded launches the corners of the cells the guards cut the grid "
                          "into); their verdict is the full grid's, their accesses are the "
                          "planned threads'"}
                 if prex else None),
        "test_threads_per_step": tot["threads"] // s,
        "violations_per_step": tot["viol"] // s,
        "roofline": {
            "bound": "alu",
            "achieved": achieved / 1e12,
            "peak": peak_ops / 1e12,
            "unit": "Tops/s (int32 lane-ops)",
            "frac": achieved / peak_ops,
            "traffic": traffic,
            "traffic_captured_with": traffic_with,
            "kernel_key": key,
            "code_key": code_key,
            "peak_source": f"{n_sm} SMs x 128 int32 lanes/clk x {sm_max:.0f} MHz (derived)",
            "alg_ops_per_step": alg_ops // s,
            "loop_heads_folded_per_step": tot["folded"] // s,
            "frac_folded_heads_uncredited": (alg_ops_folded / kernel_s / peak_ops
                                             if kernel_s > 0 else 0.0),
        },
        "e2e": {
            "value": acc_all / wall_s_max if wall_s_max > 0 else 0.0,
            "unit": UNIT,
            "h2d_bytes_per_step": h2d // s,
            "d2h_bytes_per_step": d2h // s,
            "latency_ms": {"p50": 1e3 * float(np.percentile(lats, 50)) if lats else None,
                           "p99": 1e3 * float(np.percentile(lats, 99)) if lats else None,
                           "kind": "submit-to-poll within a whole-batch step"},
        },
        "gpu_launches": launches,
        "graph_launches": int(st.graph_launches),
        "graph_failures": int(st.graph_failures),
        "last_cuda_error": int(st.last_cuda_error),
        "clocks": clk,
    }


def sub_of(line):
    """The compact form of a measured line kept inside the default line."""
    r = line["roofline"]
    return {
        "workload": line["config"]["workload"], "path": line["config"]["path"],
        "value": line["value"], "unit": line["unit"], "inputs_per_s": line["inputs_per_s"],
        "ms_per_step": line["ms_per_step"], "steps": line["steps"], "warmup": line["warmup"],
        "inputs_per_step": line["config"]["inputs_per_step"],
        "programs_compiled": line["config"]["programs_compiled"],
        "lane_mapping": line["config"]["lane_mapping"],
        "roofline": {"bound": r["bound"], "achieved": r["achieved"], "peak": r["peak"],
                     "unit": r["unit"], "frac": r["frac"],
                     "frac_folded_heads_uncredited": r["frac_folded_heads_uncredited"]},
        "e2e": {"value": line["e2e"]["value"], "unit": line["e2e"]["unit"],
                "h2d_bytes_per_step": line["e2e"]["h2d_bytes_per_step"],
                "d2h_bytes_per_step": line["e2e"]["d2h_bytes_per_step"]},
        "gpu_launches": line["gpu_launches"], "clocks": line["clocks"],
    }


# the other configurations, measured on the default run beside the headline:
# (workload, plain, timed steps, warm-up steps)
SUB_BATCH = (("c1", False, 10, 3), ("c1", True, 5, 3), ("c3", False, 5, 3), ("c3", True, 2, 3),
             ("c4", False, 5, 3), ("c4", True, 2, 3))
# serving: (offered inputs/s, seconds of arrivals) for each path
SUB_RATES = (20000.0, 100000.0, 200000.0)
SUB_SERVE_S = {False: 1.0, True: 0.5}


def run_engine(args, rank, world, local, pg):
    line = measure_engine(args, args.workload, args.plain, args.steps, args.warmup,
                          args.inputs_per_step, rank, world, local, pg, prex=args.prex)
    try:
        import torch

        from paper_2601_01048_gb300 import binding as B

        p = B.cufz_int32_peak(local, torch.cuda.current_stream(torch.device("cuda", local)).cuda_stream)
    except Exception:
        p = None
    achieved = line["roofline"]["achieved"] * 1e12
    line["roofline"]["measured_int32_peak"] = p / 1e12 if p else None
    line["roofline"]["frac_of_measured"] = achieved / p if p else None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        _, progs, inputs, _ = workload(args.workload)
        rate, irate, cores, n_in, n_acc, dt = oracle_rate(progs, inputs, args.cpu_seconds)
        line["cpu_baseline"] = {
            "value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_in} inputs of the same workload in seeded random order, "
                      f"{n_acc} checked accesses in {dt:.1f} s",
            "inputs_per_s": irate,
        }
    default_run = (args.workload == "c2" and not args.plain and not args.prex
                   and not args.inputs_per_step and world == 1 and not args.no_sub)
    if default_run:
        subs = {}
        for wl, plain, steps, warm in SUB_BATCH:
            rec = measure_engine(args, wl, plain, steps, warm, 0, rank, world, local, pg)
            subs[wl + ("_plain" if plain else "")] = sub_of(rec)
        for plain in (False, True):
            out = []
            for rate in SUB_RATES:
                rec = measure_serving(args, rate, SUB_SERVE_S[plain], plain, rank, world, local,
                                      pg)
                out.append(serving_sub(rec))
            subs["c5" + ("_plain" if plain else "")] = out
        rows, clk = measure_campaign(local, rank, (1024,), max_rounds=16)
        subs["campaign"] = {"metric": "fuzz inputs/sec", "unit": "inputs/s", "rows": rows,
                            "clocks": clk,
                            "workload": "coverage-guided rounds over the serving workload's 64 "
                                        "programs, host queue vs device-resident queue"}
        line["sub"] = subs
    if rank == 0:
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return
    wl_name, progs, inputs, cap = workload(args.workload)
    per = max(args.cpu_seconds / 2.0, 2.0)
    rates, irates = [], []
    cores = os.cpu_count() or 1
    n_tot = acc_tot = 0
    t_tot = 0.0
    for k in range(args.warmup + args.steps):
        rate, irate, cores, n_in, n_acc, dt = oracle_rate(progs, inputs, per, seed=100 + k)
        if k >= args.warmup:
            rates.append(rate)
            irates.append(irate)
            n_tot += n_in
            acc_tot += n_acc
            t_tot += dt
    value = acc_tot / t_tot
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded programs and fuzz inputs)",
        "config": {"workload": wl_name, "inputs_per_step": "bounded sample",
                   "path": "CPU oracle, serial per input, pool over inputs"},
        "inputs_per_s": n_tot / t_tot,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} steps of ~{per:.0f} s, {n_tot} inputs in "
                                   "seeded random order"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serving

def measure_serving(args, rate, duration, plain, rank, world, local, pg):
    """Config 5: an open-loop Poisson stream of mutated inputs over 64
    resident programs; delivered checked accesses/s and per-input latency
    from scheduled arrival to result."""
    import torch

    from paper_2601_01048_gb300 import binding as B
    from paper_2601_01048_gb300 import gen
    from paper_2601_01048_gb300.serve import serve_open_loop

    torch.cuda.set_device(local)
    progs = gen.c5_programs()
    corpus = gen.c5_corpus(progs)
    arrivals = gen.poisson_arrivals(rate, duration, seed=17 + rank)
    stream = gen.c5_stream(progs, corpus, len(arrivals), seed=29 + rank)
    warm_n = min(max(int(rate * 0.25), 64), len(stream))
    warm_arr = gen.poisson_arrivals(rate, 10.0, seed=5)[:warm_n]
    flags = B.CF_KEEP_BITMAPS | B.CF_AUTO_RELEASE | (B.CF_PLAIN_LAUNCH if plain else 0)
    if args.path == "jit":
        flags |= B.CF_JIT
    tune_path = tune_file("c5")[0] if args.path == "jit" else None
    E = B.Engine(device=local, max_slots=4096, record_cap=1024, flags=flags, n_lanes=args.lanes,
                 cta_threads=args.cta_threads, autotune_cache=tune_path)
    for p in progs:
        E.load(p)
    tuned = None
    if tune_path:
        tuned = autotune_or_load(B, E, "c5", corpus, len(progs))
    serve_open_loop(E, stream[:warm_n], warm_arr)
    torch.cuda.synchronize()
    barrier(pg)
    B.cufz_reset_stats(E.ctx)
    clocks = ClockSampler(local)
    clocks.start()
    res, lat, _, wall = serve_open_loop(E, stream, arrivals)
    clk = clocks.stop()
    st = B.cufz_get_stats(E.ctx)
    E.close()
    acc = float(res["n_accesses"].sum())
    wall_max = allreduce_max(pg, wall, torch.device("cuda", local))
    acc_all = allreduce_sum(pg, acc, torch.device("cuda", local))
    return {
        "metric": METRIC, "value": acc_all / wall_max, "unit": UNIT, "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": wall_max * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded programs, mutated fuzz inputs, Poisson arrivals)",
        "config": {"workload": "c5: open-loop serving over 64 resident programs (16 guarded 1D, "
                               "32 random 2D, 16 branch-heavy), mutated inputs",
                   "offered_rate": rate, "duration_s": duration, "inputs": len(stream),
                   "path": "plain one launch per input" if plain else
                           f"persistent kernels in CUDA graphs, {args.lanes} overlapping lanes",
                   "programs_compiled": tuned, "parallelism": f"replicas x{world}"},
        "inputs_per_s": len(stream) / wall,
        "latency_ms": {"p50": 1e3 * float(np.nanpercentile(lat, 50)),
                       "p99": 1e3 * float(np.nanpercentile(lat, 99)),
                       "p999": 1e3 * float(np.nanpercentile(lat, 99.9)),
                       "from": "scheduled arrival to result polled"},
        "device_busy_ms": st.kernel_ms, "batches": int(st.batches),
        "gpu_launches": int(st.kernel_launches), "clocks": clk,
        "e2e": {"value": acc_all / wall_max, "unit": UNIT,
                "h2d_bytes_per_step": len(stream) * 128, "d2h_bytes_per_step": len(stream) * 96},
    }


def serving_sub(line):
    """The compact form of a serving line kept inside the default line."""
    c = line["config"]
    return {"path": c["path"], "offered_rate": c["offered_rate"], "duration_s": c["duration_s"],
            "inputs": c["inputs"], "inputs_per_s": line["inputs_per_s"], "value": line["value"],
            "unit": line["unit"], "latency_ms": line["latency_ms"],
            "device_busy_ms": line["device_busy_ms"], "batches": line["batches"],
            "gpu_launches": line["gpu_launches"], "clocks": line["clocks"]}


def run_serving(args, rank, world, local, pg):
    line = measure_serving(args, args.rate, args.duration, args.plain, rank, world, local, pg)
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_campaign(local, rank, batches, max_rounds=64):
    """The fuzzing campaign over the serving workload's 64 programs: rounds
    per second with the queue on the host (one device batch per round, a
    host round trip between rounds) and on the device (every step of a round
    in kernels, rounds enqueued back to back), at the given round sizes.
    Returns (rows, clocks record)."""
    import torch

    from paper_2601_01048_gb300 import binding as B
    from paper_2601_01048_gb300 import gen
    from paper_2601_01048_gb300.fuzz import Campaign, DeviceCampaign, EngineExecutor

    torch.cuda.set_device(local)
    progs = gen.c5_programs()
    seeds = gen.c5_corpus(progs, per_program=2, max_blocks=64)
    n_bufs = gen.program_bufs(progs)
    rows = []
    clocks = ClockSampler(local)
    clocks.start()
    for batch in batches:
        rounds = max(4, min(max_rounds, 65536 // batch))
        row = {"batch": batch, "rounds": rounds}
        for kind in ("host", "device"):
            E = B.Engine(device=local, max_slots=max(batch, len(seeds)), record_cap=64,
                         flags=B.CF_JIT, iter_budget=4096)
            for p in progs:
                E.load(p)
            if kind == "host":
                c = Campaign(EngineExecutor(E), n_bufs, seeds, seed=1 + rank, batch=batch)
                c.run_round()                              # warm-up round
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(rounds):
                    c.run_round()
                dt = time.perf_counter() - t0
                corpus = len(c.corpus)
            else:
                d = DeviceCampaign(E, seeds, seed=1 + rank, batch=batch)
                d.run(1)
                d.sync()                                   # warm-up round
                t0 = time.perf_counter()
                d.run(rounds)
                d.sync()
                dt = time.perf_counter() - t0
                corpus = d.counters().corpus
                d.close()
            E.close()
            row[kind] = {"rounds_per_s": rounds / dt, "execs_per_s": rounds * batch / dt,
                         "ms_per_round": 1e3 * dt / rounds, "corpus_after": corpus}
        row["device_over_host"] = row["device"]["rounds_per_s"] / row["host"]["rounds_per_s"]
        rows.append(row)
    return rows, clocks.stop()


def run_campaign(args, rank, world, local, pg):
    """Fuzz inputs per second of the campaign, host queue against device
    queue, at 64 to 4,096 children per round."""
    rows, clk = measure_campaign(local, rank, (64, 256, 1024, 4096))
    if rank == 0:
        top = rows[-1]
        print(json.dumps({
            "metric": "fuzz inputs/sec", "value": top["device"]["execs_per_s"], "unit": "inputs/s",
            "n_gpus": world, "steps": top["rounds"], "warmup": 1,
            "ms_per_step": top["device"]["ms_per_round"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded programs, seed corpus, mutated children)",
            "config": {"workload": "campaign: coverage-guided rounds over the serving workload's 64 "
                                   "programs, host queue vs device-resident queue",
                       "parallelism": f"replicas x{world}"},
            "rows": rows, "clocks": clk}), flush=True)


def main():
    args = parse_args()
    rank, world, local, pg = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "campaign":
        run_campaign(args, rank, world, local, pg)
    elif args.workload == "c5":
        run_serving(args, rank, world, local, pg)
    else:
        run_engine(args, rank, world, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
