"""The bytecode interpreter's device code on the CPU, against the oracle.

The interpreter's warp loop (interp_kernel.cuh) runs inside the work-item
loop, finalize and helpers of device_common.cuh, as the persistent
interpreter kernel runs them, on one CTA of one warp whose 32 lanes are
host threads; warp collectives are exchanged at barriers
(tests/host_emulation/simt_shim.h).  The interpreter is warp-synchronous,
so this is its real execution, lane for lane, with the library's own
program loading and input building.  Built with AddressSanitizer and
UndefinedBehaviorSanitizer.  Statuses, counts, digests, first keys, record
sets and bitmaps must equal the oracle's; PREX items give the full grid's
verdict and exactly the planned threads' records.  Several CTAs at once
are the GPU tests' part.

TEST-ONLY: this executes device code on the host; the package itself has no
host execution path."""
import os
import struct
import subprocess

import numpy as np
import pytest

from paper_2601_01048_gb300 import binding as B
from paper_2601_01048_gb300 import build_ext, gen
from test_jit_host import CSRC, RESULT, SAN, SHIM, _gxx, engine_ops, record_set, workload


@pytest.fixture(scope="module")
def interp_exe(tmp_path_factory):
    gxx = _gxx()
    try:
        inc = os.path.join(os.path.dirname(os.path.dirname(build_ext.nvcc())), "include")
    except RuntimeError:
        pytest.skip("no CUDA toolkit headers")
    d = tmp_path_factory.mktemp("interp")
    objs = []
    for src, incs in ((os.path.join(CSRC, "loader.cpp"), [inc, CSRC]),
                      (os.path.join(CSRC, "prex.cpp"), [inc, CSRC]),
                      (os.path.join(SHIM, "blob_helper.cpp"), [inc, CSRC]),
                      (os.path.join(SHIM, "interp_runner.cpp"), [SHIM, CSRC])):
        obj = str(d / (os.path.basename(src) + ".o"))
        cmd = [gxx, "-std=c++17", "-O1", "-pthread", *SAN]
        for i in incs:
            cmd += ["-I", i]
        r = subprocess.run(cmd + ["-c", src, "-o", obj], capture_output=True, text=True)
        if r.returncode != 0 and "asan" in r.stderr.lower():
            pytest.skip("sanitizer runtime not available")
        assert r.returncode == 0, r.stderr[-4000:]
        objs.append(obj)
    exe = str(d / "interp_host")
    r = subprocess.run([gxx, "-pthread", *SAN, *objs, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    return exe


def run(tmp_path, exe, progs, inputs, plans=None, cap=1 << 14, budget=4096, item=96, flags=0):
    job, out = tmp_path / "job.bin", tmp_path / "out.bin"
    with open(job, "wb") as f:
        f.write(struct.pack("<6I", len(progs), cap, 256, budget, item, flags))
        for p in progs:
            f.write(struct.pack("<I", len(p)) + p)
        f.write(struct.pack("<I", len(inputs)))
        for k, x in enumerate(np.ascontiguousarray(inputs, dtype=gen.INPUT_DTYPE)):
            plan = [] if plans is None or plans[k] is None else [int(v) for v in plans[k]]
            f.write(x.tobytes() + struct.pack(f"<I{len(plan)}I", len(plan), *plan))
    r = subprocess.run([exe, str(job), str(out)], capture_output=True, text=True, timeout=900,
                       env=dict(os.environ, ASAN_OPTIONS="detect_leaks=1"))
    assert r.returncode == 0 and "runtime error" not in r.stderr, (r.stdout + r.stderr)[-4000:]
    data, pos, outs = out.read_bytes(), 0, []
    for _ in range(len(inputs)):
        res = np.frombuffer(data, RESULT, 1, pos)[0]
        pos += RESULT.itemsize
        recs = np.frombuffer(data, B.VIOLATION_DTYPE, int(res["n_records"]), pos)
        pos += B.VIOLATION_DTYPE.itemsize * int(res["n_records"])
        outs.append((res, recs, np.frombuffer(data, np.uint8, 65536, pos)))
        pos += 65536
    assert pos == len(data)
    return outs


def compare(got, ores, orecs, obms, cap, ops=None):
    for k, (res, recs, bm) in enumerate(got):
        o = ores[k]
        for f in ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch",
                  "n_edges", "n_threads"):
            assert int(res[f]) == int(o[f]), (k, f)
        if ops is not None:
            assert int(res["n_ops"]) == ops[k], k
        assert int(res["flags"]) & B.FL_BUDGET == int(o["flags"]) & B.FL_BUDGET, k
        assert bool(int(res["flags"]) & B.FL_OVERFLOW) == (int(o["n_violations"]) > cap), k
        n_o = int(o["n_violations"])
        full = record_set(orecs[k][: int(o["n_records"])])
        if n_o <= cap:
            assert record_set(recs) == full, k
        else:
            assert len(recs) == cap, k
            if int(o["n_records"]) == n_o:                      # the oracle kept them all
                assert record_set(recs) <= full, k
        assert np.array_equal(bm, obms[k]), k


@pytest.mark.parametrize("flags", [0, B.CF_NO_PRUNE])
def test_interpreter_matches_oracle(tmp_path, interp_exe, orc, flags):
    progs, ins = workload()
    got = run(tmp_path, interp_exe, progs, ins, flags=flags)
    ores, orecs, obms = orc.run_batch(progs, ins, rec_cap=1 << 17, bitmaps=True)
    compare(got, ores, orecs, obms, 1 << 14, engine_ops(orc, progs, ins, flags))
    assert 0 < sum(int(o["status"]) == 1 for o in ores) < len(ins)


def test_interpreter_budget_shapes_and_record_cap(tmp_path, interp_exe, orc):
    """A budget that stops threads in loops, random 3D launch shapes, and a
    record cap small enough to overflow (any cap of the records is kept,
    counts stay exact)."""
    progs = gen.c2_programs()[:6] + gen.c4_programs()[:2]
    ins = gen.c2_inputs(progs[:6], per_program=2, seed=309, max_grid=2)
    rng = gen.SplitMix64(310)
    shaped = ins.copy()
    for x in shaped:
        x["grid"] = [rng.randint(1, 3), rng.randint(1, 3), rng.randint(1, 3)]
        x["block"] = [rng.randint(1, 9), rng.randint(1, 6), rng.randint(1, 4)]
    c4 = gen.c4_inputs(4, n_programs=2, seed=311, max_blocks=2)
    c4["program_id"] += 6
    ins = np.concatenate([ins, shaped, c4])
    for budget, cap in ((5, 1 << 14), (4096, 16)):
        got = run(tmp_path, interp_exe, progs, ins, budget=budget, cap=cap)
        ores, orecs, obms = orc.run_batch(progs, ins, orc.opts(iter_budget=budget),
                                          rec_cap=1 << 16, bitmaps=True)
        compare(got, ores, orecs, obms, cap, engine_ops(orc, progs, ins, 0, budget))


def test_interpreter_prex_items(tmp_path, interp_exe, orc):
    progs, ins = workload(max_threads=256)
    plans = [B.cufz_prex_plan(progs[int(x["program_id"])], x) for x in ins]
    assert sum(p is not None for p in plans) >= 16
    got = run(tmp_path, interp_exe, progs, ins, plans=plans)
    ores, orecs, _ = orc.run_batch(progs, ins, rec_cap=1 << 16)
    for k, (res, recs, _) in enumerate(got):
        o = ores[k]
        assert int(res["status"]) == int(o["status"]), k
        if plans[k] is None:
            continue
        T = int(np.prod([int(v) for v in ins[k]["block"]]))
        full = orecs[k][: int(o["n_records"])]
        keep = np.isin(full["block_lin"].astype(np.int64) * T + full["thread_lin"], plans[k])
        assert record_set(recs) == record_set(full[keep]), k
        assert int(res["n_violations"]) == int(keep.sum())


@pytest.mark.parametrize("flags", [0, B.CF_NO_PRUNE])
def test_interpreter_division_programs(tmp_path, interp_exe, orc, flags):
    """Programs with signed divisions: fault records (kind 2) from lanes of
    one warp reserved together, ordinals that count divisions, values,
    pruned (dead quotients kept as checks) and unpruned, with a small record
    cap as well."""
    progs = gen.div_programs()
    ins = gen.div_inputs(48, seed=313)
    for cap in (1 << 14, 8):
        got = run(tmp_path, interp_exe, progs, ins, cap=cap, flags=flags)
        ores, orecs, obms = orc.run_batch(progs, ins, rec_cap=1 << 14, bitmaps=True)
        compare(got, ores, orecs, obms, cap, engine_ops(orc, progs, ins, flags))
        assert sum(int((r["kind"] == 2).sum()) for _, r, _ in got) > 0


@pytest.mark.parametrize("flags", [0, B.CF_NO_PRUNE])
def test_interpreter_heap_programs(tmp_path, interp_exe, orc, flags):
    """Programs on the device heap: the per-site state registers after the
    program's own, cleared per test thread; fault records of space 2 (kind 3
    for a bad free) from lanes of one warp reserved together; ordinals that
    count frees and heap accesses; pruned and unpruned, with a small record
    cap as well."""
    progs = gen.heap_programs()
    ins = gen.heap_inputs(48, seed=315)
    for cap in (1 << 14, 8):
        got = run(tmp_path, interp_exe, progs, ins, cap=cap, flags=flags)
        ores, orecs, obms = orc.run_batch(progs, ins, rec_cap=1 << 14, bitmaps=True)
        compare(got, ores, orecs, obms, cap, engine_ops(orc, progs, ins, flags))
        if cap > 8:
            assert sum(int((r["kind"] == 3).sum()) for _, r, _ in got) > 0


@pytest.mark.parametrize("flags", [0, B.CF_NO_PRUNE])
def test_interpreter_barrier_programs(tmp_path, interp_exe, orc, flags):
    """Programs with performed shared stores whose barriers BarrierElimination
    removes: the interpreter, with no store performed and no barrier, equals
    the oracle's phase-by-phase execution, pruned and unpruned, with a small
    record cap as well."""
    progs = gen.barrier_programs()
    ins = gen.barrier_inputs(48, seed=317)
    for cap in (1 << 14, 8):
        got = run(tmp_path, interp_exe, progs, ins, cap=cap, flags=flags)
        ores, orecs, obms = orc.run_batch(progs, ins, rec_cap=1 << 14, bitmaps=True)
        compare(got, ores, orecs, obms, cap, engine_ops(orc, progs, ins, flags))
