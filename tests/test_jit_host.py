"""The compiled path's generated code on the CPU, against the oracle.

The program functions the loader emits (cufz_program_cuda) are compiled for
the host together with the real device helpers of jit_kernel.cuh and
device_common.cuh, a one-lane shim of the CUDA intrinsics
(tests/host_emulation/device_shim.h) and a runner that executes each
input's work items one after another, with DevInput built by the library's
own fill_dev_input.  Built with AddressSanitizer and UndefinedBehaviorSanitizer.
Every count, the digest, the first-violation key, the record set and the
bucketed bitmap must equal the oracle's; PREX runs (single-thread items of
the plan) must give the full grid's verdict and exactly the planned
threads' records.  Warps of several lanes and several CTAs (merging,
races) are the GPU tests' part.

TEST-ONLY: this executes device code on the host to check the code
generator; the package itself has no host execution path."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from paper_2601_01048_gb300 import binding as B
from paper_2601_01048_gb300 import build_ext, bytecode as bc, gen

CSRC = os.path.join(os.path.dirname(build_ext.__file__), "csrc")
SHIM = os.path.join(os.path.dirname(os.path.abspath(__file__)), "host_emulation")
SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all"]
RESULT = np.dtype([("status", "<i4"), ("flags", "<u4"), ("n_accesses", "<u8"),
                   ("n_violations", "<u8"), ("first_key", "<u8"), ("digest", "<u8"),
                   ("n_branch", "<u8"), ("n_ops", "<u8"), ("n_threads", "<u8"),
                   ("n_records", "<u4"), ("n_edges", "<u4")])
KEYS = ("block_lin", "thread_lin", "ordinal", "site", "buf", "kind", "width", "space", "cls",
        "byte_off")


def _gxx():
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("no g++")
    return gxx


@pytest.fixture(scope="module")
def host_objs(tmp_path_factory):
    """loader.cpp and prex.cpp (for fill_dev_input) built for the host."""
    gxx = _gxx()
    try:
        inc = os.path.join(os.path.dirname(os.path.dirname(build_ext.nvcc())), "include")
    except RuntimeError:
        pytest.skip("no CUDA toolkit headers")
    d = tmp_path_factory.mktemp("objs")
    objs = []
    for src in ("loader.cpp", "prex.cpp"):
        obj = str(d / (src + ".o"))
        r = subprocess.run([gxx, "-std=c++17", "-O1", *SAN, "-I", inc, "-I", CSRC, "-c",
                            os.path.join(CSRC, src), "-o", obj], capture_output=True, text=True)
        if r.returncode != 0 and "asan" in r.stderr.lower():
            pytest.skip("sanitizer runtime not available")
        assert r.returncode == 0, r.stderr[-3000:]
        objs.append(obj)
    return objs


def build(tmp_path, objs, progs, flags=0, defines=()):
    """One host executable running `progs` (their emitted functions as the
    device's module would hold them, program k as cufz_prog_k), compiled with
    the given preprocessor definitions."""
    srcs = [B.cufz_program_cuda(p, flags).replace("cufz_prog_0", f"cufz_prog_{k}")
            for k, p in enumerate(progs)]
    cases = "".join(f"    case {k}: cufz_prog_{k}(g0, g_end); return true;\n"
                    for k in range(len(progs)))
    tu = ('#include "device_shim.h"\n#include "jit_kernel.cuh"\n#include "shim_post.h"\n'
          "namespace cufz {\n" + "".join(srcs) +
          "static bool jit_run(uint32_t prog, uint32_t g0, uint32_t g_end) {\n"
          "  switch (prog) {\n" + cases + "    default: return false;\n  }\n}\n"
          '}  // namespace cufz\n#include "runner.inc"\n')
    src = tmp_path / "module_host.cpp"
    src.write_text(tu)
    exe = str(tmp_path / "module_host")
    r = subprocess.run([_gxx(), "-std=c++17", "-O1", *SAN, "-w", *[f"-D{d}" for d in defines],
                        "-I", SHIM, "-I", CSRC, str(src), *objs, "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    return exe


def run(tmp_path, exe, progs, inputs, plans=None, cap=1 << 14, budget=4096, item=96):
    job = tmp_path / "job.bin"
    out = tmp_path / "out.bin"
    with open(job, "wb") as f:
        f.write(struct.pack("<6I", len(progs), cap, 256, budget, item, 0))
        for p in progs:
            hdr = bc.decode_header(p)
            f.write(struct.pack("<2I", hdr["n_bufs"], hdr["shared_mask"]))
        f.write(struct.pack("<I", len(inputs)))
        for k, x in enumerate(np.ascontiguousarray(inputs, dtype=gen.INPUT_DTYPE)):
            plan = [] if plans is None or plans[k] is None else [int(v) for v in plans[k]]
            f.write(x.tobytes() + struct.pack(f"<I{len(plan)}I", len(plan), *plan))
    r = subprocess.run([exe, str(job), str(out)], capture_output=True, text=True, timeout=600,
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


def engine_ops(orc, progs, ins, flags=0, budget=4096):
    """The executed-op count (n_ops) each input must report: the oracle's
    count on the program the engine runs, i.e. the bytes cufz_prune_program
    returns (the unpruned program under CF_NO_PRUNE)."""
    run_progs = progs if flags & B.CF_NO_PRUNE else [B.cufz_prune_program(p)[0] for p in progs]
    res, _, _ = orc.run_batch(run_progs, ins, orc.opts(iter_budget=budget))
    return [int(v) for v in res["n_ops"]]


def record_set(recs, fields=KEYS):
    return set(zip(*(recs[f].tolist() for f in fields)))


def workload(max_threads=128):
    progs = ([gen.c1_program()] + gen.c2_programs()[:6] + gen.c3_programs()[:4]
             + gen.c4_programs()[:3] + gen.affine_programs()[:3])
    c1 = gen.c1_inputs(4, seed=301)
    c2 = gen.c2_inputs(progs[1:7], per_program=2, seed=302, max_grid=2)
    c2["program_id"] += 1
    c3 = gen.c3_inputs(8, seed=303, max_blocks=8, max_threads=max_threads)
    c3["program_id"] = 7 + c3["program_id"] % 4
    c4 = gen.c4_inputs(6, n_programs=3, seed=304, max_blocks=2)
    c4["program_id"] += 11
    aff = gen.affine_inputs(6, seed=305, max_blocks=8, max_threads=64)
    aff["program_id"] = 14 + aff["program_id"] % 3
    return progs, np.concatenate([c1, c2, c3, c4, aff])


@pytest.mark.parametrize("flags", [0, B.CF_NO_PRUNE])
def test_generated_code_matches_oracle(tmp_path, host_objs, orc, flags):
    progs, ins = workload()
    exe = build(tmp_path, host_objs, progs, flags)
    got = run(tmp_path, exe, progs, ins)
    ores, orecs, obms = orc.run_batch(progs, ins, rec_cap=1 << 14, bitmaps=True)
    ops = engine_ops(orc, progs, ins, flags)
    assert sum(ops) > 0
    n_viol = 0
    for k, (res, recs, bm) in enumerate(got):
        o = ores[k]
        for f in ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch",
                  "n_edges", "n_records", "n_threads"):
            assert int(res[f]) == int(o[f]), (k, f)
        assert int(res["n_ops"]) == ops[k], k
        assert record_set(recs) == record_set(orecs[k][: int(o["n_records"])]), k
        assert np.array_equal(bm, obms[k]), k
        n_viol += int(o["status"]) == 1
    assert 0 < n_viol < len(ins)


def test_budget_stop_and_3d_shapes_match_oracle(tmp_path, host_objs, orc):
    """A back-edge budget small enough to stop threads inside loops, and
    random 3D launch shapes (every coordinate decomposition of the emitted
    code)."""
    progs = gen.c2_programs()[:6]
    ins = gen.c2_inputs(progs, per_program=2, seed=306, max_grid=2)
    exe = build(tmp_path, host_objs, progs)
    rng = gen.SplitMix64(308)
    shaped = np.concatenate([ins, ins, ins])
    # blocks of exactly the CTA's 256 threads and larger ones over 3D grids:
    # the stepped block coordinates (x, the carry into y, then into z)
    big = ((16, 16, 1), (8, 8, 4), (32, 16, 1), (16, 8, 4), (64, 4, 2))
    for k, x in enumerate(shaped):
        x["grid"] = [rng.randint(1, 3), rng.randint(1, 3), rng.randint(1, 3)]
        if k < 2 * len(ins):
            x["block"] = [rng.randint(1, 9), rng.randint(1, 6), rng.randint(1, 4)]
        else:
            x["block"] = big[k % len(big)]
    got = run(tmp_path, exe, progs, shaped)
    ores, orecs, obms = orc.run_batch(progs, shaped, rec_cap=1 << 14, bitmaps=True)
    for k, (res, recs, bm) in enumerate(got):
        for f in ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch",
                  "n_edges", "n_threads"):
            assert int(res[f]) == int(ores[k][f]), (k, f)
        assert record_set(recs) == record_set(orecs[k][: int(ores[k]["n_records"])]), k
        assert np.array_equal(bm, obms[k]), k
    got = run(tmp_path, exe, progs, ins, budget=3)
    ores, orecs, obms = orc.run_batch(progs, ins, orc.opts(iter_budget=3), rec_cap=1 << 14,
                                      bitmaps=True)
    ops = engine_ops(orc, progs, ins, budget=3)
    stopped = 0
    for k, (res, recs, bm) in enumerate(got):
        o = ores[k]
        assert int(res["n_ops"]) == ops[k], k
        assert int(res["flags"]) & 1 == int(o["flags"]) & 1, k
        for f in ("n_accesses", "n_violations", "first_key", "digest", "n_branch", "n_edges"):
            assert int(res[f]) == int(o[f]), (k, f)
        assert np.array_equal(bm, obms[k]), k
        stopped += int(o["flags"]) & 1
    assert stopped > 0


def test_prex_items_match_oracle(tmp_path, host_objs, orc):
    """Inputs run as their PREX plan's single-thread items (corners of
    affine programs; cell corners of guarded 1D and configuration 3 launches):
    the full grid's verdict, and exactly the planned threads' records."""
    progs, ins = workload(max_threads=256)
    exe = build(tmp_path, host_objs, progs)
    plans = [B.cufz_prex_plan(progs[int(x["program_id"])], x) for x in ins]
    assert sum(p is not None for p in plans) >= 16
    got = run(tmp_path, exe, progs, ins, plans=plans)
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
        assert int(res["n_violations"]) == int(keep.sum()) and int(res["n_threads"]) == len(plans[k])


def test_mutated_programs_match_oracle(tmp_path, host_objs, orc):
    """Random and branch-heavy programs with random bit flips in their ops,
    kept when both validators accept them (unusual opcode, operand and
    nesting mixes the generators do not produce), under the default budget
    and one that stops threads early."""
    rng = gen.SplitMix64(0x3A7E)
    progs, k = [], 0
    while len(progs) < 24:
        p = bytearray(gen.c2_program(500 + k) if k % 3 < 2 else gen.c4_program(500 + k))
        k += 1
        for _ in range(1 + rng.below(3)):
            j = 32 + rng.below(len(p) - 32)
            p[j] ^= 1 << rng.below(8)
        if B.cufz_validate_program(bytes(p)) == 0 and orc.validate(bytes(p)) == 0:
            progs.append(bytes(p))
    ins = gen.c2_inputs(progs, per_program=2, seed=307, max_grid=2)
    exe = build(tmp_path, host_objs, progs)
    for budget in (4096, 5):
        got = run(tmp_path, exe, progs, ins, budget=budget)
        ores, orecs, obms = orc.run_batch(progs, ins, orc.opts(iter_budget=budget),
                                          rec_cap=1 << 14, bitmaps=True)
        ops = engine_ops(orc, progs, ins, 0, budget)
        for i, (res, recs, bm) in enumerate(got):
            o = ores[i]
            assert int(res["n_ops"]) == ops[i], (budget, i)
            for f in ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch",
                      "n_edges", "n_records"):
                assert int(res[f]) == int(o[f]), (budget, i, f)
            assert int(res["flags"]) & 1 == int(o["flags"]) & 1, (budget, i)
            assert record_set(recs) == record_set(orecs[i][: int(o["n_records"])]), (budget, i)
            assert np.array_equal(bm, obms[i]), (budget, i)


@pytest.mark.parametrize("table_log2", [12, 1, 0])
def test_path_counting_matches_oracle(tmp_path, host_objs, orc, table_log2):
    """Branch-heavy loop-free programs run in path mode: each thread counts
    its path (its sites' outcomes) in the CTA's path table, and each distinct
    path's edges are replayed once per work item with its count.  Pruned and
    unpruned, and on bit-flipped variants of the programs.  With a table of
    two slots most paths find no room, and their threads replay them at
    once; without a table (table_log2 0: the plain kernel's CTAs) every
    thread replays its own path."""
    rng = gen.SplitMix64(0x9ED1)
    progs = gen.c4_programs()[:6]
    k = 0
    while len(progs) < 12:
        p = bytearray(gen.c4_program(700 + k))
        k += 1
        for _ in range(1 + rng.below(3)):
            j = 32 + rng.below(len(p) - 32)
            p[j] ^= 1 << rng.below(8)
        if B.cufz_validate_program(bytes(p)) == 0 and orc.validate(bytes(p)) == 0:
            progs.append(bytes(p))
    ins = gen.c4_inputs(36, n_programs=len(progs), seed=309, max_blocks=2)
    for flags in (0, B.CF_NO_PRUNE):
        exe = build(tmp_path, host_objs, progs, flags,
                    defines=(f"CUFZ_PATH_SLOTS_LOG2={table_log2}",) if table_log2
                    else ("CUFZ_SHIM_NO_PATH_TABLE",))
        got = run(tmp_path, exe, progs, ins)
        ores, orecs, obms = orc.run_batch(progs, ins, rec_cap=1 << 14, bitmaps=True)
        ops = engine_ops(orc, progs, ins, flags)
        for i, (res, recs, bm) in enumerate(got):
            o = ores[i]
            for f in ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch",
                      "n_edges", "n_records"):
                assert int(res[f]) == int(o[f]), (flags, i, f)
            assert int(res["n_ops"]) == ops[i], (flags, i)
            assert record_set(recs) == record_set(orecs[i][: int(o["n_records"])]), (flags, i)
            assert np.array_equal(bm, obms[i]), (flags, i)


@pytest.mark.parametrize("flags", [0, B.CF_NO_PRUNE])
def test_division_programs_match_oracle(tmp_path, host_objs, orc, flags):
    """Programs with signed divisions (zero divisors from coordinates, masked
    arguments and loaded bytes; quotients and remainders as indices, in
    branches and a loop): fault records (kind 2), ordinals that count
    divisions, values and every other result equal the oracle's, pruned and
    unpruned, and under a budget that stops threads early."""
    progs = gen.div_programs()
    ins = gen.div_inputs(48, seed=312)
    exe = build(tmp_path, host_objs, progs, flags)
    for budget in (4096, 2):
        got = run(tmp_path, exe, progs, ins, budget=budget)
        ores, orecs, obms = orc.run_batch(progs, ins, orc.opts(iter_budget=budget),
                                          rec_cap=1 << 14, bitmaps=True)
        ops = engine_ops(orc, progs, ins, flags, budget)
        faults = 0
        for i, (res, recs, bm) in enumerate(got):
            o = ores[i]
            assert int(res["n_ops"]) == ops[i], (budget, i)
            for f in ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch",
                      "n_edges", "n_records"):
                assert int(res[f]) == int(o[f]), (budget, i, f)
            assert int(res["flags"]) & 1 == int(o["flags"]) & 1, (budget, i)
            assert record_set(recs) == record_set(orecs[i][: int(o["n_records"])]), (budget, i)
            assert np.array_equal(bm, obms[i]), (budget, i)
            faults += int((recs["kind"] == 2).sum())
        assert faults > 0


@pytest.mark.parametrize("flags", [0, B.CF_NO_PRUNE])
def test_heap_programs_match_oracle(tmp_path, host_objs, orc, flags):
    """Programs on the device heap (blocks sized by arguments, coordinates
    and loaded bytes; frees under branches and in loops; accesses through
    live, freed, NULL and forged handles): every class of heap fault (use
    after free, double and invalid free, redzone and wild heap accesses) in
    its record, ordinals that count frees and heap accesses, digests, and
    every other result equal the oracle's, pruned and unpruned, and under a
    budget that stops threads early."""
    progs = gen.heap_programs()
    ins = gen.heap_inputs(48, seed=314)
    exe = build(tmp_path, host_objs, progs, flags)
    for budget in (4096, 2):
        got = run(tmp_path, exe, progs, ins, budget=budget)
        ores, orecs, obms = orc.run_batch(progs, ins, orc.opts(iter_budget=budget),
                                          rec_cap=1 << 14, bitmaps=True)
        ops = engine_ops(orc, progs, ins, flags, budget)
        seen = set()
        for i, (res, recs, bm) in enumerate(got):
            o = ores[i]
            assert int(res["n_ops"]) == ops[i], (budget, i)
            for f in ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch",
                      "n_edges", "n_records"):
                assert int(res[f]) == int(o[f]), (budget, i, f)
            assert int(res["flags"]) & 1 == int(o["flags"]) & 1, (budget, i)
            assert record_set(recs) == record_set(orecs[i][: int(o["n_records"])]), (budget, i)
            assert np.array_equal(bm, obms[i]), (budget, i)
            seen |= {(int(r["kind"]), int(r["cls"])) for r in recs if int(r["space"]) == 2}
        if budget == 4096:
            assert {(0, 6), (1, 6), (3, 7), (3, 8), (0, 4), (1, 2)} <= seen, seen


@pytest.mark.parametrize("flags", [0, B.CF_NO_PRUNE])
def test_barrier_programs_match_oracle(tmp_path, host_objs, orc, flags):
    """Programs with performed shared stores and barriers that
    BarrierElimination removes (no value read from a tile reaches a check):
    the generated code, which performs no store and has no barrier, equals
    the oracle, which performs the stores phase by phase, in every result,
    pruned and unpruned, and under a budget that stops threads early."""
    progs = gen.barrier_programs()
    ins = gen.barrier_inputs(48, seed=316)
    exe = build(tmp_path, host_objs, progs, flags)
    for budget in (4096, 2):
        got = run(tmp_path, exe, progs, ins, budget=budget)
        ores, orecs, obms = orc.run_batch(progs, ins, orc.opts(iter_budget=budget),
                                          rec_cap=1 << 14, bitmaps=True)
        ops = engine_ops(orc, progs, ins, flags, budget)
        for i, (res, recs, bm) in enumerate(got):
            o = ores[i]
            assert int(res["n_ops"]) == ops[i], (budget, i)
            for f in ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch",
                      "n_edges", "n_records"):
                assert int(res[f]) == int(o[f]), (budget, i, f)
            assert int(res["flags"]) & 1 == int(o["flags"]) & 1, (budget, i)
            assert record_set(recs) == record_set(orecs[i][: int(o["n_records"])]), (budget, i)
            assert np.array_equal(bm, obms[i]), (budget, i)
        assert sum(int(o["n_violations"]) for o in ores) > 0


@pytest.mark.parametrize("flags", [0, B.CF_NO_PRUNE])
def test_block_serial_barrier_programs_match_oracle(tmp_path, host_objs, orc, flags):
    """Programs whose performed shared stores reach checks, so their
    barriers must stay: the block-serial functions (a block's threads in
    thread order, phase by phase, stores performed in the block's bytes)
    equal the oracle's phased execution in every result, records included,
    pruned (stored shared values kept) and unpruned, and under a budget that
    stops threads inside loops, which then run no later phase."""
    progs = gen.barrier_programs(live=True)
    ins = gen.barrier_inputs(64, seed=331)
    exe = build(tmp_path, host_objs, progs, flags)
    for budget in (4096, 2):
        got = run(tmp_path, exe, progs, ins, budget=budget)
        ores, orecs, obms = orc.run_batch(progs, ins, orc.opts(iter_budget=budget),
                                          rec_cap=1 << 14, bitmaps=True)
        ops = engine_ops(orc, progs, ins, flags, budget)
        for i, (res, recs, bm) in enumerate(got):
            o = ores[i]
            for f in ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch",
                      "n_edges", "n_records", "n_threads"):
                assert int(res[f]) == int(o[f]), (budget, i, f)
            assert int(res["n_ops"]) == ops[i], (budget, i)
            assert int(res["flags"]) & 1 == int(o["flags"]) & 1, (budget, i)
            assert record_set(recs) == record_set(orecs[i][: int(o["n_records"])]), (budget, i)
            assert np.array_equal(bm, obms[i]), (budget, i)
        if budget == 2:
            assert any(int(o["flags"]) & 1 for o in ores)
