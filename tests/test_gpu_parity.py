"""GPU parity: the engine (through the C ABI) against the CPU oracle, bit for
bit: statuses, counts, first keys, digests, bucketed bitmaps and violation
record sets."""
import numpy as np
import pytest

from paper_2601_01048_gb300 import bytecode as bc
from paper_2601_01048_gb300 import gen
from conftest import record_keys

pytestmark = pytest.mark.gpu

COUNT_FIELDS = ("n_accesses", "n_violations", "first_key", "digest", "n_branch", "n_threads",
                "n_edges")


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_01048_gb300 import binding
    binding.lib()
    return binding




def compare(B, orc, inputs, dres, drecs, dbms, ores, orecs, obms, cap, check_newcov=False):
    bad = []
    for i in range(len(inputs)):
        d, o = dres[i], ores[i]
        try:
            assert int(d["status"]) == int(o["status"]), "status"
            for f in COUNT_FIELDS:
                assert int(d[f]) == int(o[f]), f
            mask = B.FL_BUDGET | (B.FL_NEW_COV if check_newcov else 0)
            assert int(d["flags"]) & mask == int(o["flags"]) & mask, "flags"
            # OVERFLOW is relative to the engine's record cap
            assert bool(int(d["flags"]) & B.FL_OVERFLOW) == (int(o["n_violations"]) > cap), "overflow"
            if dbms is not None and obms is not None:
                assert np.array_equal(dbms[i], obms[i]), "bitmap"
            if drecs is not None:
                n_o = int(o["n_violations"])
                dk = record_keys(drecs[i])
                if n_o <= cap:
                    assert dk == record_keys(orecs[i][:n_o]), "records"
                else:
                    assert len(dk) == cap and int(d["n_records"]) == cap
                    if orecs is not None and len(orecs[i]) >= n_o:
                        assert set(dk) <= set(record_keys(orecs[i][:n_o])), "record subset"
        except AssertionError as e:
            bad.append((i, str(e), d, o))
    assert not bad, f"{len(bad)} mismatches, first: {bad[0]}"


def run_both(B, orc, progs, inputs, cap=1 << 15, flags=None, budget=4096, redzone=256,
             max_threads=1 << 31, orc_cap=None, **kw):
    flags = B.CF_KEEP_BITMAPS if flags is None else flags
    with B.Engine(record_cap=cap, flags=flags, iter_budget=budget, redzone=redzone,
                  max_threads=max_threads, max_slots=kw.pop("max_slots", 2048), **kw) as E:
        for p in progs:
            E.load(p)
        dres, drecs, dbms = E.run(inputs, bitmaps=bool(flags & B.CF_KEEP_BITMAPS))
        st = E.stats()
    o = orc.opts(redzone=redzone, iter_budget=budget, max_threads=max_threads)
    ores, orecs, obms = orc.run_batch(progs, inputs, o, rec_cap=orc_cap or cap, bitmaps=True)
    return dres, drecs, dbms, ores, orecs, obms, st


PATHS = [0, 64]  # bytecode interpreter, compiled programs (CUFZ_CF_JIT)


@pytest.mark.parametrize("path", PATHS)
def test_c1_full(B, orc, path):
    """Config 1 at full size: 1,000 inputs of the guarded 1D kernel."""
    progs = [gen.c1_program()]
    inputs = gen.c1_inputs(1000)
    cap = 1 << 15
    dres, drecs, dbms, ores, orecs, obms, st = run_both(B, orc, progs, inputs, cap=cap,
                                                        flags=B.CF_KEEP_BITMAPS | path)
    compare(B, orc, inputs, dres, drecs, dbms, ores, orecs, obms, cap)
    assert st.kernel_launches >= 1 and int(ores["n_violations"].sum()) > 1000
    # every batch went through the lane's CUDA graph
    assert st.graph_failures == 0 and st.graph_launches == st.batches, (
        st.graph_failures, st.graph_launches, st.batches, st.last_cuda_error)


@pytest.mark.parametrize("path", PATHS)
def test_c1_plain_launch(B, orc, path):
    progs = [gen.c1_program()]
    inputs = gen.c1_inputs(64)
    cap = 1 << 15
    dres, drecs, dbms, ores, orecs, obms, st = run_both(
        B, orc, progs, inputs, cap=cap, flags=B.CF_KEEP_BITMAPS | B.CF_PLAIN_LAUNCH | path)
    compare(B, orc, inputs, dres, drecs, dbms, ores, orecs, obms, cap)
    assert st.kernel_launches == 64 and st.graph_launches == 0


def test_c1_no_graph(B, orc):
    progs = [gen.c1_program()]
    inputs = gen.c1_inputs(200, seed=99)
    dres, drecs, dbms, ores, orecs, obms, st = run_both(
        B, orc, progs, inputs, flags=B.CF_KEEP_BITMAPS | B.CF_NO_GRAPH)
    compare(B, orc, inputs, dres, drecs, dbms, ores, orecs, obms, 1 << 15)
    assert st.graph_launches == 0


def small_c2_inputs(progs, per_program, seed, max_grid=6):
    ins = gen.c2_inputs(progs, per_program=per_program, seed=seed, max_grid=max_grid)
    return ins


@pytest.mark.parametrize("path", PATHS)
def test_c2_small_grids(B, orc, path):
    """All 32 random programs, 6 inputs each, grids up to 6 x 6 blocks of 16 x 16."""
    progs = gen.c2_programs()
    inputs = small_c2_inputs(progs, 6, seed=1234)
    cap = 1 << 14
    dres, drecs, dbms, ores, orecs, obms, _ = run_both(B, orc, progs, inputs, cap=cap,
                                                       orc_cap=1 << 17,
                                                       flags=B.CF_KEEP_BITMAPS | path)
    compare(B, orc, inputs, dres, drecs, dbms, ores, orecs, obms, cap)


@pytest.mark.parametrize("path", PATHS)
def test_c2_unpruned_digest_equal(B, orc, path):
    """Sec. 5.2 invariant on the device: pruned and unpruned programs give the
    same digest, counts, bitmaps and records."""
    progs = gen.c2_programs()
    inputs = small_c2_inputs(progs, 3, seed=777)
    cap = 1 << 14
    out = []
    for flags in (B.CF_KEEP_BITMAPS | path, B.CF_KEEP_BITMAPS | B.CF_NO_PRUNE | path):
        with B.Engine(record_cap=cap, flags=flags, max_slots=512) as E:
            for p in progs:
                E.load(p)
            out.append(E.run(inputs))
            if flags & B.CF_NO_PRUNE:
                kept = sum(s.n_ops_kept for s in E.prog_stats)
            else:
                kept_pruned = sum(s.n_ops_kept for s in E.prog_stats)
    (r0, c0, b0), (r1, c1, b1) = out
    assert kept_pruned < kept
    for f in COUNT_FIELDS + ("status", "flags"):
        assert np.array_equal(r0[f], r1[f]), f
    assert np.array_equal(b0, b1)
    for k, (a, b) in enumerate(zip(c0, c1)):
        if int(r0[k]["n_violations"]) <= cap:   # overflowed record sets are any cap-subset
            assert record_keys(a) == record_keys(b)
    assert np.all(r0["n_ops"] <= r1["n_ops"]) and r0["n_ops"].sum() < r1["n_ops"].sum()


@pytest.mark.parametrize("path", PATHS)
def test_c3_ragged_blocks(B, orc, path):
    """Config-3 programs (widths 1/4/8/16, offsets) with log-uniform grids and
    block sizes that are rarely multiples of 32, persistent and plain paths."""
    progs = gen.c3_programs()
    inputs = gen.c3_inputs(160, seed=31, max_blocks=64, min_threads=1, max_threads=1024)
    cap = 1 << 15
    for flags in (B.CF_KEEP_BITMAPS | path, B.CF_KEEP_BITMAPS | B.CF_PLAIN_LAUNCH | path):
        dres, drecs, dbms, ores, orecs, obms, _ = run_both(B, orc, progs, inputs, cap=cap,
                                                           flags=flags, orc_cap=1 << 17)
        compare(B, orc, inputs, dres, drecs, dbms, ores, orecs, obms, cap)


@pytest.mark.parametrize("path", PATHS)
def test_c4_branch_heavy(B, orc, path):
    """Branch-heavy programs: on the compiled path the persistent kernel
    counts paths in its CTAs' path tables, and the plain kernel (no table)
    replays each thread's path."""
    progs = gen.c4_programs()
    inputs = gen.c4_inputs(256, seed=4, max_blocks=12)
    for flags in (B.CF_KEEP_BITMAPS | path, B.CF_KEEP_BITMAPS | B.CF_PLAIN_LAUNCH | path):
        dres, drecs, dbms, ores, orecs, obms, _ = run_both(B, orc, progs, inputs, cap=1 << 13,
                                                           orc_cap=1 << 16, flags=flags)
        compare(B, orc, inputs, dres, drecs, dbms, ores, orecs, obms, 1 << 13)
        assert int(dres["n_edges"].max()) > 50


@pytest.mark.parametrize("path", PATHS)
def test_listing_programs(B, orc, path):
    progs = [gen.vecadd_shared_program(256), gen.guarded_plus1_program(256)]
    inputs = gen.make_inputs(6)
    n = 256 * 40 - 1
    gen.set_input(inputs[0], 0, (40, 1, 1), (256, 1, 1), (), (4 * 10240,) * 3 + (1024, 1024))
    gen.set_input(inputs[1], 0, (40, 1, 1), (256, 1, 1), (), (4 * 10239, 4 * 10240, 4 * 10240, 1024, 1020))
    gen.set_input(inputs[2], 1, (40, 1, 1), (256, 1, 1), (n,), (4 * n,) * 3)
    gen.set_input(inputs[3], 1, (40, 1, 1), (256, 1, 1), (5000,), (4 * 5000,) * 3)
    gen.set_input(inputs[4], 1, (0, 1, 1), (256, 1, 1), (0,), (0,) * 3)
    gen.set_input(inputs[5], 1, (3, 1, 1), (1025, 1, 1), (5,), (0,) * 3)
    dres, drecs, dbms, ores, orecs, obms, _ = run_both(B, orc, progs, inputs,
                                                       flags=B.CF_KEEP_BITMAPS | path)
    compare(B, orc, inputs, dres, drecs, dbms, ores, orecs, obms, 1 << 15)
    assert int(dres[2]["n_violations"]) == 3
    assert int(dres[4]["status"]) == B.ST_INVALID_CONFIG
    assert int(dres[5]["status"]) == B.ST_INVALID_CONFIG


@pytest.mark.parametrize("path", PATHS)
def test_flat_loop_edges(B, orc, path):
    """Loops without branch sites in their bodies, whose head edges the
    compiled path adds in closed form: trip counts that differ between the
    lanes of a warp (0, 1 and many), a loop right after another (its first
    edge follows the previous exit), an IF after the loops, and iteration
    budgets that stop some threads inside a loop and not others."""
    A = bc.Asm(n_bufs=2)
    tx, a0, a1 = A.sreg(bc.TID_X), A.sreg(bc.ARG0), A.sreg(bc.ARG1)
    n1 = A.alu(bc.AND, A.alu(bc.ADD, tx, a0), bc.Imm(15))          # 0..15 per lane
    i = A.loop(n1, 12)
    A.ld(0, A.alu(bc.ADD, i, tx), 4)
    A.endloop()
    n2 = A.alu(bc.SUB, A.alu(bc.AND, tx, bc.Imm(3)), bc.Imm(1))     # -1..2 per lane
    j = A.loop(n2, 64)
    A.st(1, A.alu(bc.MUL, j, a1), tx, 4)
    A.endloop()
    A.if_(A.alu(bc.SETLT, tx, a1))
    A.ld(1, tx, 4)
    A.endif()
    prog = A.build()
    ins = gen.make_inputs(4)
    gen.set_input(ins[0], 0, (3, 1, 1), (96, 1, 1), (0, 40), (400, 400))
    gen.set_input(ins[1], 0, (2, 1, 1), (256, 1, 1), (7, 3), (64, 1 << 12))
    gen.set_input(ins[2], 0, (5, 1, 1), (33, 1, 1), (3, 100), (48, 96))
    gen.set_input(ins[3], 0, (1, 1, 1), (1024, 1, 1), (11, 9), (1 << 14, 4))
    for budget in (4096, 7, 1):
        dres, drecs, dbms, ores, orecs, obms, _ = run_both(
            B, orc, [prog], ins, budget=budget, flags=B.CF_KEEP_BITMAPS | path)
        compare(B, orc, ins, dres, drecs, dbms, ores, orecs, obms, 1 << 15)
        if budget < 12:
            assert all(int(r["flags"]) & B.FL_BUDGET for r in dres)


@pytest.mark.parametrize("path", PATHS)
def test_edge_cases(B, orc, path):
    """Zero-length buffers, every-access violations with a tiny record cap
    (OVERFLOW, exact counts), the back-edge budget, LIMIT, a bad program id,
    3D grids and blocks, one-thread inputs."""
    A = bc.Asm(n_bufs=2, shared_mask=0b10)
    a0, a1 = A.sreg(bc.ARG0), A.sreg(bc.ARG1)
    tz, bz = A.sreg(bc.TID_Z), A.sreg(bc.CTAID_Z)
    ty = A.sreg(bc.TID_Y)
    i = A.loop(a0, 9)
    A.if_(A.alu(bc.SETLT, i, tz))
    j = A.loop(a1, 5)
    A.st(1, A.alu(bc.ADD, j, bz), i, 8)
    A.endloop()
    A.else_()
    A.ld(0, A.alu(bc.SHR, A.alu(bc.SUB, i, ty), bc.Imm(1)), 1)
    A.endif()
    A.endloop()
    p_nested = A.build()
    progs = [p_nested, gen.c1_program()]
    ins = gen.make_inputs(10)
    gen.set_input(ins[0], 0, (3, 2, 2), (5, 3, 4), (7, 4), (5, 24))
    gen.set_input(ins[1], 0, (1, 1, 1), (1, 1, 1), (9, 5), (0, 0))
    gen.set_input(ins[2], 0, (7, 1, 3), (33, 1, 2), (9, 5), (1000, 40))
    gen.set_input(ins[3], 1, (64, 1, 1), (128, 1, 1), (-4, 8192), (0, 0, 0, 0))
    gen.set_input(ins[4], 1, (64, 1, 1), (128, 1, 1), (0, 8192), (4, 8, 12, 16))
    gen.set_input(ins[5], 7, (1, 1, 1), (32, 1, 1), (0, 1), (4, 4, 4, 4))
    gen.set_input(ins[6], 1, (1 << 16, 1, 1), (1024, 1, 1), (0, 1), (4, 4, 4, 4))
    gen.set_input(ins[7], 1, (1, 1, 1), (1, 1, 1), (0, 1), (1 << 48, 4, 4, 4))
    gen.set_input(ins[8], 0, (2, 2, 2), (4, 4, 4), (9, 5), (3, 17))
    # a shape CUDA accepts whose thread count wraps 64 bits to 88,342,528
    gen.set_input(ins[9], 1, (72093556, 65352, 65000), (1024, 1, 1), (0, 1), (4, 4, 4, 4))
    cap = 64
    for budget in (4096, 12):
        with B.Engine(record_cap=cap, iter_budget=budget, max_threads=1 << 24, max_slots=64,
                      flags=B.CF_KEEP_BITMAPS | path) as E:
            E.load(progs[0])
            E.load(progs[1])
            dres, drecs, dbms = E.run(ins)
        o = orc.opts(iter_budget=budget, max_threads=1 << 24)
        keep = [k for k in range(len(ins)) if k != 5]
        ores = np.zeros(len(ins), orc.RESULT_DTYPE)
        orecs = [None] * len(ins)
        obms = np.zeros((len(ins), 65536), np.uint8)
        for k in keep:
            r, rc, bm = orc.run(progs[int(ins[k]["program_id"])], ins[k], o, rec_cap=1 << 20)
            ores[k], orecs[k], obms[k] = r, rc, bm
        sub = np.array(keep)
        compare(B, orc, ins[sub], dres[sub], [drecs[k] for k in keep], dbms[sub], ores[sub],
                [orecs[k] for k in keep], obms[sub], cap)
        assert int(dres[5]["status"]) == B.ST_BAD_PROGRAM
        assert int(dres[6]["status"]) == B.ST_LIMIT and int(dres[7]["status"]) == B.ST_LIMIT
        assert int(dres[9]["status"]) == B.ST_LIMIT and int(dres[9]["n_accesses"]) == 0
        assert int(dres[3]["flags"]) & B.FL_OVERFLOW and int(dres[3]["n_records"]) == cap
        if budget == 12:
            assert int(dres[0]["flags"]) & B.FL_BUDGET


def test_union_and_new_coverage(B, orc):
    progs = gen.c4_programs()[:4]
    inputs = gen.c4_inputs(64, n_programs=4, seed=8, max_blocks=4)
    with B.Engine(record_cap=256, max_slots=128) as E:
        for p in progs:
            E.load(p)
        r1, _, b1 = E.run(inputs, records=False)
        u1 = E.union()
        E.new_epoch()
        r2, _, b2 = E.run(inputs, records=False)
    assert np.array_equal(u1, np.bitwise_or.reduce(b1, axis=0))
    assert np.array_equal(b1, b2)
    assert all((int(r["flags"]) & B.FL_NEW_COV) == (B.FL_NEW_COV if int(r["n_edges"]) else 0)
               for r in r1)
    assert not any(int(r["flags"]) & B.FL_NEW_COV for r in r2)


def test_int32_peak_probe(B):
    v = B.cufz_int32_peak(0, 0)
    assert 1e12 < v < 1e14


def test_mixed_paths_and_autotune(B, orc):
    """Compiled and interpreted programs in one batch (config-5 style mix of
    1D guarded, random 2D and branch-heavy programs): the default (all
    compiled), an alternating split, every program interpreted, and the
    autotuner's choice all agree with the oracle."""
    progs = gen.c3_programs()[:4] + gen.c2_programs()[:4] + gen.c4_programs()[:4]
    c3 = gen.c3_inputs(24, seed=5, max_blocks=16, max_threads=300)
    c3["program_id"] %= 4
    c2 = gen.c2_inputs(progs[4:8], per_program=4, seed=6, max_grid=3)
    c2["program_id"] += 4
    c4 = gen.c4_inputs(16, n_programs=4, seed=7, max_blocks=6)
    c4["program_id"] += 8
    inputs = np.concatenate([c3, c2, c4])
    cap = 1 << 14
    ores, orecs, obms = orc.run_batch(progs, inputs, rec_cap=1 << 17, bitmaps=True)
    with B.Engine(record_cap=cap, max_slots=256, flags=B.CF_KEEP_BITMAPS | B.CF_JIT) as E:
        for p in progs:
            E.load(p)
        default = [B.cufz_get_program_path(E.ctx, k) for k in range(len(progs))]
        assert all(default)
        runs = [E.run(inputs)]
        for split in ((lambda k: k % 2 == 0), (lambda k: False)):
            for k in range(len(progs)):
                B.cufz_set_program_path(E.ctx, k, split(k))
            assert [B.cufz_get_program_path(E.ctx, k) for k in range(len(progs))] == \
                [split(k) for k in range(len(progs))]
            runs.append(E.run(inputs))
        n_comp = B.cufz_autotune(E.ctx, inputs[::3])
        assert 0 <= n_comp <= len(progs)
        runs.append(E.run(inputs))
    for dres, drecs, dbms in runs:
        compare(B, orc, inputs, dres, drecs, dbms, ores, orecs, obms, cap)


@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_lane_mappings(B, orc, lanes):
    """Each lane mapping (test threads per lane per loop iteration of the
    compiled program), forced for every program: configuration 1 and 3
    programs over launch shapes of every kind (blocks smaller than, equal
    to and larger than the CTA, 1D-3D), a few random programs, and a budget
    that stops threads inside loops, bit-exact with the oracle."""
    progs = [gen.c1_program()] + gen.c3_programs()[:4] + gen.c2_programs()[:3]
    c1 = gen.c1_inputs(40, seed=71)
    c3 = gen.c3_inputs(64, seed=72, max_blocks=64)
    c3["program_id"] = 1 + c3["program_id"] % 4
    c2 = gen.c2_inputs(progs[5:], per_program=6, seed=73, max_grid=6)
    c2["program_id"] += 5
    ins = np.concatenate([c1, c3, c2])
    rng = gen.SplitMix64(74)
    for x in ins[-12:]:
        x["grid"] = [rng.randint(1, 4), rng.randint(1, 4), rng.randint(1, 3)]
        x["block"] = [(8, 8, 4), (16, 16, 1), (32, 8, 2), (5, 7, 3)][rng.below(4)]
    for budget in (4096, 9):
        with B.Engine(record_cap=1 << 15, max_slots=512, iter_budget=budget,
                      flags=B.CF_KEEP_BITMAPS | B.CF_JIT) as E:
            for p in progs:
                E.load(p)
            for p in range(len(progs)):
                B.cufz_set_program_lanes(E.ctx, p, lanes)
                assert B.cufz_get_program_lanes(E.ctx, p) == lanes
            dres, drecs, dbms = E.run(ins)
        o = orc.opts(iter_budget=budget)
        ores, orecs, obms = orc.run_batch(progs, ins, o, rec_cap=1 << 15, bitmaps=True)
        compare(B, orc, ins, dres, drecs, dbms, ores, orecs, obms, 1 << 15)
    with B.Engine(flags=B.CF_JIT) as E:
        E.load(progs[0])
        with pytest.raises(B.CufzError):
            B.cufz_set_program_lanes(E.ctx, 0, 3)
