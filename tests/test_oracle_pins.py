"""Pins of the CPU oracle to facts that do not come from the oracle itself:
published hash vectors, AFL's bucket table, the paper's worked examples,
closed forms for affine kernels, the PREX corner theorem and brute force on
tiny grids (an independent evaluator, tests/bruteforce.py)."""
import numpy as np
import pytest

import bruteforce as bf
from conftest import golden
from paper_2601_01048_gb300 import bytecode as bc
from paper_2601_01048_gb300 import gen
from paper_2601_01048_gb300.bytecode import Asm, Imm


def mk(grid=(1, 1, 1), block=(1, 1, 1), args=(), lens=(), pid=0):
    a = gen.make_inputs(1)
    gen.set_input(a[0], pid, grid, block, args, lens)
    return a[0]


def rec_tuples(recs):
    return [(int(r["block_lin"]), int(r["thread_lin"]), int(r["ordinal"]), int(r["site"]),
             int(r["buf"]), int(r["kind"]), int(r["width"]), int(r["space"]), int(r["cls"]),
             int(r["byte_off"])) for r in recs]


# ---------------------------------------------------------------- hashing / tables

def test_fmix32_published_vectors(orc):
    for seed, h in golden("murmur3_fmix32.txt"):
        assert orc.fmix32(int(seed, 16)) == int(h, 16)


def test_splitmix64_published_vectors():
    for row in golden("splitmix64.txt"):
        r = gen.SplitMix64(int(row[0]))
        assert [r.next() for _ in range(3)] == [int(x) for x in row[1:]]


def test_bucket_table_matches_afl(orc):
    for lo, hi, val in golden("afl_buckets.txt"):
        lo, hi, val = int(lo), int(hi), int(val)
        for n in {lo, hi, (lo + hi) // 2}:
            assert orc.bucket(n) == val, n
    assert orc.bucket(1 << 40) == 128


def test_loop_edge_counts_closed_form(orc):
    """A loop of trip t: the first head decision is edge LOC1 (prev = 0), the
    t-1 later 'continue' decisions are edge LOC1 ^ (LOC1 >> 1), the exit is
    LOC0 ^ (LOC1 >> 1); the bitmap holds the AFL bucket of each count."""
    A = Asm(n_bufs=1)
    n = A.sreg(bc.ARG0)
    A.loop(n, 65535)
    A.endloop()
    prog = A.build()
    l0, l1 = bc.loc_of(prog)[0]
    P = orc.Program(prog)
    for t in [0, 1, 2, 3, 4, 7, 8, 31, 32, 127, 128, 300]:
        res, _, bm = orc.run(P, mk(args=(t,)))
        expect = {}
        if t == 0:
            expect[l0] = 1
        else:
            for e, c in ((l1, 1), (l1 ^ (l1 >> 1), t - 1), (l0 ^ (l1 >> 1), 1)):
                expect[e] = expect.get(e, 0) + c
        want = {e: bf.afl_class(c) for e, c in expect.items() if c}
        got = {int(e): int(bm[e]) for e in np.nonzero(bm)[0]}
        assert got == want, t
        assert int(res["n_branch"]) == t + 1


# ---------------------------------------------------------------- worked examples

def test_listing3_paper_worked_example(orc):
    for n, bs, blk, thr, off in golden("listing3_guarded.txt"):
        n, bs, blk, thr, off = map(int, (n, bs, blk, thr, off))
        prog = gen.guarded_plus1_program(bs)
        grid = -(-n // bs)
        assert blk == grid - 1 and thr == bs - 2  # the paper's statement for these rows
        res, recs, _ = orc.run(prog, mk((grid, 1, 1), (bs, 1, 1), (n,), (4 * n,) * 3))
        assert int(res["status"]) == orc.ST_VIOLATION
        t = rec_tuples(recs)
        assert {(r[0], r[1]) for r in t} == {(blk, thr)}
        assert sorted(r[3] for r in t) == [0, 1, 2]       # all three access sites
        assert all(r[9] == off and r[8] == orc.CLS_OVERFLOW_RZ for r in t)


@pytest.mark.parametrize("n,bs", [(1000, 256), (1024, 256), (1, 32), (257, 128), (5000, 1024)])
def test_listing3_general_case(orc, n, bs):
    """For any N >= 1 exactly one thread violates, id = N - 1."""
    prog = gen.guarded_plus1_program(bs)
    grid = -(-n // bs)
    res, recs, _ = orc.run(prog, mk((grid, 1, 1), (bs, 1, 1), (n,), (4 * n,) * 3))
    t = rec_tuples(recs)
    assert {(r[0], r[1]) for r in t} == {((n - 1) // bs, (n - 1) % bs)}
    assert len(t) == 3 and int(res["n_violations"]) == 3
    assert int(res["n_accesses"]) == 3 * n


def test_listing3_zero_n_is_invalid_config(orc):
    prog = gen.guarded_plus1_program(64)
    res, _, _ = orc.run(prog, mk((0, 1, 1), (64, 1, 1), (0,), (0,) * 3))
    assert int(res["status"]) == orc.ST_INVALID_CONFIG


def test_listing1_vecadd(orc):
    per_thread = int(golden("listing1_vecadd.txt")[0][0])
    bs, nb = 64, 6
    prog = gen.vecadd_shared_program(bs)
    nel = bs * nb
    lens = (4 * nel, 4 * nel, 4 * nel, 4 * bs, 4 * bs)
    res, recs, _ = orc.run(prog, mk((nb, 1, 1), (bs, 1, 1), (), lens))
    assert int(res["n_accesses"]) == per_thread * nel
    assert int(res["n_violations"]) == 0 and int(res["status"]) == orc.ST_OK
    for short in (0, 1):
        l2 = list(lens)
        l2[short] -= 4
        res, recs, _ = orc.run(prog, mk((nb, 1, 1), (bs, 1, 1), (), l2))
        t = rec_tuples(recs)
        assert len(t) == 1 and (t[0][0], t[0][1]) == (nb - 1, bs - 1) and t[0][4] == short


# ---------------------------------------------------------------- config 1 closed form

def c1_expect(a0, a1, lens_bytes, threads=8192):
    hi = min(a0 + threads, a1)
    g = max(hi - a0, 0)
    neg = max(min(hi, 0) - a0, 0) if g else 0
    viol = []
    for k in range(3):
        L = lens_bytes[k] // 4
        over = max(hi - max(L, a0), 0) if g else 0
        viol.append(neg + over)
    return g, viol


def test_c1_closed_form(orc):
    prog = gen.c1_program()
    inputs = gen.c1_inputs(1000)
    res, recs, bms = orc.run_batch([prog], inputs, rec_cap=1 << 15, bitmaps=True)
    l0, l1 = bc.loc_of(prog)[0]
    for k in range(len(inputs)):
        a0, a1 = int(inputs[k]["args"][0]), int(inputs[k]["args"][1])
        g, viol = c1_expect(a0, a1, [int(x) for x in inputs[k]["buf_len"]])
        r = res[k]
        assert int(r["n_accesses"]) == 3 * g
        assert int(r["n_violations"]) == sum(viol)
        assert int(r["n_branch"]) == 8192
        got = recs[k][: int(r["n_records"])]
        for site in range(3):
            assert int((got["site"] == site).sum()) == viol[site]
        assert np.all(got["cls"][got["byte_off"] < 0] == orc.CLS_UNDERFLOW_RZ)
        want = {}
        for e, c in ((l1, g), (l0, 8192 - g)):
            if c:
                want[e] = want.get(e, 0) + c
        bm = bms[k]
        assert {int(e): int(bm[e]) for e in np.nonzero(bm)[0]} == \
            {e: bf.afl_class(c) for e, c in want.items()}


# ---------------------------------------------------------------- hand-built cases

def unguarded_1d(width=4, n_bufs=1, shared_mask=0, buf=0):
    A = Asm(n_bufs=n_bufs, shared_mask=shared_mask)
    i = A.alu(bc.ADD, A.sreg(bc.TID_X), A.sreg(bc.ARG0))
    A.ld(buf, i, width)
    return A.build()


@pytest.mark.parametrize("k", [1, 5, 64, 100])
def test_negative_index(orc, k):
    prog = unguarded_1d()
    res, recs, _ = orc.run(prog, mk((1, 1, 1), (128, 1, 1), (-k,), (4 * 128,)))
    t = rec_tuples(recs)
    assert [r[1] for r in t] == list(range(k))
    assert [r[9] for r in t] == [4 * (tid - k) for tid in range(k)]
    for r in t:
        assert r[8] == (orc.CLS_UNDERFLOW_RZ if r[9] >= -256 else orc.CLS_WILD)


def test_other_alloc_and_wild(orc):
    # A (64 B) at base 256, B (64 B) at base align256(256+64+256) = 768
    A = Asm(n_bufs=2)
    A.ld(0, A.sreg(bc.ARG0), 4)
    prog = A.build()
    cases = [(128, orc.CLS_OTHER_ALLOC),   # off 512 -> address 768 = start of B
             (143, orc.CLS_OTHER_ALLOC),   # last word of B
             (144, orc.CLS_WILD),          # just past B
             (16, orc.CLS_OVERFLOW_RZ),    # off 64 = len
             (79, orc.CLS_OVERFLOW_RZ),    # off 316 < len + R = 320
             (80, orc.CLS_WILD),           # off 320
             (-64, orc.CLS_UNDERFLOW_RZ),  # off -256 = -R
             (-65, orc.CLS_WILD)]
    for idx, cls in cases:
        _, recs, _ = orc.run(prog, mk(args=(idx,), lens=(64, 64)))
        assert len(recs) == 1 and int(recs[0]["cls"]) == cls, idx


def test_other_alloc_needs_same_space(orc):
    # buffer 1 shared: an access of global buffer 0 cannot land in it
    A = Asm(n_bufs=2, shared_mask=0b10)
    A.ld(0, A.sreg(bc.ARG0), 4)
    _, recs, _ = orc.run(A.build(), mk(args=(128,), lens=(64, 64)))
    assert int(recs[0]["cls"]) == orc.CLS_WILD


def test_shared_overflow_per_block(orc):
    prog = unguarded_1d(n_bufs=1, shared_mask=1)
    bs, nb = 32, 5
    res, recs, _ = orc.run(prog, mk((nb, 1, 1), (bs, 1, 1), (0,), (4 * bs - 4,)))
    t = rec_tuples(recs)
    assert [(r[0], r[1]) for r in t] == [(b, bs - 1) for b in range(nb)]
    assert all(r[7] == 1 and r[8] == orc.CLS_OVERFLOW_RZ for r in t)


def test_zero_length_buffer(orc):
    prog = unguarded_1d()
    res, recs, _ = orc.run(prog, mk((2, 1, 1), (16, 1, 1), (0,), (0,)))
    assert int(res["n_violations"]) == int(res["n_accesses"]) == 32


def test_loaded_values_are_seeded_content(orc):
    """A loaded value steers a branch: the IF is taken iff the loaded word's
    low bit (fmix32 of seed ^ buf*0x9E3779B9 ^ word) is set."""
    A = Asm(n_bufs=2, seed=1234)
    i = A.sreg(bc.TID_X)
    v = A.ld(1, i, 4)
    A.if_(A.alu(bc.AND, v, Imm(1)))
    A.endif()
    prog = A.build()
    l0, l1 = bc.loc_of(prog)[0]
    res, _, bm = orc.run(prog, mk((1, 1, 1), (64, 1, 1), (), (0, 4 * 64)))
    taken = sum(orc.fmix32(1234 ^ 0x9E3779B9 ^ j) & 1 for j in range(64))
    assert bm[l1] == bf.afl_class(taken) and bm[l0] == bf.afl_class(64 - taken)


INVALID = [((0, 1, 1), (1, 1, 1)), ((1, 0, 1), (1, 1, 1)), ((1, 1, 0), (1, 1, 1)),
           ((1, 1, 1), (0, 1, 1)), ((1, 1, 1), (1025, 1, 1)), ((1, 1, 1), (1, 1, 65)),
           ((1, 1, 1), (64, 32, 1)), ((1, 65536, 1), (1, 1, 1)), ((1, 1, 65536), (1, 1, 1)),
           ((2 ** 31, 1, 1), (1, 1, 1))]


@pytest.mark.parametrize("grid,block", INVALID)
def test_invalid_launch_configs(orc, grid, block):
    res, recs, bm = orc.run(unguarded_1d(), mk(grid, block, (0,), (4,)))
    assert int(res["status"]) == orc.ST_INVALID_CONFIG
    assert int(res["n_accesses"]) == 0 and not bm.any()


WRAPPING_GRID = (72093556, 65352, 65000)


def test_limit_status(orc):
    o = orc.opts(max_threads=1000)
    res, _, _ = orc.run(unguarded_1d(), mk((4, 1, 1), (256, 1, 1), (0,), (4,)), o)
    assert int(res["status"]) == orc.ST_LIMIT
    res, _, _ = orc.run(unguarded_1d(), mk((1, 1, 1), (1, 1, 1), (0,), (1 << 48,)))
    assert int(res["status"]) == orc.ST_LIMIT
    # a shape CUDA accepts whose thread count (about 3e20) wraps 64 bits to
    # 88,342,528: above every limit, so LIMIT, never run as the wrapped count
    res, _, _ = orc.run(unguarded_1d(), mk(WRAPPING_GRID, (1024, 1, 1), (0,), (4,)))
    assert int(res["status"]) == orc.ST_LIMIT


def test_budget_closed_form(orc):
    A = Asm(n_bufs=1)
    a0, a1 = A.sreg(bc.ARG0), A.sreg(bc.ARG1)
    A.loop(a0, 100)
    j = A.loop(a1, 100)
    A.ld(0, j, 4)
    A.endloop()
    A.endloop()
    prog = A.build()
    budget, t0, t1 = 50, 10, 7
    res, _, _ = orc.run(prog, mk((1, 1, 1), (3, 1, 1), (t0, t1), (4 * 100,)),
                        orc.opts(iter_budget=budget))
    bodies = (budget + 1) - (budget + 1) // (t1 + 1)
    assert int(res["flags"]) & orc.FL_BUDGET
    assert int(res["n_accesses"]) == 3 * bodies
    res, _, _ = orc.run(prog, mk((1, 1, 1), (3, 1, 1), (t0, t1), (4 * 100,)),
                        orc.opts(iter_budget=t0 * (t1 + 1)))
    assert not int(res["flags"]) & orc.FL_BUDGET and int(res["n_accesses"]) == 3 * t0 * t1


def test_loop_counter_after_exit(orc):
    """for (i = 0; i < trip; i++) leaves i == trip (also for trip 0): the
    counter indexes an access after the loop."""
    A = Asm(n_bufs=1)
    r = A.imm(5)
    c = A.loop(A.sreg(bc.ARG0), 9)
    A.endloop()
    A.ld(0, A.alu(bc.ADD, c, Imm(-100)), 4)
    prog = A.build()
    assert r != c
    for t, want in ((0, 0), (3, 3), (50, 9)):
        _, recs, _ = orc.run(prog, mk(args=(t,), lens=(4,)))
        assert int(recs[0]["byte_off"]) == 4 * (want - 100)


def test_overflow_flag_and_exact_count(orc):
    prog = unguarded_1d()
    res, recs, _ = orc.run(prog, mk((4, 1, 1), (64, 1, 1), (-1000,), (4,)), rec_cap=10)
    assert int(res["n_violations"]) == 256 and len(recs) == 10
    assert int(res["flags"]) & orc.FL_OVERFLOW
    assert int(res["first_key"]) == 0


def test_first_key_packing(orc):
    prog = gen.guarded_plus1_program(128)
    res, recs, _ = orc.run(prog, mk((4, 1, 1), (128, 1, 1), (300,), (1200,) * 3))
    assert int(res["first_key"]) == (2 << 32) | (299 - 256) << 22 | 0


# ---------------------------------------------------------------- validation

def _bad_programs():
    out = {}
    A = Asm(n_bufs=1)
    c = A.loop(A.sreg(bc.ARG0), 4)
    A.raw(bc.ADD | bc.IMM_FORM, c, c, 0, 1)   # writes its own loop counter
    A.endloop()
    out["loopctr"] = A.build()
    good = gen.c1_program()
    out["truncated"] = good[:-1]
    b = bytearray(good)
    b[0] ^= 1
    out["magic"] = bytes(b)
    A = Asm(n_bufs=1)
    A.raw(bc.LD, 0, 0, 0, 3)                  # width 3
    A.n_regs = 1
    out["width"] = A.build()
    A = Asm(n_bufs=1)
    A.raw(bc.LD, 0, 0, 1, 4)                  # buffer 1 of 1
    A.n_regs = 1
    out["buf"] = A.build()
    A = Asm(n_bufs=1)
    A.raw(bc.ENDIF)
    out["unbalanced"] = A.build()
    A = Asm(n_bufs=1)
    r = A.imm(1)
    for _ in range(17):
        A.if_(r)
    for _ in range(17):
        A.endif()
    out["depth"] = A.build()
    return out


@pytest.mark.parametrize("name", ["loopctr", "truncated", "magic", "width", "buf", "unbalanced",
                                  "depth"])
def test_rejects_malformed(orc, name):
    assert orc.validate(_bad_programs()[name]) < 0


# ---------------------------------------------------------------- PREX theorem

def affine_program(rng, dims, n_access):
    """Unguarded accesses whose indices are sum_d M_d tid_d + N_d ctaid_d + C
    with thread-invariant coefficients (the paper's affine-access class)."""
    A = Asm(n_bufs=3)
    tids = [A.sreg(bc.TID_X + d) for d in range(dims)]
    ctas = [A.sreg(bc.CTAID_X + d) for d in range(dims)]
    for _ in range(n_access):
        acc = A.sreg(bc.ARG0 + rng.below(4))
        for v in tids + ctas:
            acc = A.alu(bc.ADD, acc, A.alu(bc.MUL, v, Imm(rng.randint(-6, 6))))
        acc = A.alu(bc.ADD, acc, Imm(rng.randint(-8, 8)))
        if rng.chance(0.5):
            A.ld(rng.below(3), acc, rng.choice(bc.WIDTHS))
        else:
            A.st(rng.below(3), acc, acc, rng.choice(bc.WIDTHS))
    return A.build()


def test_prex_corner_theorem(orc):
    """Sec. 5.1.1 Theorem: in an affine-access kernel with unguarded accesses,
    if any thread violates at a site then one of the corner threads (each
    block and thread coordinate first or last) violates there too."""
    rng = gen.SplitMix64(77)
    checked = 0
    for trial in range(60):
        dims = 1 + trial % 3
        prog = affine_program(rng, dims, 4)
        P = orc.Program(prog)
        for _ in range(4):
            grid = [rng.randint(1, 5) for _ in range(dims)] + [1] * (3 - dims)
            block = [rng.randint(1, 6) for _ in range(dims)] + [1] * (3 - dims)
            args = [rng.randint(-20, 60) for _ in range(4)]
            lens = [rng.randint(0, 400) for _ in range(3)]
            res, recs, _ = orc.run(P, mk(grid, block, args, lens), rec_cap=1 << 17)
            assert int(res["n_records"]) == int(res["n_violations"])

            def corner(lin, ext):
                c = [lin % ext[0], (lin // ext[0]) % ext[1], lin // (ext[0] * ext[1])]
                return all(v in (0, e - 1) for v, e in zip(c, ext))

            sites = {int(r["site"]) for r in recs}
            corner_sites = {int(r["site"]) for r in recs
                            if corner(int(r["block_lin"]), grid) and corner(int(r["thread_lin"]), block)}
            assert sites == corner_sites
            checked += len(sites)
    assert checked > 20


def test_prex_guarded_1d_interval_theorem(orc):
    """The extension of Sec. 5.1.1's theorem to guarded 1D kernels (the case
    the paper leaves to its heuristic Alg. 1): when every value is affine in
    lin = ctaid.x * ntid.x + tid.x and the guard is `lin + c < a1`, the threads
    reaching the accesses are an interval of lin, so the threads at 0, N - 1
    and the guard's threshold t = a1 - c (and t +- 1) decide, site by site,
    whether any thread violates.  Checked on configuration 3's guarded
    program family over random small launches with off-by-one lengths."""
    rng = gen.SplitMix64(99)
    progs = gen.c3_programs()
    offsets = []
    rp = gen.SplitMix64(gen.sub_seed("c3prog"))
    for p in range(16):
        offsets.append(rp.randint(-3, 3) if p else 0)
        rp.next32()
    sites_checked = 0
    for trial in range(120):
        p = trial % 16
        w = gen.C3_WIDTHS[p]
        nb, nt = rng.randint(1, 9), rng.randint(1, 40)
        n = nb * nt
        a0, a1 = rng.randint(-4, 4), rng.randint(-2, n + 3)
        lens = [w * max(rng.randint(a1 - 3, a1 + 2), 0) for _ in range(4)]
        res, recs, _ = orc.run(orc.Program(progs[p]), mk((nb, 1, 1), (nt, 1, 1), (a0, a1), lens),
                               rec_cap=1 << 16)
        assert int(res["n_records"]) == int(res["n_violations"])
        t = a1 - (a0 + offsets[p])
        cand = {0, n - 1} | {v for v in (t - 1, t, t + 1) if 0 <= v < n}

        def lin(r):
            return int(r["block_lin"]) * nt + int(r["thread_lin"])

        sites = {int(r["site"]) for r in recs}
        assert sites == {int(r["site"]) for r in recs if lin(r) in cand}
        sites_checked += len(sites)
    assert sites_checked > 40


# ---------------------------------------------------------------- brute force

def _compare_bruteforce(orc, prog, inp_kwargs, budget=4096):
    rec = mk(**inp_kwargs)
    res, recs, bm = orc.run(prog, rec, orc.opts(iter_budget=budget), rec_cap=1 << 16)
    ref = bf.evaluate(prog, dict(grid=inp_kwargs["grid"], block=inp_kwargs["block"],
                                 args=list(inp_kwargs["args"]) + [0] * 4,
                                 lens=inp_kwargs["lens"]), budget=budget)
    assert rec_tuples(recs) == ref["records"]
    assert int(res["digest"]) == ref["digest"]
    assert int(res["n_accesses"]) == ref["n_accesses"]
    assert int(res["n_branch"]) == ref["n_branch"]
    assert int(res["first_key"]) == ref["first_key"]
    assert int(res["n_ops"]) == ref["n_ops"]
    assert int(res["flags"]) & 1 == ref["flags"]
    assert {int(e): int(bm[e]) for e in np.nonzero(bm)[0]} == bf.bitmap_of(ref["counts"])


@pytest.mark.parametrize("index", range(12))
def test_bruteforce_random_programs(orc, index):
    prog = gen.c2_program(index)
    h = bc.decode_header(prog)
    rng = gen.SplitMix64(1000 + index)
    for _ in range(2):
        lens = [rng.choice((0, 1, 4, 16, 64, 256, 1024, 4096)) + rng.randint(-1, 1) * 4
                for _ in range(h["n_bufs"])]
        lens = [max(x, 0) for x in lens]
        args = [rng.choice((0, -1, 1, 3, 16, 255, -7)) for _ in range(4)]
        _compare_bruteforce(orc, prog, dict(grid=(rng.randint(1, 3), rng.randint(1, 2), 1),
                                            block=(rng.randint(1, 4), rng.randint(1, 4), 1),
                                            args=args, lens=lens))


@pytest.mark.parametrize("index", range(4))
def test_bruteforce_branchy_programs(orc, index):
    prog = gen.c4_program(index)
    rng = gen.SplitMix64(2000 + index)
    for _ in range(2):
        args = [rng.choice((0, -1, 1, 5, 100, 1 << 20, -(1 << 30))) for _ in range(4)]
        _compare_bruteforce(orc, prog, dict(grid=(rng.randint(1, 3), 1, 1), block=(8, 1, 1),
                                            args=args, lens=(4 * 4096, 4 * 1024, 64)))


def test_bruteforce_budget_and_3d(orc):
    A = Asm(n_bufs=2, shared_mask=0b10)
    a0, a1 = A.sreg(bc.ARG0), A.sreg(bc.ARG1)
    tz = A.sreg(bc.TID_Z)
    bz = A.sreg(bc.CTAID_Z)
    i = A.loop(a0, 9)
    A.if_(A.alu(bc.SETLT, i, tz))
    j = A.loop(a1, 5)
    A.st(1, A.alu(bc.ADD, j, bz), i, 8)
    A.endloop()
    A.else_()
    A.ld(0, A.alu(bc.SHR, A.alu(bc.SUB, i, Imm(3)), Imm(1)), 1)
    A.endif()
    A.endloop()
    prog = A.build()
    for budget in (3, 12, 4096):
        _compare_bruteforce(orc, prog, dict(grid=(1, 2, 2), block=(2, 1, 3), args=(7, 4),
                                            lens=(5, 24)), budget=budget)


def test_batch_equals_single_runs(orc):
    progs = [gen.c1_program(), gen.c2_program(3)]
    ins = gen.c1_inputs(6)
    ins2 = gen.c2_inputs([progs[1]], per_program=3, max_grid=3)
    ins2["program_id"] = 1
    allin = np.concatenate([ins, ins2])
    res, recs, bms = orc.run_batch(progs, allin, rec_cap=4096, bitmaps=True, threads=3)
    for k in range(len(allin)):
        r1, rc1, bm1 = orc.run(progs[int(allin[k]["program_id"])], allin[k], rec_cap=4096)
        assert res[k].tobytes() == r1.tobytes()
        assert recs[k][: int(r1["n_records"])].tobytes() == rc1.tobytes()
        assert np.array_equal(bms[k], bm1)


def _trunc_div(x, y):
    """C's truncating division, from Python's floor division."""
    q = abs(x) // abs(y)
    return q if (x >= 0) == (y >= 0) else -q


def test_division_values_faults_and_ordinals(orc):
    """q = a0 / (tid - a1); r = a0 % (tid - a1); two 1-byte loads at q and r
    from a zero-length buffer, so every load violates and its record's
    byte offset shows the index.  Values: C truncation (checked against
    Python's floor division), INT_MIN / -1 = INT_MIN with remainder 0.  A
    zero divisor: two fault records (kind 2, class DIV_ZERO, division sites 0
    and 1) and 0 as both results.  Ordinals count divisions and accesses
    alike (faults at 0 and 1, loads at 2 and 3); n_accesses counts loads
    only."""
    A = Asm(n_bufs=1)
    d = A.alu(bc.SUB, A.sreg(bc.TID_X), A.sreg(bc.ARG1))
    a0 = A.sreg(bc.ARG0)
    q, r = A.div(a0, d), A.rem(a0, d)
    A.ld(0, q, 1)
    A.ld(0, r, 1)
    prog = A.build()
    for a0v, a1v in ((-7, 5), (7, 3), (-(1 << 31), 1), (1 << 31 - 1, 15)):
        res, recs, _ = orc.run(orc.Program(prog), mk((2, 1, 1), (16, 1, 1), (a0v, a1v), (0,)),
                               rec_cap=1 << 10)
        assert int(res["n_accesses"]) == 64
        faults = [x for x in recs if int(x["kind"]) == 2]
        loads = [x for x in recs if int(x["kind"]) == 0]
        assert len(loads) == 64 and int(res["n_violations"]) == 64 + len(faults)
        zero_threads = [t for t in range(16) if t - a1v == 0]
        assert len(faults) == 2 * 2 * len(zero_threads)
        for f in faults:
            assert int(f["thread_lin"]) in zero_threads and int(f["cls"]) == 5
            assert int(f["ordinal"]) == int(f["site"]) and int(f["buf"]) == 0
            assert int(f["width"]) == 0 and int(f["byte_off"]) == 0
        for x in loads:
            t, dv = int(x["thread_lin"]), int(x["thread_lin"]) - a1v
            if dv == 0:
                want = 0
            elif a0v == -(1 << 31) and dv == -1:
                want = -(1 << 31) if int(x["ordinal"]) == 2 else 0
            else:
                qv = _trunc_div(a0v, dv)
                want = qv if int(x["ordinal"]) == 2 else a0v - dv * qv
            assert int(x["byte_off"]) == want, (a0v, a1v, t, int(x["ordinal"]))
            assert int(x["ordinal"]) in (2, 3)
        assert int(res["first_key"]) == 2 or (0 in zero_threads and int(res["first_key"]) == 0)


def test_division_leaves_the_digest_and_counts_as_a_check(orc):
    """A division whose result is unused changes neither the digest nor the
    access count; it moves the accesses' ordinals (and so the first key) by
    one, and faults in every thread whose divisor is 0."""
    def prog(with_div):
        A = Asm(n_bufs=1)
        tx = A.sreg(bc.TID_X)
        if with_div:
            A.div(A.sreg(bc.ARG0), tx)
        A.ld(0, A.alu(bc.SUB, tx, Imm(3)), 4)
        return A.build()
    inp = mk((3, 1, 1), (8, 1, 1), (11,), (4 * 8,))
    r0, c0, _ = orc.run(orc.Program(prog(False)), inp, rec_cap=64)
    r1, c1, _ = orc.run(orc.Program(prog(True)), inp, rec_cap=64)
    assert int(r0["digest"]) == int(r1["digest"]) and int(r0["n_accesses"]) == int(r1["n_accesses"])
    assert int(r1["n_violations"]) == int(r0["n_violations"]) + 3          # tid 0 in each block
    assert int(r0["first_key"]) == 0 and int(r1["first_key"]) == 0          # the fault, ordinal 0
    assert sorted(int(x["ordinal"]) for x in c1 if int(x["kind"]) == 0) == \
        sorted(int(x["ordinal"]) + 1 for x in c0)


@pytest.mark.parametrize("index", range(8))
def test_bruteforce_division_programs(orc, index):
    """Random programs with divisions (zero divisors from coordinates,
    masked arguments and loaded bytes; quotients as indices, in branches and
    in a loop): the oracle equals the independent evaluator exactly."""
    prog = gen.div_program(index)
    for x in gen.div_inputs(3, n_programs=1, seed=3000 + index, max_blocks=3):
        _compare_bruteforce(orc, prog, dict(grid=tuple(int(v) for v in x["grid"]),
                                            block=tuple(int(v) for v in x["block"]),
                                            args=[int(v) for v in x["args"]],
                                            lens=[int(v) for v in x["buf_len"][:3]]))
    res, recs, _ = orc.run(orc.Program(prog), gen.div_inputs(1, n_programs=1, seed=9)[0],
                           rec_cap=1 << 12)
    assert int(res["n_accesses"]) > 0


def test_heap_faults_by_class(orc):
    """One block of a0 = 16 bytes per thread: a 4-byte store at tid * 4
    overflows for tid >= 4; after the free, a load is a use after free and a
    second free a double free; freeing handle 3 (no such block) is an
    invalid free and freeing 0 nothing; a zero-size allocation gives the
    NULL handle, through which a load is wild.  Ordinals count every heap
    access and free (NULL included) but no allocation."""
    A = Asm(n_bufs=0)
    tx, a0, a1 = A.sreg(bc.TID_X), A.sreg(bc.ARG0), A.sreg(bc.ARG1)
    h = A.halloc(a0)
    A.hst(h, tx, tx, 4)                    # ordinal 0
    A.hfree(h)                             # 1
    A.hld(h, A.imm(0), 4)                  # 2: use after free
    A.hfree(h)                             # 3: double free
    A.hfree(A.imm(3))                      # 4: invalid free
    A.hfree(A.imm(0))                      # 5: free(NULL)
    A.hld(A.halloc(a1), A.imm(0), 1)       # 6: NULL handle, wild
    res, recs, _ = orc.run(orc.Program(A.build()), mk((1, 1, 1), (8, 1, 1), (16, 0), ()),
                           rec_cap=256)
    got = sorted((int(r["thread_lin"]), int(r["ordinal"]), int(r["kind"]), int(r["cls"]),
                  int(r["space"]), int(r["byte_off"])) for r in recs)
    want = sorted([(t, 0, 1, 2, 2, 4 * t) for t in range(4, 8)] +
                  [(t, 2, 0, 6, 2, 0) for t in range(8)] + [(t, 3, 3, 7, 2, 0) for t in range(8)] +
                  [(t, 4, 3, 8, 2, 0) for t in range(8)] + [(t, 6, 0, 4, 2, 0) for t in range(8)])
    assert got == want
    assert int(res["n_accesses"]) == 3 * 8 and int(res["n_violations"]) == len(want)
    assert int(res["first_key"]) == 2                      # thread 0's use after free


def test_heap_reallocation_and_failed_frees(orc):
    """A site's later HALLOC replaces its block (sizes 1 then 2 in a loop,
    after a NULL allocation that changes nothing); a failed free leaves the
    heap as it was (the freed block stays freed: the next load is a use
    after free); a second site's block has its own handle and size."""
    A = Asm(n_bufs=0)
    k = A.loop(A.imm(3), 3)
    A.hst(A.halloc(k), A.imm(1), k, 1)     # ordinals 0-2: NULL (wild), 1 byte (over), 2 bytes
    A.endloop()
    one = A.imm(1)
    A.hld(one, A.imm(1), 1)                # 3: block 0 has 2 bytes
    A.hfree(one)                           # 4
    A.hfree(A.imm(5))                      # 5: invalid free, nothing changes
    A.hld(one, A.imm(0), 1)                # 6: use after free
    h2 = A.halloc(A.imm(8))                # site 1: handle 2
    A.hld(h2, A.imm(7), 1)                 # 7: in bounds
    A.hst(h2, A.imm(2), h2, 4)             # 8: bytes 8-11 of 8
    res, recs, _ = orc.run(orc.Program(A.build()), mk((1, 1, 1), (1, 1, 1), (), ()), rec_cap=64)
    assert rec_tuples(recs) == [(0, 0, 0, 0, 0, 1, 1, 2, 4, 1), (0, 0, 1, 0, 0, 1, 1, 2, 2, 1),
                                (0, 0, 5, 1, 0, 3, 0, 2, 8, 0), (0, 0, 6, 2, 0, 0, 1, 2, 6, 0),
                                (0, 0, 8, 4, 1, 1, 4, 2, 2, 8)]
    assert int(res["n_accesses"]) == 7


@pytest.mark.parametrize("index", range(8))
def test_bruteforce_heap_programs(orc, index):
    """Random heap programs (allocation sizes from arguments and
    coordinates, fabricated handles, frees under guards and in a loop): the
    oracle equals the independent evaluator exactly."""
    prog = gen.heap_program(index)
    for x in gen.heap_inputs(3, n_programs=1, seed=4000 + index, max_blocks=2):
        _compare_bruteforce(orc, prog, dict(grid=tuple(int(v) for v in x["grid"]),
                                            block=tuple(int(v) for v in x["block"]),
                                            args=[int(v) for v in x["args"]],
                                            lens=[int(v) for v in x["buf_len"][:1]]))


# ------------------------------------------------ performed shared stores and barriers

def _exchange_program(flag, barrier):
    """Each thread t of 8 stores 3 t to its tile word S[t]; then, after the
    barrier, reads its neighbour's word S[(t + 1) & 7] and loads G at that
    value - 12 (G: 8 words)."""
    A = Asm(n_bufs=2, shared_mask=0b10, shared_stores=flag)
    t = A.sreg(bc.TID_X)
    A.st(1, t, A.alu(bc.MUL, t, Imm(3)), 4)
    if barrier:
        A.bar()
    v = A.ld(1, A.alu(bc.AND, A.alu(bc.ADD, t, Imm(1)), Imm(7)), 4)
    A.ld(0, A.alu(bc.SUB, v, Imm(12)), 4)
    return A.build()


def test_shared_stores_cross_a_barrier(orc):
    """Sec. 5.2's barriers order shared stores: after the barrier thread t
    reads 3 u, u = (t + 1) & 7, written by thread u, and its index 3 u - 12
    leaves G (8 words) for u in {0, 1, 2, 3, 7}, i.e. t in {7, 0, 1, 2, 6}."""
    res, recs, _ = orc.run(orc.Program(_exchange_program(True, True)),
                           mk((2, 1, 1), (8, 1, 1), (), (32, 32)), rec_cap=64)
    got = sorted((int(r["block_lin"]), int(r["thread_lin"]), int(r["ordinal"]), int(r["buf"]),
                  int(r["byte_off"])) for r in recs)
    want = sorted((b, t, 2, 0, 4 * (3 * ((t + 1) & 7) - 12))
                  for b in range(2) for t in (7, 0, 1, 2, 6))
    assert got == want and int(res["n_accesses"]) == 2 * 8 * 3


def test_shared_stores_without_the_barrier_run_in_thread_order(orc):
    """Without the barrier a block runs as one phase, thread after thread:
    thread t < 7 reads S[t + 1] before its owner wrote it (0, index -12);
    thread 7 reads S[0] = 0, written by thread 0.  Without the flag nothing
    is stored and every read gives 0."""
    inp = mk((1, 1, 1), (8, 1, 1), (), (32, 32))
    for flag, barrier in ((True, False), (False, True), (False, False)):
        res, recs, _ = orc.run(orc.Program(_exchange_program(flag, barrier)), inp, rec_cap=64)
        assert sorted((int(r["thread_lin"]), int(r["byte_off"])) for r in recs) == \
            [(t, -48) for t in range(8)], (flag, barrier)


def test_shared_store_widths(orc):
    """Thread 0 stores 0x1234 at width 1 (byte 0x34) to byte 0, -1 at width
    8 (ff ff ff ff 00 00 00 00) to bytes 8-15, and 7 at width 4 to bytes
    16-19; after the barrier each thread reads them back and uses them as
    indices into G (length 0: every access violates, byte_off = 4 index).
    An out-of-bounds store (bytes 64-67) stores nothing."""
    A = Asm(n_bufs=2, shared_mask=0b10, shared_stores=True)
    t = A.sreg(bc.TID_X)
    A.if_(A.alu(bc.SETEQ, t, Imm(0)))
    A.st(1, A.imm(0), A.imm(0x1234), 1)
    A.st(1, A.imm(1), A.imm(-1), 8)
    A.st(1, A.imm(4), A.imm(7), 4)
    A.st(1, A.imm(16), A.imm(9), 4)
    A.endif()
    A.bar()
    for idx, w in ((0, 1), (1, 1), (2, 4), (3, 4), (4, 4), (8, 1), (16, 4)):
        A.ld(0, A.ld(1, A.imm(idx), w), 4)
    res, recs, _ = orc.run(orc.Program(A.build()), mk((1, 1, 1), (2, 1, 1), (), (0, 64)),
                           rec_cap=64)
    loads = sorted((int(r["thread_lin"]), int(r["ordinal"]), int(r["byte_off"]))
                   for r in recs if int(r["buf"]) == 0)
    values = [0x34, 0, -1, 0, 7, 0xFF, 0]     # byte 1 was never written; byte 8 is ff
    base = (4, 0)                             # thread 0 ran the four stores first
    want = sorted((th, base[th] + 2 * k + 1, 4 * v) for th in range(2)
                  for k, v in enumerate(values))
    assert loads == want
    tile = sorted((int(r["thread_lin"]), int(r["ordinal"]), int(r["kind"]), int(r["byte_off"]))
                  for r in recs if int(r["buf"]) == 1)
    # the store at bytes 64-67 and both threads' read of them leave the tile
    assert tile == [(0, 3, 1, 64), (0, 16, 0, 64), (1, 12, 0, 64)]


@pytest.mark.parametrize("index", range(8))
def test_bruteforce_barrier_programs(orc, index):
    """Random programs with performed shared stores in phases (values read
    from the tiles stored on, and, for odd indices, used as indices and
    branch conditions): the oracle equals the independent evaluator, which
    runs each block's threads as generators from barrier to barrier."""
    prog = gen.barrier_program(index // 2, live=bool(index & 1))
    for x in gen.barrier_inputs(3, n_programs=1, seed=5000 + index, max_blocks=2):
        _compare_bruteforce(orc, prog, dict(grid=tuple(int(v) for v in x["grid"]),
                                            block=tuple(int(v) for v in x["block"]),
                                            args=[int(v) for v in x["args"]],
                                            lens=[int(v) for v in x["buf_len"][:4]]))


def test_a_thread_stopped_by_the_budget_runs_no_later_phase(orc):
    """Thread 0 alone loops past the back-edge budget in the first phase
    and stops; after the barrier only threads 1-3 reach the out-of-bounds
    load, and the input carries the budget flag."""
    A = Asm(n_bufs=2, shared_mask=0b10, shared_stores=True)
    t = A.sreg(bc.TID_X)
    A.if_(A.alu(bc.SETEQ, t, Imm(0)))
    A.loop(A.imm(10), 10)
    A.endloop()
    A.endif()
    A.bar()
    A.ld(0, A.imm(-1), 4)
    res, recs, _ = orc.run(orc.Program(A.build()), mk((1, 1, 1), (4, 1, 1), (), (16, 16)),
                           orc.opts(iter_budget=3), rec_cap=64)
    assert [(int(r["thread_lin"]), int(r["byte_off"])) for r in recs] == [(1, -4), (2, -4), (3, -4)]
    assert int(res["flags"]) & orc.FL_BUDGET and int(res["n_accesses"]) == 3


# ---------------------------------------------------------------- digest and op count

def test_digest_hand_derived_golden(orc):
    """The digest, op count, edges and first key of a tiny program equal the
    values worked out by hand in tests/golden/digest_tiny.txt."""
    want = {k: int(v) for k, v in golden("digest_tiny.txt")}
    A = Asm(n_bufs=2, seed=0x7E57)
    tx = A.sreg(bc.TID_X)
    i0 = A.alu(bc.ADD, A.alu(bc.MUL, tx, Imm(3)), Imm(5))
    A.ld(0, i0, 4)
    n = A.sreg(bc.ARG0)
    c = A.loop(n, 4)
    A.ld(1, c, 1)
    A.endloop()
    prog = A.build(loc=[(0x1234, 0xABCD)])
    inp = mk((1, 1, 1), (2, 1, 1), (2,), (64, 1))
    res, recs, bm = orc.run(prog, inp)
    for k in ("digest", "n_ops", "n_accesses", "n_branch", "n_violations", "first_key"):
        assert int(res[k]) == want[k], k
    edges = {int(k[5:], 16): v for k, v in want.items() if k.startswith("edge_")}
    assert {int(e): int(bm[e]) for e in np.nonzero(bm)[0]} == edges
    assert rec_tuples(recs[:2]) == [(0, 0, 2, 1, 1, 0, 1, 0, 2, 1), (0, 1, 2, 1, 1, 0, 1, 0, 2, 1)]


def test_digest_changes_with_each_access(orc):
    """One changed index, two accesses in swapped order, one access dropped:
    each changes D (a constant or order-free digest would fail here)."""
    def prog(index_plus=0, order=("x", "i0"), drop=False):
        A = Asm(n_bufs=2, seed=0x7E57)
        tx = A.sreg(bc.TID_X)
        i0 = A.alu(bc.ADD, A.alu(bc.MUL, tx, Imm(3)), Imm(5))
        x = A.alu(bc.ADD, tx, Imm(1))
        regs = dict(x=x, i0=i0)
        for name in order:
            if not (drop and name == "x"):
                A.ld(0, regs[name], 4)
        n = A.sreg(bc.ARG0)
        c = A.loop(n, 4)
        A.ld(1, A.alu(bc.ADD, c, Imm(index_plus)) if index_plus else c, 1)
        A.endloop()
        return A.build(loc=[(0x1234, 0xABCD)])

    inp = mk((2, 1, 1), (3, 1, 1), (2,), (64, 4))
    base = orc.run(prog(), inp)[0]
    variants = {"index": prog(index_plus=1), "swap": prog(order=("i0", "x")),
                "drop": prog(drop=True)}
    for name, p in variants.items():
        r = orc.run(p, inp)[0]
        assert int(r["digest"]) != int(base["digest"]), name
        # each variant is also what the independent evaluator computes
        ref = bf.evaluate(p, dict(grid=(2, 1, 1), block=(3, 1, 1), args=[2, 0, 0, 0],
                                  lens=[64, 4]))
        assert int(r["digest"]) == ref["digest"], name
    assert int(orc.run(variants["drop"], inp)[0]["n_accesses"]) == int(base["n_accesses"]) - 6


def _ops_of(prog):
    return [prog[32 + 4 * bc.decode_header(prog)["n_sites"] + 8 * k:][:8]
            for k in range(bc.decode_header(prog)["n_ops"])]


def _rebuild(prog, ops):
    h = bytearray(prog[:32 + 4 * bc.decode_header(prog)["n_sites"]])
    h[6:8] = len(ops).to_bytes(2, "little")
    return bytes(h) + b"".join(ops)


@pytest.mark.parametrize("index", range(6))
def test_digest_sensitivity_on_random_programs(orc, index):
    """Random programs with one store dropped, or two adjacent stores
    swapped: whenever some thread's sequence of (site, index) changes (by
    the independent evaluator's trace), the oracle's digest changes, and it
    stays the same when no sequence changes."""
    prog = gen.c2_program(40 + index)
    ops = _ops_of(prog)
    st = [k for k, o in enumerate(ops) if o[0] == bc.ST]
    h = bc.decode_header(prog)
    rng = gen.SplitMix64(4000 + index)
    lens = [rng.choice((16, 64, 256, 1024)) for _ in range(h["n_bufs"])]
    args = [rng.choice((0, 1, 3, 16, -7)) for _ in range(4)]
    kw = dict(grid=(2, 1, 1), block=(3, 2, 1), args=args, lens=lens)
    inp = mk(**kw)
    base_d = int(orc.run(prog, inp)[0]["digest"])
    base_t = bf.evaluate(prog, dict(kw, args=args + [0] * 4))["traces"]
    variants = [ops[:k] + ops[k + 1:] for k in st[:4]]
    variants += [ops[:k] + [ops[k + 1], ops[k]] + ops[k + 2:] for k in st if k + 1 in st][:4]
    changed = 0
    for v in variants:
        p = _rebuild(prog, v)
        assert orc.validate(p) == 0
        d = int(orc.run(p, inp)[0]["digest"])
        t = bf.evaluate(p, dict(kw, args=args + [0] * 4))["traces"]
        assert (d != base_d) == (t != base_t)
        changed += t != base_t
    assert changed >= 1


def test_n_ops_closed_form(orc):
    """Executed ops: a loop of trip t with k ops in its body runs k * t of
    them, the ops of an IF arm run only in the threads taking it, SREG reads
    and accesses are not ops, and a division is one."""
    A = Asm(n_bufs=1)
    tx = A.sreg(bc.TID_X)
    n = A.sreg(bc.ARG0)
    c = A.loop(n, 64)
    v = A.alu(bc.ADD, c, tx)            # 3 ops per iteration
    v = A.alu(bc.XOR, v, Imm(5))
    A.ld(0, A.alu(bc.AND, v, Imm(3)), 4)
    A.endloop()
    A.if_(A.alu(bc.SETLT, tx, Imm(2)))  # 1 op per thread (the condition)
    A.imm(7)                            # 1 op in threads 0 and 1
    A.div(tx, tx)                       # 1 op in threads 0 and 1
    A.endif()
    prog = A.build()
    for t in (0, 1, 5, 64, 100):
        res = orc.run(prog, mk((1, 1, 1), (8, 1, 1), (t,), (16,)))[0]
        trip = min(t, 64)
        assert int(res["n_ops"]) == 8 * 3 * trip + 8 + 2 * 2, t
