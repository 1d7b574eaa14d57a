"""PREX (Sec. 5.1): the engine's eligibility check and plan, pinned to the
oracle.

For every input the corner check accepts, the oracle's full-grid verdict
(some thread violates or none does) must equal the verdict of the corner
threads alone (every block and thread coordinate first or last).  For every
input the plan covers (the corners, or for guarded launches the corners of
the cells the guards cut the launch box into), each access site's verdict
must equal the planned threads' verdict there.  The GPU runs exactly the
plan under CUFZ_CF_PREX.  Inputs that must be refused: thread-dependent
loop trips, indices that are not affine in the thread and block indices,
guards across dimensions, affine values that could wrap int32 in the launch
box, budget stops."""
import numpy as np
import pytest

from paper_2601_01048_gb300 import binding as B
from paper_2601_01048_gb300 import bytecode as bc
from paper_2601_01048_gb300 import gen
from paper_2601_01048_gb300.bytecode import Asm, Imm


def mk(grid, block, args, lens, prog=0):
    ins = gen.make_inputs(1)
    gen.set_input(ins[0], prog, tuple(grid), tuple(block), tuple(args), tuple(lens))
    return ins[0]


def corner(lin, ext):
    c = [lin % ext[0], (lin // ext[0]) % ext[1], lin // (ext[0] * ext[1])]
    return all(v in (0, e - 1) for v, e in zip(c, ext))


def corner_verdict_matches(orc, prog, inp):
    res, recs, _ = orc.run(orc.Program(prog), inp, rec_cap=1 << 20)
    grid, block = [int(v) for v in inp["grid"]], [int(v) for v in inp["block"]]
    full = int(res["n_violations"]) > 0
    at_corners = any(corner(int(r["block_lin"]), grid) and corner(int(r["thread_lin"]), block)
                     for r in recs)
    return full == at_corners, full


def affine_with_extras(rng, dims):
    """Affine accesses (some through a uniform loop, one under a uniform
    branch, a load at a uniform index steering a uniform branch)."""
    A = Asm(n_bufs=3, seed=rng.next32())
    tids = [A.sreg(bc.TID_X + d) for d in range(dims)]
    ctas = [A.sreg(bc.CTAID_X + d) for d in range(dims)]
    a0, a1 = A.sreg(bc.ARG0), A.sreg(bc.ARG1)
    nx = A.sreg(bc.NTID_X)
    lin = A.alu(bc.ADD, A.alu(bc.MUL, ctas[0], nx), tids[0])
    idx = lin
    for v in tids[1:] + ctas[1:]:
        idx = A.alu(bc.ADD, idx, A.alu(bc.MUL, v, Imm(rng.randint(-5, 5))))
    idx = A.alu(bc.ADD, idx, a0)
    A.ld(0, idx, rng.choice(bc.WIDTHS))
    k = A.loop(a1, 6)
    A.st(1, A.alu(bc.SUB, idx, A.alu(bc.SHL, k, Imm(2))), idx, 4)
    A.endloop()
    u = A.ld(2, A.alu(bc.AND, a0, Imm(15)), 4)                   # uniform index: uniform value
    A.if_(A.alu(bc.SETLT, A.alu(bc.AND, u, Imm(7)), Imm(4)))       # uniform branch
    A.ld(2, A.alu(bc.ADD, idx, Imm(rng.randint(-3, 3))), 1)
    A.endif()
    return A.build()


def test_prex_accepts_affine_and_corners_decide(orc):
    rng = gen.SplitMix64(2024)
    from test_oracle_pins import affine_program
    accepted = violating = 0
    for trial in range(48):
        dims = 1 + trial % 3
        prog = affine_program(rng, dims, 4) if trial % 2 else affine_with_extras(rng, dims)
        for _ in range(3):
            grid = [rng.randint(1, 5) for _ in range(dims)] + [1] * (3 - dims)
            block = [rng.randint(1, 6) for _ in range(dims)] + [1] * (3 - dims)
            args = [rng.randint(-20, 60) for _ in range(2)] + [rng.randint(-3, 3) for _ in range(2)]
            inp = mk(grid, block, args, [rng.randint(0, 400) for _ in range(3)])
            assert B.cufz_prex_check(prog, inp)
            ok, full = corner_verdict_matches(orc, prog, inp)
            assert ok
            accepted += 1
            violating += full
    assert accepted == 144 and 20 < violating < 140


def _prog(build):
    A = Asm(n_bufs=2)
    build(A)
    return A.build()


def test_prex_refuses(orc):
    inp = mk((4, 1, 1), (32, 1, 1), (3, 5), (100, 100))
    tx = lambda A: A.sreg(bc.TID_X)
    refused = {
        "thread-dependent branch": _prog(lambda A: (A.if_(A.alu(bc.SETLT, tx(A), A.sreg(bc.ARG0))),
                                                    A.ld(0, tx(A), 4), A.endif())),
        "masked index": _prog(lambda A: A.ld(0, A.alu(bc.AND, tx(A), Imm(7)), 4)),
        "clamped index": _prog(lambda A: A.ld(0, A.alu(bc.MIN, tx(A), A.sreg(bc.ARG1)), 4)),
        "thread-dependent trip": _prog(lambda A: (A.loop(tx(A), 8), A.ld(0, Imm(0) and A.imm(0), 4),
                                                  A.endloop())),
        "loaded index": _prog(lambda A: A.ld(1, A.ld(0, tx(A), 4), 4)),
        "product of indices": _prog(lambda A: A.ld(0, A.alu(bc.MUL, tx(A), A.sreg(bc.CTAID_X)), 4)),
    }
    for name, prog in refused.items():
        assert not B.cufz_prex_check(prog, inp), name
    # an affine index that wraps int32 inside the box is refused; within range accepted
    wrap = _prog(lambda A: A.ld(0, A.alu(bc.MUL, tx(A), A.sreg(bc.ARG0)), 4))
    assert B.cufz_prex_check(wrap, mk((1, 1, 1), (1024, 1, 1), (1 << 20, 0), (64, 64)))
    assert not B.cufz_prex_check(wrap, mk((1, 1, 1), (1024, 1, 1), (1 << 22, 0), (64, 64)))
    # a thread-dependent branch over a 1-thread extent is uniform there
    guarded = refused["thread-dependent branch"]
    assert B.cufz_prex_check(guarded, mk((4, 1, 1), (1, 1, 1), (3, 5), (100, 100)))
    ok, _ = corner_verdict_matches(orc, guarded, mk((4, 1, 1), (1, 1, 1), (3, 5), (100, 100)))
    assert ok


def test_prex_wrap_case_really_breaks_the_theorem(orc):
    """Why values that could wrap are refused: idx = tid.x * (-2^30) in 32-bit
    arithmetic is 0 and 2^30 at the corner threads 0 and 3 (in bounds) but
    wraps to negative indices at the middle threads 1 and 2."""
    A = Asm(n_bufs=1)
    A.ld(0, A.alu(bc.MUL, A.sreg(bc.TID_X), A.sreg(bc.ARG0)), 1)
    prog = A.build()
    inp = mk((1, 1, 1), (4, 1, 1), (-(1 << 30),), (1 << 31,))
    ok, full = corner_verdict_matches(orc, prog, inp)
    assert full and not ok
    assert not B.cufz_prex_check(prog, inp)


# ---------------------------------------------------------------------------
# the plan: the corners, or for guarded launches the cells' corners
# ---------------------------------------------------------------------------

def plan_decides_every_site(orc, prog, inp, plan):
    """The oracle's full grid against the planned threads alone: for every
    access site, some thread violates there iff a planned thread does."""
    res, recs, _ = orc.run(orc.Program(prog), inp, rec_cap=1 << 17, bitmap=False)
    assert int(res["n_records"]) == int(res["n_violations"])        # every record kept
    T = int(np.prod([int(v) for v in inp["block"]]))
    g = recs["block_lin"].astype(np.int64) * T + recs["thread_lin"]
    full = set(recs["site"].tolist())
    planned = set(recs["site"][np.isin(g, plan)].tolist())
    return full == planned, bool(full)


def guarded_1d_program(rng):
    """Accesses at indices affine in lin = ctaid.x * ntid.x + tid.x, under
    nested guards comparing affine values with arguments (<, <=, ==, !=, a
    value tested against zero), with else arms, and inside a uniform loop
    whose guard threshold moves with the counter."""
    A = Asm(n_bufs=3, seed=rng.next32())
    lin = A.alu(bc.ADD, A.alu(bc.MUL, A.sreg(bc.CTAID_X), A.sreg(bc.NTID_X)), A.sreg(bc.TID_X))
    a0, a1, a2 = A.sreg(bc.ARG0), A.sreg(bc.ARG1), A.sreg(bc.ARG2)

    def aff():
        c = rng.choice((1, 1, 2, -1, 3))
        v = lin if c == 1 else A.alu(bc.MUL, lin, Imm(c))
        return A.alu(bc.ADD, A.alu(bc.ADD, v, a0), Imm(rng.randint(-3, 3)))

    def guard():
        kind = rng.below(5)
        if kind == 0:
            return A.alu(bc.SETLT, aff(), a1)
        if kind == 1:
            return A.alu(bc.SETLE, a1, aff())
        if kind == 2:
            return A.alu(bc.SETEQ, lin, a2)
        if kind == 3:
            return A.alu(bc.SETNE, aff(), a2)
        return A.alu(bc.SUB, lin, a2)                            # "lin - a2 != 0"

    def body(depth):
        for _ in range(rng.randint(1, 3)):
            r = rng.below(4)
            if r == 0 or depth >= 2:
                A.ld(rng.below(3), aff(), rng.choice(bc.WIDTHS))
            elif r == 1:
                A.st(rng.below(3), aff(), A.imm(1), rng.choice(bc.WIDTHS))
            elif r == 2:
                A.if_(guard())
                body(depth + 1)
                if rng.below(2):
                    A.else_()
                    body(depth + 1)
                A.endif()
            else:
                k = A.loop(A.sreg(bc.ARG3), 4)
                A.if_(A.alu(bc.SETLT, A.alu(bc.ADD, lin, A.alu(bc.SHL, k, Imm(3))), a1))
                A.ld(rng.below(3), A.alu(bc.ADD, aff(), k), 4)
                A.endif()
                A.endloop()

    body(0)
    return A.build()


def test_plan_decides_random_guarded_1d(orc):
    rng = gen.SplitMix64(1048)
    planned = violating = 0
    for trial in range(60):
        prog = guarded_1d_program(rng)
        for _ in range(4):
            nx, gx = rng.randint(1, 40), rng.randint(1, 6)
            n = nx * gx
            args = (rng.randint(-4, 4), rng.randint(-5, n + 5), rng.randint(-2, n + 2),
                    rng.randint(0, 4))
            inp = mk((gx, 1, 1), (nx, 1, 1), args,
                     [rng.randint(0, 4 * (3 * n + 12)) for _ in range(3)])
            plan = B.cufz_prex_plan(prog, inp)
            assert plan is not None
            assert np.all(np.diff(plan.astype(np.int64)) > 0) and plan[0] == 0 and plan[-1] == n - 1
            ok, full = plan_decides_every_site(orc, prog, inp, plan)
            assert ok, (trial, args)
            planned += 1
            violating += full
    assert planned == 240 and 40 < violating < 220


def test_plan_decides_guarded_configs(orc):
    """The guarded 1D workloads (one program over grids of 64 x 128, sixteen
    programs of the family with offsets and widths over log-uniform
    launches): a plan for every input, a handful of threads each, and every
    site's verdict decided by it."""
    c1 = gen.c1_inputs(24, seed=77)
    c3 = gen.c3_inputs(48, seed=78, max_blocks=64, max_threads=256)
    progs = gen.c3_programs()
    for inp, prog in [(x, gen.c1_program()) for x in c1] + [(x, progs[int(x["program_id"])]) for x in c3]:
        assert not B.cufz_prex_check(prog, inp) or int(inp["args"][1]) <= 0
        plan = B.cufz_prex_plan(prog, inp)
        assert plan is not None and len(plan) <= 5
        ok, _ = plan_decides_every_site(orc, prog, inp, plan)
        assert ok


def test_plan_needs_the_threshold_threads(orc):
    """Why the guard's change point is planned: with i < 100 guarding A[i]
    and A 99 elements long, thread 99 alone violates; threads 0 and N - 1
    (the corners) see nothing."""
    prog = gen.c1_program()
    inp = mk((64, 1, 1), (128, 1, 1), (0, 100), (4 * 99, 4 * 8192, 4 * 8192, 4 * 8192))
    plan = B.cufz_prex_plan(prog, inp)
    assert 99 in plan.tolist()
    res, recs, _ = orc.run(orc.Program(prog), inp, rec_cap=64, bitmap=False)
    assert int(res["n_violations"]) == 1 and int(recs[0]["block_lin"]) * 128 + int(recs[0]["thread_lin"]) == 99
    ok, full = plan_decides_every_site(orc, prog, inp, np.array([0, 64 * 128 - 1]))
    assert full and not ok


def test_plan_is_the_corners_when_the_check_holds():
    rng = gen.SplitMix64(9)
    from test_oracle_pins import affine_program
    for dims in (1, 2, 3):
        prog = affine_program(rng, dims, 4)
        grid = [3, 2, 2][:dims] + [1] * (3 - dims)
        block = [5, 4, 3][:dims] + [1] * (3 - dims)
        inp = mk(grid, block, (1, 2, 0, 0), (400, 400, 400))
        assert B.cufz_prex_check(prog, inp)
        T = int(np.prod(block))
        want = sorted({B_ * T + t
                       for B_ in range(int(np.prod(grid))) if corner(B_, grid)
                       for t in range(T) if corner(t, block)})
        assert B.cufz_prex_plan(prog, inp).tolist() == want


def guarded_nd_program(rng, dims, piecewise=False):
    """Guards on one dimension's coordinate each (global G = ctaid * ntid +
    tid, tid alone or ctaid alone, scaled), compared with arguments by <,
    <=, ==, != or tested against zero, combined by AND / OR or nested, with
    else arms; accesses at indices affine in all coordinates, at guard
    values, and at selections between uniform values by a guard; a guard on
    a value loaded at such an index; a guard inside a uniform loop.  With
    `piecewise`, also indices that are affine only per cell: a clamped
    coordinate plus an affine term, a register the arms of a guard set to
    different affine values, a selection between affine values by a guard."""
    A = Asm(n_bufs=3, seed=rng.next32())
    t = [A.sreg(bc.TID_X + d) for d in range(dims)]
    b = [A.sreg(bc.CTAID_X + d) for d in range(dims)]
    G = [A.alu(bc.ADD, A.alu(bc.MUL, b[d], A.sreg(bc.NTID_X + d)), t[d]) for d in range(dims)]
    a0, a1, a2 = A.sreg(bc.ARG0), A.sreg(bc.ARG1), A.sreg(bc.ARG2)

    def coord():
        d, r = rng.below(dims), rng.below(4)
        return G[d] if r < 2 else t[d] if r == 2 else b[d]

    def aff():
        v = A.alu(bc.ADD, a0, Imm(rng.randint(-3, 3)))
        for _ in range(rng.randint(1, dims + 1)):
            c = rng.choice((1, 1, 2, -1, 3, 8))
            x = coord()
            v = A.alu(bc.ADD, v, x if c == 1 else A.alu(bc.MUL, x, Imm(c)))
        return v

    def guard(truth_value=True):
        x = coord()
        if rng.below(3) == 0:
            x = A.alu(bc.MUL, x, Imm(rng.choice((2, -1, 3))))
        kind = rng.below(5 if truth_value else 4)
        if kind == 0:
            return A.alu(bc.SETLT, x, a1)
        if kind == 1:
            return A.alu(bc.SETLE, a2, x)
        if kind == 2:
            return A.alu(bc.SETEQ, x, a2)
        if kind == 3:
            return A.alu(bc.SETNE, A.alu(bc.ADD, x, Imm(1)), a1)
        return A.alu(bc.SUB, x, a2)

    def cond():
        r = rng.below(4)
        if r == 0:   # comparisons only: AND of 0/1 values is the logical and
            return A.alu(bc.AND, guard(False), guard(False))
        if r == 1:
            return A.alu(bc.OR, guard(False), guard(False))
        return guard()

    def body(depth):
        for _ in range(rng.randint(1, 3)):
            r = rng.below(10 if piecewise else 7)
            if r <= 1 or depth >= 2:
                A.ld(rng.below(3), aff(), rng.choice(bc.WIDTHS))
            elif r == 2:
                A.st(rng.below(3), aff(), A.imm(1), rng.choice((1, 4)))
            elif r == 3:
                A.if_(cond())
                body(depth + 1)
                if rng.below(2):
                    A.else_()
                    body(depth + 1)
                A.endif()
            elif r == 4:
                sel = A.sel(guard(False), A.imm(rng.randint(-2, 40)), a0)
                v = A.ld(rng.below(3), sel, 4)
                A.if_(A.alu(bc.SETLT, A.alu(bc.AND, v, Imm(7)), Imm(3)))
                A.ld(rng.below(3), aff(), 4)
                A.endif()
            elif r == 5:
                A.ld(rng.below(3), guard(False), 8)
            elif r == 7:
                x = A.alu(bc.ADD, coord(), Imm(rng.randint(-3, 3)))
                cl = A.alu(bc.MAX, A.alu(bc.MIN, x, a1), a0)
                A.ld(rng.below(3), A.alu(bc.ADD, cl, aff()), rng.choice(bc.WIDTHS))
            elif r == 8:
                v = A.alu(bc.ADD, a0, Imm(0))
                A.if_(cond())
                A.mov(aff(), dst=v)
                if rng.below(2):
                    A.else_()
                    A.mov(aff(), dst=v)
                A.endif()
                A.ld(rng.below(3), v, 4)
            elif r == 9:
                A.ld(rng.below(3), A.sel(guard(False), aff(), aff()), 4)
            else:
                k = A.loop(A.sreg(bc.ARG3), 3)
                A.if_(A.alu(bc.SETLT, A.alu(bc.ADD, coord(), k), a1))
                A.ld(rng.below(3), A.alu(bc.ADD, aff(), k), 4)
                A.endif()
                A.endloop()

    body(0)
    return A.build()


def test_plan_decides_random_guarded_nd(orc):
    rng = gen.SplitMix64(0x2D3D)
    planned = violating = 0
    sizes = []
    for trial in range(72):
        dims = 1 + trial % 3
        prog = guarded_nd_program(rng, dims)
        for _ in range(3):
            block = [rng.randint(1, 8) for _ in range(dims)] + [1] * (3 - dims)
            grid = [rng.randint(1, 4) for _ in range(dims)] + [1] * (3 - dims)
            span = max(n * g for n, g in zip(block, grid))
            args = (rng.randint(-4, 4), rng.randint(-3, span + 3), rng.randint(-2, span + 2),
                    rng.randint(0, 3))
            lens = [rng.randint(0, 4 * (12 * span + 16)) for _ in range(3)]
            inp = mk(grid, block, args, lens)
            plan = B.cufz_prex_plan(prog, inp)
            assert plan is not None, (trial, args)
            ok, full = plan_decides_every_site(orc, prog, inp, plan)
            assert ok, (trial, args)
            planned += 1
            violating += full
            sizes.append(len(plan) / float(np.prod(block) * np.prod(grid)))
    assert planned == 216 and 30 < violating < 200
    assert np.median(sizes) < 0.6                   # the plan is a fraction of the grid


def test_plan_for_a_2d_bounds_guard_is_small(orc):
    """row = ctaid.y * ntid.y + tid.y, col likewise; if (row < n && col < m)
    C[row * m + col]: both dimensions stay merged, each contributes its ends
    and the two threads around its bound, 16 threads of 65,536."""
    A = Asm(n_bufs=1)
    row = A.alu(bc.ADD, A.alu(bc.MUL, A.sreg(bc.CTAID_Y), A.sreg(bc.NTID_Y)), A.sreg(bc.TID_Y))
    col = A.alu(bc.ADD, A.alu(bc.MUL, A.sreg(bc.CTAID_X), A.sreg(bc.NTID_X)), A.sreg(bc.TID_X))
    m = A.sreg(bc.ARG1)
    A.if_(A.alu(bc.AND, A.alu(bc.SETLT, row, A.sreg(bc.ARG0)), A.alu(bc.SETLT, col, m)))
    A.st(0, A.alu(bc.ADD, A.alu(bc.MUL, row, m), col), A.imm(1), 4)
    A.endif()
    prog = A.build()
    for lens in (4 * 200 * 150, 4 * 200 * 150 - 4):          # exact, one element short
        inp = mk((16, 16, 1), (16, 16, 1), (200, 150), (lens,))
        plan = B.cufz_prex_plan(prog, inp)
        assert len(plan) == 16
        ok, full = plan_decides_every_site(orc, prog, inp, plan)
        assert ok and full == (lens < 4 * 200 * 150)


def test_plan_accepts_and_refuses(orc):
    tx, ty = (lambda A: A.sreg(bc.TID_X)), (lambda A: A.sreg(bc.TID_Y))
    lin = lambda A: A.alu(bc.ADD, A.alu(bc.MUL, A.sreg(bc.CTAID_X), A.sreg(bc.NTID_X)), tx(A))
    lt = lambda A, x, y: A.alu(bc.SETLT, x, y)

    def guarded_by(cond):
        return _prog(lambda A: (A.if_(cond(A)), A.ld(0, lin(A), 4), A.endif()))

    def diverged(A):
        r = A.imm(0)
        A.if_(lt(A, lin(A), A.sreg(bc.ARG0)))
        A.mov(lin(A), dst=r)
        A.endif()
        A.ld(0, r, 4)

    def looped(A):
        k = A.loop(A.sreg(bc.ARG1), 200)
        A.if_(lt(A, A.alu(bc.ADD, lin(A), k), A.sreg(bc.ARG0)))
        A.ld(0, lin(A), 4)
        A.endif()
        A.endloop()

    one_d = mk((4, 1, 1), (32, 1, 1), (50, 100), (400, 400))
    two_d = mk((4, 1, 1), (8, 4, 1), (5, 100), (400, 400))
    clamp = lambda A, x: A.alu(bc.MAX, A.alu(bc.MIN, x, A.alu(bc.SUB, A.sreg(bc.ARG1), Imm(1))),
                               Imm(0))
    accepted = {
        "arms leaving different indices": (_prog(diverged), one_d),
        "a clamped index": (_prog(lambda A: A.ld(0, clamp(A, A.alu(bc.SUB, lin(A), Imm(2))), 4)),
                            mk((4, 1, 1), (32, 1, 1), (50, 90), (400, 400))),
        "a selection between indices by a guard":
            (_prog(lambda A: A.ld(0, A.sel(lt(A, tx(A), A.sreg(bc.ARG0)), lin(A),
                                           A.alu(bc.MUL, lin(A), Imm(2))), 4)),
             mk((4, 1, 1), (32, 1, 1), (7, 0), (400, 400))),
        "guard on the global index": (guarded_by(lambda A: lt(A, lin(A), A.sreg(bc.ARG0))), one_d),
        "guard on tid.x over four blocks": (guarded_by(lambda A: lt(A, tx(A), A.sreg(bc.ARG0))), one_d),
        "guard in a 2D block": (guarded_by(lambda A: lt(A, ty(A), Imm(2))), two_d),
        "two guards and-ed": (guarded_by(lambda A: A.alu(bc.AND, lt(A, lin(A), A.sreg(bc.ARG0)),
                                                         lt(A, A.sreg(bc.ARG1), lin(A)))), one_d),
    }
    for name, (prog, inp) in accepted.items():
        plan = B.cufz_prex_plan(prog, inp)
        assert plan is not None, name
        assert plan_decides_every_site(orc, prog, inp, plan)[0], name
    refused = {
        "a guard across two dimensions": (guarded_by(lambda A: lt(A, A.alu(bc.ADD, tx(A), ty(A)),
                                                                  Imm(5))), two_d),
        "a clamp across two dimensions": (_prog(lambda A: A.ld(0, A.alu(bc.MIN, tx(A), ty(A)), 4)),
                                          two_d),
        "a masked index": (_prog(lambda A: A.ld(0, A.alu(bc.AND, lin(A), Imm(7)), 4)), one_d),
        "tid.x and ctaid.x in another mix than the global index":
            (guarded_by(lambda A: lt(A, A.alu(bc.ADD, A.alu(bc.SHL, tx(A), Imm(1)),
                                              A.sreg(bc.CTAID_X)), A.sreg(bc.ARG0))), one_d),
        "a guard and-ed bitwise with a non-guard":
            (guarded_by(lambda A: A.alu(bc.AND, lt(A, lin(A), A.sreg(bc.ARG0)),
                                        A.alu(bc.SUB, lin(A), A.sreg(bc.ARG1)))), one_d),
        "a loaded index": (_prog(lambda A: (A.if_(lt(A, lin(A), A.sreg(bc.ARG0))),
                                            A.ld(1, A.ld(0, lin(A), 4), 4), A.endif())), one_d),
        "an index plus a guard": (_prog(lambda A: A.ld(0, A.alu(bc.ADD, lin(A),
                                                                lt(A, lin(A), A.sreg(bc.ARG0))),
                                                      4)), one_d),
        "a thread-dependent trip": (_prog(lambda A: (A.loop(tx(A), 8), A.ld(0, A.imm(0), 4),
                                                     A.endloop())), one_d),
    }
    for name, (prog, inp) in refused.items():
        assert B.cufz_prex_plan(prog, inp) is None, name
    budget = _prog(looped)
    assert B.cufz_prex_plan(budget, one_d, iter_budget=4096) is not None
    assert B.cufz_prex_plan(budget, one_d, iter_budget=50) is None     # a budget stop


def test_no_plan_for_launches_the_engine_does_not_run():
    """Invalid shapes complete as INVALID_CONFIG and launches above 2^31
    threads as LIMIT without running, so neither has a plan."""
    prog = gen.c1_program()
    for grid, block in (((0, 1, 1), (32, 1, 1)), ((4, 1, 1), (0, 1, 1)), ((1, 1, 1), (2048, 1, 1)),
                        ((1, 70000, 1), (1, 1, 1)), ((2**31 - 1, 1, 1), (1024, 1, 1)),
                        ((72093556, 65352, 65000), (1024, 1, 1))):  # thread count wraps 2^64
        inp = mk(grid, block, (0, 100), (400, 400, 400, 400))
        assert B.cufz_prex_plan(prog, inp) is None, (grid, block)
        assert not B.cufz_prex_check(prog, inp), (grid, block)
    assert B.cufz_prex_plan(prog, mk((2**21, 1, 1), (1024, 1, 1), (0, 100), (400,) * 4)) is not None


def test_plan_decides_guard2d_workload(orc):
    """The bounds-guarded 2D workload (if (row < n && col < m) over the
    matrix): at most 16 planned threads per input, every site decided."""
    progs = gen.guard2d_programs()
    ins = gen.guard2d_inputs(32, seed=9, max_grid=6)
    violating = 0
    for x in ins:
        prog = progs[int(x["program_id"])]
        plan = B.cufz_prex_plan(prog, x)
        assert plan is not None and len(plan) <= 16
        ok, full = plan_decides_every_site(orc, prog, x, plan)
        assert ok
        violating += full
    assert 0 < violating < len(ins)


def test_plan_decides_random_piecewise_indices(orc):
    """Indices that are affine only per cell (clamps, diverging arms,
    selections by guards) within the random guarded programs."""
    rng = gen.SplitMix64(0x9A7C)
    planned = violating = 0
    for trial in range(72):
        dims = 1 + trial % 3
        prog = guarded_nd_program(rng, dims, piecewise=True)
        for _ in range(3):
            block = [rng.randint(1, 8) for _ in range(dims)] + [1] * (3 - dims)
            grid = [rng.randint(1, 4) for _ in range(dims)] + [1] * (3 - dims)
            span = max(n * g for n, g in zip(block, grid))
            args = (rng.randint(-4, 4), rng.randint(-3, span + 3), rng.randint(-2, span + 2),
                    rng.randint(0, 3))
            inp = mk(grid, block, args, [rng.randint(0, 4 * (12 * span + 16)) for _ in range(3)])
            plan = B.cufz_prex_plan(prog, inp)
            if plan is None:
                continue
            ok, full = plan_decides_every_site(orc, prog, inp, plan)
            assert ok, (trial, args)
            planned += 1
            violating += full
    assert planned > 150 and 30 < violating < planned


def test_head_tail_heuristic_misses_what_the_plan_finds(orc):
    """Why the plan replaces the paper's Alg. 1.  j = (a0 <= i < a1) ? i +
    4096 : i; load A[j].  The load runs in every thread, so the first and
    last blocks cover every access instruction, and neither violates: Alg. 1
    stops there and reports no bug.  The middle threads read past A.  The
    plan cuts the launch at a0 and a1 and finds them."""
    A = Asm(n_bufs=1)
    i = A.alu(bc.ADD, A.alu(bc.MUL, A.sreg(bc.CTAID_X), A.sreg(bc.NTID_X)), A.sreg(bc.TID_X))
    mid = A.alu(bc.AND, A.alu(bc.SETLE, A.sreg(bc.ARG0), i), A.alu(bc.SETLT, i, A.sreg(bc.ARG1)))
    A.ld(0, A.sel(mid, A.alu(bc.ADD, i, Imm(4096)), i), 4)
    prog = A.build()
    inp = mk((16, 1, 1), (64, 1, 1), (300, 700), (4 * 1024,))
    res, recs, _ = orc.run(orc.Program(prog), inp, rec_cap=1 << 12, bitmap=False)
    blocks = set(recs["block_lin"].tolist())
    assert int(res["n_violations"]) == 400 and 0 not in blocks and 15 not in blocks
    plan = B.cufz_prex_plan(prog, inp)
    assert plan is not None and len(plan) <= 8
    ok, full = plan_decides_every_site(orc, prog, inp, plan)
    assert ok and full


def test_no_plan_for_programs_that_divide():
    """A division is a check of its own that neither analysis models: an
    otherwise affine program with a division gets no plan."""
    A = Asm(n_bufs=1)
    i = A.alu(bc.ADD, A.alu(bc.MUL, A.sreg(bc.CTAID_X), A.sreg(bc.NTID_X)), A.sreg(bc.TID_X))
    A.div(A.sreg(bc.ARG0), A.alu(bc.SUB, i, A.sreg(bc.ARG1)))
    A.ld(0, i, 4)
    inp = mk((4, 1, 1), (32, 1, 1), (1, 7), (400,))
    assert not B.cufz_prex_check(A.build(), inp) and B.cufz_prex_plan(A.build(), inp) is None


@pytest.mark.parametrize("op", ["halloc", "hfree", "hld", "hst"])
def test_no_plan_for_programs_on_the_heap(op):
    """Heap operations keep per-thread state (blocks live or freed) that
    neither analysis models: an otherwise affine program with any heap
    operation gets no plan."""
    A = Asm(n_bufs=1)
    i = A.alu(bc.ADD, A.alu(bc.MUL, A.sreg(bc.CTAID_X), A.sreg(bc.NTID_X)), A.sreg(bc.TID_X))
    if op == "halloc":
        A.halloc(A.sreg(bc.ARG0))
    elif op == "hfree":
        A.hfree(A.sreg(bc.ARG0))
    elif op == "hld":
        A.hld(A.sreg(bc.ARG0), i, 4)
    else:
        A.hst(A.sreg(bc.ARG0), i, i, 4)
    A.ld(0, i, 4)
    inp = mk((4, 1, 1), (32, 1, 1), (1, 7), (400,))
    assert not B.cufz_prex_check(A.build(), inp) and B.cufz_prex_plan(A.build(), inp) is None


def _tile_program():
    """A tiled copy with a barrier (the shape of Sec. 5.2's example): each
    thread stores A[i] into its tile slot, and after the barrier copies the
    mirrored slot to C[i]; under the guard i < a1 it also reads A[i + 1]."""
    A = Asm(n_bufs=3, shared_mask=0b100, shared_stores=True)
    t, T = A.sreg(bc.TID_X), A.sreg(bc.NTID_X)
    i = A.alu(bc.ADD, A.alu(bc.MUL, A.sreg(bc.CTAID_X), T), t)
    A.st(2, t, A.ld(0, i, 4), 4)
    A.bar()
    A.st(1, i, A.ld(2, A.alu(bc.SUB, A.alu(bc.SUB, T, Imm(1)), t), 4), 4)
    A.if_(A.alu(bc.SETLT, i, A.sreg(bc.ARG1)))
    A.ld(0, A.alu(bc.ADD, i, Imm(1)), 4)
    A.endif()
    return A.build()


def test_plans_for_eliminated_barriers_decide_the_phased_grid(orc):
    """Programs whose barriers BarrierElimination removes keep PREX: where a
    plan exists, its threads decide every access site's verdict under the
    oracle's phase-by-phase execution with performed stores."""
    prog = _tile_program()
    rng = gen.SplitMix64(901)
    planned = violating = 0
    for _ in range(48):
        T, nb = rng.choice((32, 64, 128)), rng.randint(1, 6)
        n = T * nb
        inp = mk((nb, 1, 1), (T, 1, 1), (0, n - rng.randint(0, 2)),
                 (4 * (n - rng.randint(0, 1)), 4 * (n - rng.randint(0, 1)),
                  4 * (T - rng.randint(0, 1))))
        plan = B.cufz_prex_plan(prog, inp)
        assert plan is not None and len(plan) < n
        planned += 1
        ok, full = plan_decides_every_site(orc, prog, inp, plan)
        assert ok, inp
        violating += full
    for which in range(16):          # the random ones, where a plan exists
        p = gen.barrier_program(which)
        for inp in gen.barrier_inputs(8, n_programs=1, seed=900 + which, max_blocks=4):
            plan = B.cufz_prex_plan(p, inp)
            if plan is not None:
                assert plan_decides_every_site(orc, p, inp, plan)[0], (which, inp)
    assert planned == 48 and 8 <= violating < 48
