"""PREX (Sec. 5.1): the engine's eligibility check, pinned to the oracle.

For every input the check accepts, the oracle's full-grid verdict (some
thread violates or none does) must equal the verdict of the corner threads
alone (every block and thread coordinate first or last), which is what the
GPU runs under CUFZ_CF_PREX.  Inputs it must refuse: thread-dependent
branches or loop trips, indices that are not affine in the thread and block
indices, affine values that could wrap int32 in the launch box."""
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
