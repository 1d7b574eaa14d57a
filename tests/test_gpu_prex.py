"""PREX on the GPU (Sec. 5.1): with CUFZ_CF_PREX, an input with a plan
(cufz_prex_plan: the corner threads of an unguarded affine program, or the
corners of the cells the guards cut a guarded launch into) runs only the
planned threads.
Its verdict (violation or not) is the full grid's, the oracle's, and its
records are exactly the full run's records of the planned threads.  Inputs
without a plan run the full grid, bit-exact with the oracle."""
import numpy as np
import pytest

from paper_2601_01048_gb300 import bytecode as bc
from paper_2601_01048_gb300 import gen
from paper_2601_01048_gb300.bytecode import Asm

pytestmark = pytest.mark.gpu

KEYS = ("block_lin", "thread_lin", "ordinal", "site", "buf", "kind", "width", "space", "cls",
        "byte_off")


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_01048_gb300 import binding
    binding.lib()
    return binding


def bounds_guard_2d_program():
    """row = ctaid.y * ntid.y + tid.y, col likewise; if (row < arg0 && col <
    arg1) C[row * arg1 + col] = 1."""
    A = Asm(n_bufs=1, seed=0x2D)
    row = A.alu(bc.ADD, A.alu(bc.MUL, A.sreg(bc.CTAID_Y), A.sreg(bc.NTID_Y)), A.sreg(bc.TID_Y))
    col = A.alu(bc.ADD, A.alu(bc.MUL, A.sreg(bc.CTAID_X), A.sreg(bc.NTID_X)), A.sreg(bc.TID_X))
    m = A.sreg(bc.ARG1)
    A.if_(A.alu(bc.AND, A.alu(bc.SETLT, row, A.sreg(bc.ARG0)), A.alu(bc.SETLT, col, m)))
    A.st(0, A.alu(bc.ADD, A.alu(bc.MUL, row, m), col), A.imm(1), 4)
    A.endif()
    return A.build()


def bounds_guard_2d_inputs(n, seed):
    rng = gen.SplitMix64(seed)
    x = gen.make_inputs(n)
    for k in range(n):
        block = (rng.choice((8, 16, 32)), rng.choice((4, 8, 16)), 1)
        grid = (rng.randint(1, 12), rng.randint(1, 12), 1)
        rows, cols = rng.randint(1, grid[1] * block[1]), rng.randint(1, grid[0] * block[0])
        short = rng.below(3) == 0
        gen.set_input(x[k], 0, grid, block, (rows, cols), (4 * (rows * cols - short),), tag=k)
    return x


def planned_records(orecs, o, plan, T):
    """The oracle's full-run records of the planned threads, as key tuples."""
    r = orecs[: int(o["n_records"])]
    keep = np.isin(r["block_lin"].astype(np.int64) * T + r["thread_lin"], plan)
    return set(zip(*(r[f][keep].tolist() for f in KEYS)))


@pytest.mark.parametrize("path", [0, 64])
def test_prex_verdicts(B, orc, path):
    progs = (gen.affine_programs()[:6] + [gen.c1_program()] + gen.c2_programs()[:1]
             + gen.c3_programs() + [bounds_guard_2d_program()])
    aff = gen.affine_inputs(36, seed=61, max_blocks=24, max_threads=96)
    aff["program_id"] %= 6
    c1 = gen.c1_inputs(8, seed=62)
    c1["program_id"] = 6
    c2 = gen.c2_inputs(progs[7:8], per_program=4, seed=63, max_grid=2)
    c2["program_id"] = 7
    c3 = gen.c3_inputs(16, seed=64, max_blocks=64, max_threads=256)
    c3["program_id"] += 8
    b2 = bounds_guard_2d_inputs(12, seed=65)
    b2["program_id"] = 24
    ins = np.concatenate([aff, c1, c2, c3, b2])
    progs_of = [progs[int(x["program_id"])] for x in ins]
    corner = [B.cufz_prex_check(p, x) for p, x in zip(progs_of, ins)]
    plans = [B.cufz_prex_plan(p, x) for p, x in zip(progs_of, ins)]
    n_aff, n_c1, n_c2 = len(aff), len(c1), len(c2)
    assert all(corner[:n_aff]) and not any(corner[n_aff:])
    guarded = list(range(n_aff, n_aff + n_c1)) + list(range(n_aff + n_c1 + n_c2, len(ins)))
    assert all(plans[k] is not None for k in guarded)          # guarded launches: cell plans
    # random programs: masked, clamped and loaded indices
    assert all(plans[k] is None for k in range(n_aff + n_c1, n_aff + n_c1 + n_c2))
    with B.Engine(max_slots=128, record_cap=1 << 15, flags=B.CF_KEEP_BITMAPS | B.CF_PREX | path) as E:
        for p in progs:
            E.load(p)
        dres, drecs, dbms = E.run(ins)
    ores, orecs, obms = orc.run_batch(progs, ins, rec_cap=1 << 15, bitmaps=True)
    assert np.array_equal(ores["n_records"], ores["n_violations"])   # every record kept
    n_viol = [0, 0]
    for k in range(len(ins)):
        d, o = dres[k], ores[k]
        assert int(d["status"]) == int(o["status"]), k
        if plans[k] is not None and len(plans[k]) <= B.PREX_MAX_PLAN:
            assert int(d["flags"]) & B.FL_PARTIAL
            assert int(d["n_threads"]) == len(plans[k])
            if corner[k]:
                assert len(plans[k]) == n_corners(ins[k])
            T = int(np.prod([int(v) for v in ins[k]["block"]]))
            want = planned_records(orecs[k], o, plans[k], T)
            got = set(zip(*(drecs[k][f].tolist() for f in KEYS)))
            assert got == want, k
            assert int(d["n_violations"]) == len(want), k
            n_viol[0 if corner[k] else 1] += int(o["status"]) == B.ST_VIOLATION
        else:
            assert not int(d["flags"]) & B.FL_PARTIAL
            for f in ("n_accesses", "n_violations", "first_key", "digest", "n_branch", "n_edges"):
                assert int(d[f]) == int(o[f]), (k, f)
            assert np.array_equal(dbms[k], obms[k])
    assert 0 < n_viol[0] < n_aff and 0 < n_viol[1] < len(guarded)


def n_corners(inp):
    g = [int(v) for v in inp["grid"]] + [int(v) for v in inp["block"]]
    return int(np.prod([2 if v > 1 else 1 for v in g]))
