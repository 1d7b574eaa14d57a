"""The allocation-free entry point (cufz_run_noalloc) gives the same results
as a context does for the same inputs, and the oracle's.

It exists for callers that cannot allocate device memory: plugins whose
host framework owns every device allocation and hands out only the buffers
of one call, and services that must keep a fixed device footprint after
start-up.  Its scratch is a fixed array inside the library, shared by every
call, so two calls in a row must not see each other's leftovers.  This file
is collected last on purpose (tests/conftest.py orders it after every other
test), so a run that stops at its first failure has run everything else."""
import numpy as np
import pytest
from conftest import record_keys

pytestmark = pytest.mark.gpu

FIELDS = ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch",
          "n_threads", "n_records", "n_edges")
ORACLE_FIELDS = ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch",
                 "n_edges")


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


class NoAlloc:
    """Caller-owned output buffers and one call of the entry point."""

    def __init__(self, torch, cap):
        from paper_2601_01048_gb300 import binding as B

        self.B, self.torch, self.cap = B, torch, cap
        self.dev = torch.device("cuda", 0)
        self.stream = torch.cuda.current_stream(self.dev).cuda_stream
        self.records = torch.empty(max(cap, 1) * 32, dtype=torch.uint8, device=self.dev)
        self.bitmap = torch.empty(65536, dtype=torch.uint8, device=self.dev)
        self.result = torch.empty(96, dtype=torch.uint8, device=self.dev)

    def __call__(self, prog, inp, flags=0):
        B = self.B
        # poison every output, so that stale or unwritten bytes show
        self.records.fill_(0xAB)
        self.bitmap.fill_(0xCD)
        self.result.fill_(0xEF)
        self.torch.cuda.synchronize(self.dev)
        B.cufz_run_noalloc(prog, inp, self.records.data_ptr(), self.cap, self.bitmap.data_ptr(),
                           self.result.data_ptr(), flags=flags, stream=self.stream)
        res = np.frombuffer(self.result.cpu().numpy().tobytes(), dtype=B.RESULT_DTYPE)[0]
        n = int(res["n_records"])
        recs = np.frombuffer(self.records.cpu().numpy().tobytes(), dtype=B.VIOLATION_DTYPE)[:n]
        return res, recs, self.bitmap.cpu().numpy()


def _oracle_check(orc, prog, inp, res, recs, bm, flags_expected):
    ores, orecs, obm = orc.run(prog, inp, rec_cap=1 << 20)
    for f in ORACLE_FIELDS:
        assert int(res[f]) == int(ores[f]), f
    assert int(res["flags"]) == flags_expected
    assert np.array_equal(bm, obm)
    full = record_keys(orecs[:int(ores["n_violations"])])
    if int(ores["n_violations"]) <= len(recs):
        assert record_keys(recs) == full
    else:                                    # any cap of the violations, each a real one
        assert set(record_keys(recs)) <= set(full)


def test_noalloc_matches_context_on_two_calls_in_a_row(orc):
    torch = _cuda()
    from paper_2601_01048_gb300 import binding as B
    from paper_2601_01048_gb300 import gen

    progs = [gen.c1_program(), gen.c2_program(5)]
    a = gen.c1_inputs(40, seed=123)
    a = a[np.argmax(a["args"][:, 0] < 0)]                      # an input with violations
    b = gen.c2_inputs([progs[1]], per_program=1, seed=77, max_grid=1)[0]
    b["program_id"] = 1
    inputs = np.array([a, b], dtype=gen.INPUT_DTYPE)
    cap = 1 << 14

    with B.Engine(record_cap=cap, max_slots=8) as E:              # the existing entry points
        for p in progs:
            E.load(p)
        ref, ref_recs, ref_bms = E.run(inputs)

    call = NoAlloc(torch, cap)
    for k in (0, 1, 0):                                           # calls in a row
        res, recs, bm = call(progs[int(inputs[k]["program_id"])], inputs[k])
        for f in FIELDS:
            assert int(res[f]) == int(ref[k][f]), (k, f)
        assert int(res["flags"]) == int(ref[k]["flags"]), k
        assert int(res["user_tag"]) == int(ref[k]["user_tag"])
        assert int(ref[k]["n_violations"]) <= cap          # record sets are unique then
        assert record_keys(recs) == record_keys(ref_recs[k])
        assert np.array_equal(bm, ref_bms[k])
        # NEW_COV is against an empty union, as for a context's first epoch
        _oracle_check(orc, progs[int(inputs[k]["program_id"])], inputs[k], res, recs, bm,
                      int(ref[k]["flags"]))
    assert int(ref[0]["n_violations"]) > 0 and int(ref[1]["n_edges"]) > 0


def test_noalloc_rejected_launches_overflow_and_largest_program(orc):
    """The paths beside the launched one: launch shapes that complete without
    running (INVALID_CONFIG, LIMIT with a thread count that wraps 64 bits),
    a record cap far below the violations (OVERFLOW, n_records clamped,
    counts exact), and the largest valid program (2,048 ops, unpruned),
    whose loaded form stays under the entry point's 64 KiB program limit.
    Each result is compared with a context's and with the oracle's."""
    torch = _cuda()
    from paper_2601_01048_gb300 import binding as B
    from paper_2601_01048_gb300 import bytecode as bc
    from paper_2601_01048_gb300 import gen

    c1 = gen.c1_program()
    A = bc.Asm(n_bufs=2, seed=0x5EED)
    x = A.sreg(bc.TID_X)
    a0 = A.sreg(bc.ARG0)
    t, v = A.new_reg(), A.new_reg()
    while len(A.ops) < bc.MAX_OPS - 2:
        A.alu(bc.ADD, x, bc.Imm(1), dst=x)
        if len(A.ops) % 7 == 0:
            A.ld(len(A.ops) % 2, A.alu(bc.SUB, x, a0, dst=t), 4, dst=v)
    big = A.build()
    assert len(A.ops) <= bc.MAX_OPS

    ins = gen.make_inputs(5)
    gen.set_input(ins[0], 0, (0, 1, 1), (32, 1, 1), (0, 1), (4, 4, 4, 4))          # INVALID_CONFIG
    gen.set_input(ins[1], 0, (72093556, 65352, 65000), (1024, 1, 1), (0, 1), (4, 4, 4, 4))
    gen.set_input(ins[2], 0, (64, 1, 1), (128, 1, 1), (-4, 8192), (0, 0, 0, 0))    # every access
    gen.set_input(ins[3], 1, (3, 1, 1), (64, 1, 1), (100, 0), (4000, 4000))
    gen.set_input(ins[4], 1, (2, 1, 1), (32, 1, 1), (-3, 0), (16, 9000))
    progs = {0: c1, 1: big}
    cap = 16

    with B.Engine(record_cap=cap, max_slots=8, flags=B.CF_KEEP_BITMAPS | B.CF_NO_PRUNE) as E:
        E.load(c1)
        E.load(big)
        ref, ref_recs, ref_bms = E.run(ins)

    call = NoAlloc(torch, cap)
    for k in range(len(ins)):
        prog = progs[int(ins[k]["program_id"])]
        res, recs, bm = call(prog, ins[k], flags=B.CF_NO_PRUNE)
        for f in FIELDS:
            assert int(res[f]) == int(ref[k][f]), (k, f)
        assert int(res["flags"]) == int(ref[k]["flags"]), k
        assert np.array_equal(bm, ref_bms[k]), k
        _oracle_check(orc, prog, ins[k], res, recs, bm, int(ref[k]["flags"]))
    assert int(ref[0]["status"]) == B.ST_INVALID_CONFIG
    assert int(ref[1]["status"]) == B.ST_LIMIT
    for k in (2, 3, 4):
        assert int(ref[k]["n_violations"]) > cap
        assert int(ref[k]["flags"]) & B.FL_OVERFLOW and int(ref[k]["n_records"]) == cap
