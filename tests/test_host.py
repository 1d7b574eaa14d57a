"""Host-side tests of the engine library (no GPU): exported symbols, the
validator, the prune pass (checked by running the CPU oracle on pruned and
unpruned programs) and the division magic numbers."""
import re

import numpy as np
import pytest

from conftest import ROOT, checks_of
from paper_2601_01048_gb300 import binding as B
from paper_2601_01048_gb300 import bytecode as bc
from paper_2601_01048_gb300 import gen
from paper_2601_01048_gb300.bytecode import Asm, Imm


def header_functions():
    src = open(f"{ROOT}/include/cufz.h").read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"\b(cufz_[a-z0-9_]+)\s*\(", src))


def test_library_exports_every_declared_function():
    names = header_functions()
    assert len(names) >= 19
    L = B.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(B.EXPORTS) == names


def test_status_strings():
    for st in range(0, -11, -1):
        assert B.cufz_status_str(st) and B.cufz_status_str(st) != b"unknown status"


def test_header_constants_match_binding():
    """Every CUFZ_E_/ST_/FL_/CF_/PREX_ constant of the header has the same value in
    the binding (they are written twice: C for the ABI, Python for ctypes)."""
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "cufz.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in
            re.finditer(r"#define CUFZ_((?:E|ST|FL|CF|PREX)_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", hdr)}
    assert len(defs) >= 25
    for name, value in defs.items():
        assert getattr(B, name) == value, name


def test_traffic_key_ignores_comments_only():
    """The bench's DRAM-traffic figure is keyed by the kernel code without
    comments: comments and blank lines do not change the key, code does."""
    import bench
    code = 'int f(int x) {  // twice\n  /* c */ return 2 * x;\n}\nconst char* s = "// kept";\n'
    same = 'int f(int x) {\n\n  return 2 * x;  // doubled\n}\nconst char* s = "// kept";\n'
    assert bench._code_only(code) == bench._code_only(same)
    assert bench._code_only(code) != bench._code_only(code.replace("2 * x", "3 * x"))
    assert '"// kept"' in bench._code_only(code)


def all_programs():
    progs = [gen.c1_program(), gen.vecadd_shared_program(64), gen.guarded_plus1_program(128)]
    progs += gen.c3_programs() + gen.c2_programs() + gen.c4_programs()
    return progs


def small_inputs(prog, n, seed):
    h = bc.decode_header(prog)
    rng = gen.SplitMix64(seed)
    out = gen.make_inputs(n)
    for k in range(n):
        grid = (rng.randint(1, 3), rng.randint(1, 2), 1)
        block = (rng.randint(1, 40), rng.randint(1, 3), 1)
        args = [rng.choice((0, -1, 1, 7, 33, 200, -5, 1 << 20)) for _ in range(4)]
        lens = [rng.choice((0, 4, 60, 256, 1024, 4096, 1 << 16)) for _ in range(h["n_bufs"])]
        gen.set_input(out[k], 0, grid, block, args, lens)
    return out


@pytest.mark.parametrize("which", range(67))
def test_prune_keeps_every_access_and_branch(orc, which):
    """Sec. 5.2: AXIPrune may change values but preserves every memory access.
    The oracle on the pruned program must give the same records (site,
    ordinal, byte offset), digest, counts and bitmap as on the original."""
    prog = all_programs()[which]
    pruned, st = B.cufz_prune_program(prog)
    assert orc.validate(pruned) == 0
    assert B.cufz_validate_program(pruned) == 0
    ops0, ops1 = bc.ops_of(prog), bc.ops_of(pruned)
    kinds = (bc.LD, bc.ST, bc.IF, bc.ELSE, bc.ENDIF, bc.LOOP, bc.ENDLOOP)
    assert [o[0] for o in ops0 if o[0] in kinds] == [o[0] for o in ops1 if o[0] in kinds]
    assert st.n_ops_kept <= st.n_ops_in and st.n_regs_alloc <= max(st.n_regs_in, 1)
    ins = small_inputs(prog, 4, 77 + which)
    for o in (orc.opts(), orc.opts(iter_budget=5)):
        r0, c0, b0 = orc.run_batch([prog], ins, o, rec_cap=1 << 15, bitmaps=True, threads=2)
        r1, c1, b1 = orc.run_batch([pruned], ins, o, rec_cap=1 << 15, bitmaps=True, threads=2)
        assert checks_of(r0) == checks_of(r1)
        assert (r1["n_ops"] <= r0["n_ops"]).all()           # pruning only removes ops
        assert c0.tobytes() == c1.tobytes()
        assert np.array_equal(b0, b1)


def test_prune_removes_dead_math():
    pruned, st = B.cufz_prune_program(gen.c1_program())
    assert st.n_ops_kept == st.n_ops_in - 1          # the stored sum x + y
    assert st.n_loads_value_dead == 2                # both loads kept only as checks
    c2 = [B.cufz_prune_program(p)[1] for p in gen.c2_programs()]
    assert sum(s.n_ops_kept for s in c2) < 0.95 * sum(s.n_ops_in for s in c2)


def test_prune_keeps_values_that_steer_branches_and_indices():
    """Listing-in-Sec.-5.2 shape: an expensive value feeding a branch that
    guards an access stays; one only stored goes."""
    A = Asm(n_bufs=2)
    t = A.sreg(bc.TID_X)
    a = A.sreg(bc.ARG0)
    dead = A.alu(bc.MUL, A.alu(bc.MUL, t, t), a)       # only stored
    live = A.alu(bc.XOR, A.alu(bc.MUL, t, a), Imm(5))   # steers the branch
    A.if_(A.alu(bc.SETLT, live, Imm(100)))
    A.st(0, t, dead)
    A.endif()
    idx = A.alu(bc.ADD, A.ld(1, t), Imm(0))             # a loaded value used as index
    A.ld(0, idx)
    pruned, st = B.cufz_prune_program(A.build())
    assert st.n_ops_kept == st.n_ops_in - 2
    assert st.n_loads_value_dead == 1


@pytest.mark.parametrize("seed", range(40))
def test_validator_agrees_with_oracle(orc, seed):
    rng = gen.SplitMix64(seed)
    prog = bytearray(rng.choice(all_programs()))
    for _ in range(rng.randint(1, 3)):
        pos = rng.randint(0, len(prog) - 1)
        prog[pos] = rng.below(256)
    if rng.chance(0.2):
        prog = prog[: rng.randint(0, len(prog))]
    p = bytes(prog)
    assert (B.cufz_validate_program(p) == 0) == (orc.validate(p) == 0)


def test_division_magic_identity():
    """The device divides n < 2^32 by a launch dimension d with
    m = ceil(2^64 / d): floor(n/d) = (m_hi*n + (m_lo*n >> 32)) >> 32."""
    rng = gen.SplitMix64(5)
    ds = [1, 2, 3, 5, 7, 31, 32, 33, 100, 1023, 1024, 65535, 65536, (1 << 31) - 1, 1 << 31,
          (1 << 32) - 1] + [rng.randint(1, (1 << 32) - 1) for _ in range(200)]
    ns = [0, 1, 2, (1 << 32) - 1, (1 << 31), (1 << 31) - 1] + [rng.next32() for _ in range(300)]
    for d in ds:
        m = 0 if d <= 1 else ((1 << 64) - 1) // d + 1
        for n in ns + [d - 1, d, d + 1, 2 * d - 1, 2 * d]:
            n &= (1 << 32) - 1
            if m == 0:
                q = n
            else:
                t = (m & 0xFFFFFFFF) * n
                q = (((m >> 32) * n + (t >> 32)) >> 32)
            assert q == n // d, (n, d)


def test_arena_sizing():
    cfg = B.cufz_config_default()
    a = B.cufz_arena_bytes(cfg, 16)
    b = B.cufz_arena_bytes(cfg, 32)
    assert 0 < a < b
    cfg.record_cap = 1 << 15
    assert B.cufz_arena_bytes(cfg, 16) > a


def test_engine_needs_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(B.CufzError):
        B.Engine()


@pytest.mark.parametrize("which", ["listings", "c3", "c2", "c4", "div", "heap"])
def test_generated_code_compiles_for_sm103a(which):
    """The compiled path: every workload program's generated CUDA compiles
    for sm_103a with the runtime compiler (no device needed)."""
    progs = {"listings": [gen.c1_program(), gen.vecadd_shared_program(64),
                          gen.guarded_plus1_program(128)],
             "c3": gen.c3_programs(), "c2": gen.c2_programs()[:8],
             "c4": gen.c4_programs()[:3], "div": gen.div_programs()[:8],
             "heap": gen.heap_programs()}[which]
    st, log, nbytes = B.cufz_compile_check(progs)
    assert st == 0, log[-4000:]
    assert nbytes > 0


def test_generated_code_shape():
    src = B.cufz_program_cuda(gen.c1_program())
    assert "cufz_prog_0" in src and "jit_record" in src and "jit_cover" in src
    assert src.count("dh = access_step(") == 3         # three checked accesses
    assert "r11" not in src                            # the pruned sum x + y is gone
    full = B.cufz_program_cuda(gen.c1_program(), B.CF_NO_PRUNE)
    assert "r11 =" in full


def test_abi_rejects_missing_arguments():
    """Every entry point answers a missing context or output pointer with
    CUFZ_E_INVALID_ARG (checked before any device call), and the host-only
    calls report the size they need when the caller's buffer is too small."""
    import ctypes
    L = B.lib()
    u32, u64, sz = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_size_t()
    ref = ctypes.byref
    null_ctx = {
        "cufz_destroy": (), "cufz_unload_program": (0,), "cufz_new_epoch": (), "cufz_release": (1,),
        "cufz_sync": (0,), "cufz_reset_stats": (), "cufz_set_program_path": (0, 1),
        "cufz_compile_programs": (None, 0), "cufz_get_union": (None,),
        "cufz_get_bitmap": (1, None), "cufz_get_program_path": (0, ref(u32)),
        "cufz_load_program": (None, 0, ref(u32), None),
        "cufz_submit_inputs": (None, 0, ref(u32), ref(u64)),
        "cufz_poll_results": (None, 0, ref(u32), 0), "cufz_get_records": (1, None, 0, ref(u32)),
        "cufz_autotune": (None, 0, ref(u32)), "cufz_verify_prune": (0, None, 0, ref(u32)),
        "cufz_get_stats": (None,), "cufz_set_program_lanes": (0, 1),
        "cufz_get_program_lanes": (0, ref(u32)),
    }
    for name, args in null_ctx.items():
        assert getattr(L, name)(None, *args) == B.E_INVALID_ARG, name
    prog = gen.c1_program()
    inp = gen.c1_inputs(1)
    assert L.cufz_create(None, None) == B.E_INVALID_ARG
    assert L.cufz_validate_program(None, 0) == B.E_INVALID_PROGRAM
    assert L.cufz_prex_check(None, 0, None, 0, ref(u32)) == B.E_INVALID_ARG
    assert L.cufz_prex_plan(prog, len(prog), inp.ctypes.data, 0, None, 4, ref(u32)) == B.E_INVALID_ARG
    assert L.cufz_prex_plan(prog, len(prog), inp.ctypes.data, 0, None, 0, ref(u32)) == B.E_NOMEM
    assert u32.value == 4                                     # the plan's size
    assert L.cufz_run_noalloc(None, 0, None, 0, 0, 0, None, 0, None, None, None) == B.E_INVALID_ARG
    assert L.cufz_int32_peak(0, None, None) == B.E_INVALID_ARG
    assert L.cufz_program_cuda(prog, len(prog), 0, None, 0, ref(sz)) == B.E_NOMEM and sz.value > 100
    stats = B.cufz_prog_stats()
    assert L.cufz_prune_program(prog, len(prog), None, 0, ref(sz), ref(stats)) == B.E_NOMEM
    assert sz.value == len(B.cufz_prune_program(prog)[0])


@pytest.mark.parametrize("which", range(16))
def test_prune_keeps_every_division(orc, which):
    """Divisions are checks: pruning keeps every DIV/REM (and the values that
    decide their faults), so the oracle gives the same fault and access
    records, ordinals, digest, counts and bitmap on the pruned program."""
    prog = gen.div_program(which)
    pruned, st = B.cufz_prune_program(prog)
    assert orc.validate(pruned) == 0 and B.cufz_validate_program(pruned) == 0
    kinds = (bc.LD, bc.ST, bc.IF, bc.ELSE, bc.ENDIF, bc.LOOP, bc.ENDLOOP, bc.DIV, bc.REM)
    assert [o[0] for o in bc.ops_of(prog) if o[0] in kinds] == \
        [o[0] for o in bc.ops_of(pruned) if o[0] in kinds]
    ins = gen.div_inputs(4, n_programs=1, seed=400 + which)
    for o in (orc.opts(), orc.opts(iter_budget=2)):
        r0, c0, b0 = orc.run_batch([prog], ins, o, rec_cap=1 << 14, bitmaps=True, threads=2)
        r1, c1, b1 = orc.run_batch([pruned], ins, o, rec_cap=1 << 14, bitmaps=True, threads=2)
        assert checks_of(r0) == checks_of(r1) and c0.tobytes() == c1.tobytes()
        assert np.array_equal(b0, b1)


@pytest.mark.parametrize("which", range(16))
def test_prune_keeps_every_heap_op(orc, which):
    """Heap operations are checks with state: pruning keeps every HALLOC,
    HFREE, HLD and HST and the values of their sizes, handles and indices,
    so the oracle gives the same records (use after free, double and invalid
    free, heap bounds), ordinals, digest, counts and bitmap on the pruned
    program."""
    prog = gen.heap_program(which)
    pruned, st = B.cufz_prune_program(prog)
    assert orc.validate(pruned) == 0 and B.cufz_validate_program(pruned) == 0
    kinds = (bc.LD, bc.ST, bc.IF, bc.ELSE, bc.ENDIF, bc.LOOP, bc.ENDLOOP, bc.HALLOC, bc.HFREE,
             bc.HLD, bc.HST)
    assert [o[0] for o in bc.ops_of(prog) if o[0] in kinds] == \
        [o[0] for o in bc.ops_of(pruned) if o[0] in kinds]
    ins = gen.heap_inputs(4, n_programs=1, seed=420 + which)
    for o in (orc.opts(), orc.opts(iter_budget=2)):
        r0, c0, b0 = orc.run_batch([prog], ins, o, rec_cap=1 << 14, bitmaps=True, threads=2)
        r1, c1, b1 = orc.run_batch([pruned], ins, o, rec_cap=1 << 14, bitmaps=True, threads=2)
        assert checks_of(r0) == checks_of(r1) and c0.tobytes() == c1.tobytes()
        assert np.array_equal(b0, b1)


def test_prune_drops_the_value_of_a_heap_load_and_a_stored_value(orc):
    """A heap load whose value nothing reads and a heap store's value are
    not roots: the arithmetic that only they use goes, the accesses (index
    and handle) stay."""
    A = Asm(n_bufs=1)
    t, a0 = A.sreg(bc.TID_X), A.sreg(bc.ARG0)
    h = A.halloc(A.imm(16))
    v = A.hld(h, t, 4)
    A.hst(h, A.alu(bc.SUB, t, Imm(1)), A.alu(bc.MUL, A.alu(bc.ADD, v, a0), a0), 4)
    A.hfree(h)
    A.hfree(h)
    prog = A.build()
    pruned, st = B.cufz_prune_program(prog)
    assert st.n_ops_kept == st.n_ops_in - 3                    # add, mul and the read of a0
    inp = gen.make_inputs(1)
    gen.set_input(inp[0], 0, (2, 1, 1), (8, 1, 1), (3, 5), (16,))
    r0, c0, _ = orc.run(orc.Program(prog), inp[0], rec_cap=64)
    r1, c1, _ = orc.run(orc.Program(pruned), inp[0], rec_cap=64)
    assert checks_of(r0) == checks_of(r1) and c0.tobytes() == c1.tobytes()
    # per block: loads at t >= 4, stores at t - 1 outside [0, 4), and every
    # thread's second free
    assert int(r0["n_violations"]) == 2 * (4 + 4 + 8)


def test_prune_drops_the_dividend_of_a_dead_quotient(orc):
    """q = (t * t * a0) / (t - a1) with q unused: the division stays (its
    divisor decides the fault); the dividend's two multiplications and the
    read of a0 that only they use go."""
    A = Asm(n_bufs=1)
    t, a0, a1 = A.sreg(bc.TID_X), A.sreg(bc.ARG0), A.sreg(bc.ARG1)
    A.div(A.alu(bc.MUL, A.alu(bc.MUL, t, t), a0), A.alu(bc.SUB, t, a1))
    A.ld(0, t, 4)
    prog = A.build()
    pruned, st = B.cufz_prune_program(prog)
    assert st.n_ops_kept == st.n_ops_in - 3
    assert [o[0] for o in bc.ops_of(pruned)].count(bc.DIV) == 1
    inp = gen.make_inputs(1)
    gen.set_input(inp[0], 0, (2, 1, 1), (8, 1, 1), (3, 5), (16,))
    r0, c0, _ = orc.run(orc.Program(prog), inp[0], rec_cap=64)
    r1, c1, _ = orc.run(orc.Program(pruned), inp[0], rec_cap=64)
    assert checks_of(r0) == checks_of(r1) and c0.tobytes() == c1.tobytes()
    assert int(r0["n_violations"]) == 2 + 2 * 4                 # t == 5 faults; loads of t >= 4


@pytest.mark.parametrize("seed", range(24))
def test_validator_agrees_with_oracle_on_division_programs(orc, seed):
    rng = gen.SplitMix64(seed + 500)
    prog = bytearray(gen.div_program(seed % 16))
    for _ in range(rng.randint(1, 3)):
        pos = rng.randint(32, len(prog) - 1)
        prog[pos] = rng.choice((0x05, 0x06, rng.below(256)))
    p = bytes(prog)
    assert (B.cufz_validate_program(p) == 0) == (orc.validate(p) == 0)


@pytest.mark.parametrize("seed", range(24))
def test_validator_agrees_with_oracle_on_heap_programs(orc, seed):
    rng = gen.SplitMix64(seed + 700)
    prog = bytearray(gen.heap_program(seed % 16))
    for _ in range(rng.randint(1, 3)):
        pos = rng.randint(32, len(prog) - 1)
        prog[pos] = rng.choice((0x07, 0x08, 0x42, 0x43, rng.below(256)))
    p = bytes(prog)
    assert (B.cufz_validate_program(p) == 0) == (orc.validate(p) == 0)


def _without_barriers(prog: bytes) -> bytes:
    """The same program with its BARs as NOPs and its stores not performed."""
    ops = [(0, 0, 0, 0, 0) if o[0] == bc.BAR else o for o in bc.ops_of(prog)]
    h = bc.decode_header(prog)
    return bc.encode(ops, h["n_regs"], h["n_bufs"], h["shared_mask"], h["seed"], bc.loc_of(prog))


def _same_results(orc, a, b, ins, o):
    ra, ca, ma = orc.run_batch([a], ins, o, rec_cap=1 << 14, bitmaps=True, threads=2)
    rb, cb, mb = orc.run_batch([b], ins, o, rec_cap=1 << 14, bitmaps=True, threads=2)
    from conftest import record_keys
    return (checks_of(ra) == checks_of(rb) and np.array_equal(ma, mb) and
            all(record_keys(ca[k][: int(ra[k]["n_records"])]) ==
                record_keys(cb[k][: int(rb[k]["n_records"])]) for k in range(len(ins))))


@pytest.mark.parametrize("which", range(16))
def test_barrier_elimination_keeps_every_check(orc, which):
    """BarrierElimination (Sec. 5.2, Alg. 2): when no value read from a
    shared buffer reaches a check, the barriers and the stores' effect can
    go.  The oracle, which performs the stores phase by phase, gives the same
    results (records, counts, digest, bitmap) for the program, for it
    without barriers and without performed stores (what the engine runs),
    and for the library's pruned program (flag kept, barriers gone)."""
    prog = gen.barrier_program(which)
    pruned, st = B.cufz_prune_program(prog)
    assert bc.BAR not in [o[0] for o in bc.ops_of(pruned)]
    assert bc.decode_header(pruned)["flags"] == bc.PF_SHARED_STORES
    plain = _without_barriers(prog)
    assert orc.validate(plain) == 0 and orc.validate(pruned) == 0
    ins = gen.barrier_inputs(6, n_programs=1, seed=600 + which)
    for o in (orc.opts(), orc.opts(iter_budget=2)):
        assert _same_results(orc, prog, plain, ins, o)
        assert _same_results(orc, prog, pruned, ins, o)


def test_barriers_stay_where_shared_values_reach_checks(orc):
    """Where a value read from a shared buffer reaches an index or a branch,
    BarrierElimination does not apply, and the oracle shows why: without its
    barriers and stores the program's checks change.  Such a program takes
    the block-serial form: pruning keeps its barriers and the values its
    shared stores write (MathElimination with those values as uses), and
    the oracle gives the pruned program the same results; it compiles, and
    PREX plans nothing for it."""
    differs = 0
    for which in range(16):
        prog = gen.barrier_program(which, live=True)
        assert B.cufz_validate_program(prog) == 0 and orc.validate(prog) == 0
        pruned, st = B.cufz_prune_program(prog)
        assert orc.validate(pruned) == 0
        assert [o[0] for o in bc.ops_of(pruned)].count(bc.BAR) == \
            [o[0] for o in bc.ops_of(prog)].count(bc.BAR)
        assert bc.decode_header(pruned)["flags"] == bc.PF_SHARED_STORES
        ins = gen.barrier_inputs(4, n_programs=1, seed=700 + which)
        for o in (orc.opts(), orc.opts(iter_budget=2)):
            assert _same_results(orc, prog, pruned, ins, o)
        assert all(B.cufz_prex_plan(prog, x) is None and not B.cufz_prex_check(prog, x)
                   for x in ins)
        differs += not _same_results(orc, prog, _without_barriers(prog), ins, orc.opts())
    st, log, _ = B.cufz_compile_check(gen.barrier_programs(live=True))
    assert st == 0, log
    assert differs >= 8


@pytest.mark.parametrize("seed", range(24))
def test_validator_agrees_with_oracle_on_barrier_programs(orc, seed):
    """Barriers inside IF/LOOP, unknown flag bits and stray BARs are format
    errors for both validators alike."""
    rng = gen.SplitMix64(seed + 800)
    prog = bytearray(gen.barrier_program(seed % 16, live=bool(seed & 1)))
    for _ in range(rng.randint(1, 3)):
        if rng.below(3) == 0:
            prog[11] = rng.choice((0, 1, 2, 3, 0x81))
        else:
            pos = rng.randint(32, len(prog) - 1)
            prog[pos] = rng.choice((0x55, 0x50, 0x53, rng.below(256)))
    p = bytes(prog)
    assert (B.cufz_validate_program(p) == 0) == (orc.validate(p) == 0)


def test_disassembler_names_every_op():
    progs = (gen.c2_programs()[:4] + gen.c4_programs()[:2] + gen.div_programs()[:2]
             + gen.heap_programs()[:2] + gen.barrier_programs(2) + [gen.c1_program()])
    for p in progs:
        text = bc.disasm(p)
        assert "op0x" not in text and len(text.splitlines()) == bc.decode_header(p)["n_ops"]
