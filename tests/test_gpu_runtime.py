"""Runtime behaviour on the GPU: admission by free slots (a prefix is
accepted, BUSY otherwise), slots reused after release, error codes for
unknown tickets and programs, host-completed statuses, bounded waits,
program unloading and id reuse."""
import numpy as np
import pytest

from paper_2601_01048_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_01048_gb300 import binding
    binding.lib()
    return binding


def test_admission_busy_and_reuse(B, orc):
    prog = gen.c1_program()
    inputs = gen.c1_inputs(40, seed=4)
    ores, _, _ = orc.run_batch([prog], inputs, rec_cap=0)
    with B.Engine(max_slots=8, record_cap=1024, n_lanes=2) as E:
        E.load(prog)
        st, acc, first = B.cufz_submit_inputs(E.ctx, inputs)
        assert st == B.E_BUSY and acc == 8                       # a prefix, then BUSY
        st2, acc2, _ = B.cufz_submit_inputs(E.ctx, inputs[acc:])
        assert st2 == B.E_BUSY and acc2 == 0                     # nothing released yet
        B.cufz_sync(E.ctx, -1)
        done = B.cufz_poll_results(E.ctx, 64, 0)
        assert len(done) == 8
        assert B.cufz_submit_inputs(E.ctx, inputs[acc:])[0] == B.E_BUSY   # held until release
        for r in done:
            B.cufz_release(E.ctx, int(r["ticket"]))
        with pytest.raises(B.CufzError) as ei:
            B.cufz_release(E.ctx, int(done[0]["ticket"]))        # released twice
        assert ei.value.status == B.E_NOT_FOUND
        res, _, _ = E.run(inputs[acc:], records=False, bitmaps=False)
        assert np.array_equal(res["n_accesses"], ores["n_accesses"][acc:])
        assert np.array_equal(res["digest"], ores["digest"][acc:])
        for r in done:
            i = int(r["ticket"]) - first
            assert int(r["digest"]) == int(ores[i]["digest"])


def test_errors_and_host_completed_inputs(B):
    prog = gen.c1_program()
    ins = gen.make_inputs(3)
    gen.set_input(ins[0], 0, (0, 1, 1), (32, 1, 1), (), (4,))      # invalid launch
    gen.set_input(ins[1], 5, (1, 1, 1), (32, 1, 1), (), (4,))      # no such program
    gen.set_input(ins[2], 0, (1, 1, 1), (32, 1, 1), (0, 32), (128, 128, 128, 0))
    with B.Engine(max_slots=4) as E:
        with pytest.raises(B.CufzError) as ei:
            B.cufz_load_program(E.ctx, prog[:-3])
        assert ei.value.status == B.E_INVALID_PROGRAM
        E.load(prog)
        res, recs, bms = E.run(ins)
        assert [int(r["status"]) for r in res] == [B.ST_INVALID_CONFIG, B.ST_BAD_PROGRAM, B.ST_OK]
        assert not bms[0].any() and len(recs[0]) == 0
        with pytest.raises(B.CufzError) as ei:
            B.cufz_get_bitmap(E.ctx, 10 ** 9)
        assert ei.value.status == B.E_NOT_FOUND
        assert len(B.cufz_poll_results(E.ctx, 8, 1000)) == 0          # bounded, nothing pending
        B.cufz_sync(E.ctx, 1000)


@pytest.mark.parametrize("path", [0, 64])
def test_unload_and_reload(B, orc, path):
    """Unloading is refused while the program's inputs are in flight; after
    it the id's inputs complete as BAD_PROGRAM, a new load takes the id and
    its space, and the new program's results match the oracle (the compiled
    module is rebuilt for the reused id)."""
    p_old, p_other = gen.c1_program(), gen.c3_programs()[3]
    p_new = gen.c3_programs()[5]
    c1 = gen.c1_inputs(12, seed=21)
    c3 = gen.c3_inputs(12, seed=22, max_blocks=8, max_threads=256)
    with B.Engine(max_slots=64, record_cap=1 << 14, flags=B.CF_KEEP_BITMAPS | path) as E:
        assert E.load(p_old) == 0 and E.load(p_other) == 1
        st, acc, first = B.cufz_submit_inputs(E.ctx, c1)
        assert acc == len(c1)
        with pytest.raises(B.CufzError) as ei:
            B.cufz_unload_program(E.ctx, 0)                      # its inputs are in flight
        assert ei.value.status == B.E_BUSY
        B.cufz_sync(E.ctx, -1)
        for r in B.cufz_poll_results(E.ctx, 64, 0):
            B.cufz_release(E.ctx, int(r["ticket"]))
        B.cufz_unload_program(E.ctx, 0)
        with pytest.raises(B.CufzError) as ei:
            B.cufz_unload_program(E.ctx, 0)                      # not loaded any more
        assert ei.value.status == B.E_NOT_FOUND
        res, _, _ = E.run(c1[:3], records=False, bitmaps=False)
        assert all(int(r["status"]) == B.ST_BAD_PROGRAM for r in res)
        assert E.load(p_new) == 0                                # the freed id
        ins = c3.copy()
        ins["program_id"] = np.arange(len(ins)) % 2               # new program 0 and program 1
        dres, drecs, dbms = E.run(ins)
    ores, orecs, obms = orc.run_batch([p_new, p_other], ins, rec_cap=1 << 20, bitmaps=True)
    for k in range(len(ins)):
        for f in ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch", "n_edges"):
            assert int(dres[k][f]) == int(ores[k][f]), (k, f)
        assert np.array_equal(dbms[k], obms[k]), k


def _tune_key(prog: bytes, cta_threads: int, jit_min_ctas: int, flags: int) -> int:
    """The cache key (64-bit FNV-1a of the program bytes, then the kernel
    shape as little-endian u32s), restated from the cache's definition."""
    h = 0xCBF29CE484222325
    for b in prog + b"".join(int(v).to_bytes(4, "little") for v in (cta_threads, jit_min_ctas, flags & (4 | 32))):
        h = ((h ^ b) * 0x100000001B3) & ((1 << 64) - 1)
    return h


def test_autotune_cache(B, orc, tmp_path):
    """A cache file's choices (a first-version file: paths only) apply at
    load in a new context, results stay exact on the cached paths, and
    cufz_autotune rewrites the file in the current version: per program its
    path and lane mapping, which a new context applies at load."""
    progs = [gen.c3_programs()[k] for k in (0, 1, 2)]
    cache = tmp_path / "tune.txt"
    keys = [_tune_key(p, 256, 0, B.CF_JIT) for p in progs]
    cache.write_text("cufz-autotune 1\n" + f"{keys[1]:016x} 0\n")
    ins = gen.c3_inputs(24, seed=31, max_blocks=8, max_threads=256)
    ins["program_id"] %= 3
    with B.Engine(max_slots=64, flags=B.CF_KEEP_BITMAPS | B.CF_JIT, autotune_cache=str(cache)) as E:
        for p in progs:
            E.load(p)
        assert [B.cufz_get_program_path(E.ctx, k) for k in range(3)] == [True, False, True]
        dres, _, dbms = E.run(ins)
        B.cufz_autotune(E.ctx, ins)
    ores, _, obms = orc.run_batch(progs, ins, rec_cap=1 << 20, bitmaps=True)
    for k in range(len(ins)):
        assert int(dres[k]["digest"]) == int(ores[k]["digest"]) and np.array_equal(dbms[k], obms[k])
    lines = cache.read_text().split("\n")
    assert lines[0] == "cufz-autotune 2"
    got = {int(a, 16): (int(b), int(c)) for a, b, c in (l.split() for l in lines[1:] if l)}
    assert set(keys) <= set(got)
    assert all(p in (0, 1) and k in (1, 2, 4) and (p or k == 1) for p, k in got.values())
    # a forced choice written by hand is what a new context loads
    cache.write_text("cufz-autotune 2\n" + "".join(f"{k:016x} 1 {l}\n" for k, l in zip(keys, (1, 2, 4))))
    with B.Engine(max_slots=64, flags=B.CF_KEEP_BITMAPS | B.CF_JIT, autotune_cache=str(cache)) as E:
        for p in progs:
            E.load(p)
        assert [B.cufz_get_program_lanes(E.ctx, k) for k in range(3)] == [1, 2, 4]
        dres, _, dbms = E.run(ins)
    for k in range(len(ins)):
        assert int(dres[k]["digest"]) == int(ores[k]["digest"]) and np.array_equal(dbms[k], obms[k])


@pytest.mark.parametrize("path", [0, 64])
def test_verify_prune(B, path):
    """The library's own pruning check finds no difference between pruned and
    unpruned runs of random and branch-heavy programs, records included, and
    leaves the context as it found it (the temporary program is unloaded)."""
    progs = gen.c2_programs()[:3] + gen.c4_programs()[:2]
    c2 = gen.c2_inputs(progs[:3], per_program=3, seed=41, max_grid=3)
    c4 = gen.c4_inputs(6, n_programs=2, seed=42, max_blocks=4)
    with B.Engine(max_slots=64, record_cap=1 << 14, flags=B.CF_KEEP_BITMAPS | path) as E:
        for p in progs:
            E.load(p)
        for k in range(3):
            assert B.cufz_verify_prune(E.ctx, k, c2[c2["program_id"] == k]) == 0
        for k in range(2):
            assert B.cufz_verify_prune(E.ctx, 3 + k, c4[c4["program_id"] == k]) == 0
        assert E.load(gen.c1_program()) == 5                     # the temporary id was freed
        with pytest.raises(B.CufzError) as ei:
            B.cufz_verify_prune(E.ctx, 9, c2[:1])
        assert ei.value.status == B.E_NOT_FOUND


def test_admission_by_staging_memory(B, orc):
    """A batch admits inputs while its staging memory holds their work
    items: with room for 64 items of 2,048 test threads, a submit of inputs
    of 8 items each admits 8 of them and answers BUSY; resubmitting the rest
    as slots and lanes free up runs every input, and each equals the oracle.
    An input whose items exceed that memory on their own completes as
    LIMIT."""
    prog = gen.c1_program()
    ins = gen.c1_inputs(20, seed=51)
    for x in ins:
        x["grid"] = [128, 1, 1]                       # 16,384 threads: 8 items
    big = gen.make_inputs(1)
    gen.set_input(big[0], 0, (2048, 1, 1), (128, 1, 1), (0, 100), (400, 400, 400, 400))  # 128 items
    with B.Engine(max_slots=64, n_lanes=1, item_threads=2048, lane_items=64,
                  flags=B.CF_KEEP_BITMAPS | B.CF_AUTO_RELEASE) as E:
        E.load(prog)
        st, acc, first = B.cufz_submit_inputs(E.ctx, ins)
        assert st == B.E_BUSY and acc == 8, (st, acc)
        B.cufz_sync(E.ctx)
        out = list(B.cufz_poll_results(E.ctx, 64, 0))
        pos = acc
        while pos < len(ins):
            st, acc, _ = B.cufz_submit_inputs(E.ctx, ins[pos:])
            assert acc > 0
            pos += acc
            B.cufz_sync(E.ctx)
            out += list(B.cufz_poll_results(E.ctx, 64, 0))
        st, acc, _ = B.cufz_submit_inputs(E.ctx, big)
        assert acc == 1
        B.cufz_sync(E.ctx)
        lim = B.cufz_poll_results(E.ctx, 4, 0)
    assert [int(r["status"]) for r in lim] == [B.ST_LIMIT]
    res = sorted(out, key=lambda r: int(r["ticket"]))
    assert len(res) == len(ins)
    ores, _, _ = orc.run_batch([prog], ins)
    for k in range(len(ins)):
        for f in ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch"):
            assert int(res[k][f]) == int(ores[k][f]), (k, f)
