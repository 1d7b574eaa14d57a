"""Performed shared stores and barriers on the GPU (AXIPrune's
BarrierElimination, Sec. 5.2): programs whose barriers the loader removes
run on both engines without performing a store and equal the oracle, which
performs the stores phase by phase (statuses, counts, first keys, digests,
records, bitmaps), pruned and unpruned.  Programs whose barriers must stay
run compiled in the block-serial form (each test block's threads in thread
order, phase by phase, stores performed) and equal the oracle the same way;
the interpreter refuses them, and launches beyond the form's limits
complete as LIMIT."""
import numpy as np
import pytest

from paper_2601_01048_gb300 import gen
from conftest import record_keys

pytestmark = pytest.mark.gpu

FIELDS = ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch", "n_threads",
          "n_edges")


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_01048_gb300 import binding
    binding.lib()
    return binding


@pytest.mark.parametrize("path", [0, 64])
@pytest.mark.parametrize("prune", [True, False])
def test_eliminated_barriers(B, orc, path, prune):
    progs = gen.barrier_programs()
    ins = gen.barrier_inputs(96, seed=323)
    ores, orecs, obms = orc.run_batch(progs, ins, rec_cap=1 << 15, bitmaps=True)
    assert np.array_equal(ores["n_records"], ores["n_violations"])
    flags = B.CF_KEEP_BITMAPS | path | (0 if prune else B.CF_NO_PRUNE)
    with B.Engine(max_slots=128, record_cap=1 << 14, flags=flags) as E:
        for p in progs:
            E.load(p)
        if not path:                          # the interpreter runs no block-serial program
            with pytest.raises(B.CufzError) as e:
                E.load(gen.barrier_program(0, live=True))
            assert e.value.status == B.E_UNSUPPORTED
        dres, drecs, dbms = E.run(ins)
    for k in range(len(ins)):
        d, o = dres[k], ores[k]
        for f in FIELDS:
            assert int(d[f]) == int(o[f]), (k, f)
        assert np.array_equal(dbms[k], obms[k]), k
        assert record_keys(drecs[k]) == record_keys(orecs[k][: int(o["n_records"])]), k


@pytest.mark.parametrize("prune", [True, False])
def test_block_serial_barriers(B, orc, prune):
    """Programs whose barriers must stay, on the compiled path, over many
    blocks (several blocks per work item and per CUDA thread), with a normal
    and a small record cap and a budget that stops threads in loops: every
    result equals the oracle's phased execution.  cufz_verify_prune finds no
    difference between the pruned and unpruned forms, and the form's limits
    (64 threads per block, 1 KiB of shared buffers) give LIMIT."""
    progs = gen.barrier_programs(live=True)
    ins = gen.barrier_inputs(96, seed=341, max_blocks=300)
    flags = B.CF_KEEP_BITMAPS | B.CF_JIT | (0 if prune else B.CF_NO_PRUNE)
    for budget, cap in ((4096, 1 << 14), (2, 16)):
        with B.Engine(max_slots=128, record_cap=cap, flags=flags, iter_budget=budget) as E:
            for p in progs:
                E.load(p)
            assert all(B.cufz_get_program_path(E.ctx, k) for k in range(len(progs)))
            dres, drecs, dbms = E.run(ins)
            if budget == 4096:
                assert B.cufz_verify_prune(E.ctx, 3, ins[ins["program_id"] == 3]) == 0
                big = gen.make_inputs(2)
                gen.set_input(big[0], 0, (2, 1, 1), (65, 1, 1), (1, 2), (64, 64, 260, 65))
                gen.set_input(big[1], 0, (2, 1, 1), (16, 1, 1), (1, 2), (64, 64, 1000, 100))
                lim, _, _ = E.run(big)
                assert [int(r["status"]) for r in lim] == [B.ST_LIMIT, B.ST_LIMIT]
        o = orc.opts(iter_budget=budget)
        ores, orecs, obms = orc.run_batch(progs, ins, o, rec_cap=1 << 15, bitmaps=True)
        for k in range(len(ins)):
            d, r = dres[k], ores[k]
            for f in FIELDS:
                assert int(d[f]) == int(r[f]), (budget, k, f)
            assert int(d["flags"]) & B.FL_BUDGET == int(r["flags"]) & B.FL_BUDGET, (budget, k)
            assert np.array_equal(dbms[k], obms[k]), (budget, k)
            n = int(r["n_violations"])
            if n <= cap:
                assert record_keys(drecs[k]) == record_keys(orecs[k][:n]), (budget, k)
            elif int(r["n_records"]) == n:               # the oracle kept them all
                assert set(record_keys(drecs[k])) <= set(record_keys(orecs[k][:n])), (budget, k)
        if budget == 2:
            assert any(int(r["flags"]) & B.FL_BUDGET for r in ores)
