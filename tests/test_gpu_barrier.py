"""Performed shared stores and barriers on the GPU (AXIPrune's
BarrierElimination, Sec. 5.2): programs whose barriers the loader removes
run on both engines without performing a store and equal the oracle, which
performs the stores phase by phase (statuses, counts, first keys, digests,
records, bitmaps), pruned and unpruned; programs whose barriers must stay
are refused at load."""
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
