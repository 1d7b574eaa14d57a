"""Device-heap faults on the GPU (the temporal errors of Sec. 2.3): programs
whose test threads allocate, access, free and misuse heap blocks, on both
engines, bit-exact with the oracle (statuses, counts, first keys, digests,
use-after-free, double-free, invalid-free and heap-bounds records, access
records, bitmaps), pruned and unpruned, and with a record cap small enough
to overflow."""
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
def test_heap_faults(B, orc, path, prune):
    progs = gen.heap_programs()
    ins = gen.heap_inputs(96, seed=322)
    ores, orecs, obms = orc.run_batch(progs, ins, rec_cap=1 << 15, bitmaps=True)
    assert np.array_equal(ores["n_records"], ores["n_violations"])
    for cap in (1 << 14, 8):
        flags = B.CF_KEEP_BITMAPS | path | (0 if prune else B.CF_NO_PRUNE)
        with B.Engine(max_slots=128, record_cap=cap, flags=flags) as E:
            for p in progs:
                E.load(p)
            dres, drecs, dbms = E.run(ins)
        seen = set()
        for k in range(len(ins)):
            d, o = dres[k], ores[k]
            for f in FIELDS:
                assert int(d[f]) == int(o[f]), (cap, k, f)
            assert bool(int(d["flags"]) & B.FL_OVERFLOW) == (int(o["n_violations"]) > cap), k
            assert np.array_equal(dbms[k], obms[k]), (cap, k)
            full = record_keys(orecs[k][: int(o["n_records"])])
            if int(o["n_violations"]) <= cap:
                assert record_keys(drecs[k]) == full, (cap, k)
            else:
                assert len(drecs[k]) == cap and set(record_keys(drecs[k])) <= set(full), (cap, k)
            seen |= {(int(r["kind"]), int(r["cls"])) for r in drecs[k] if int(r["space"]) == 2}
        if cap > 8:
            assert {(0, 6), (1, 6), (3, 7), (3, 8)} <= seen, seen
