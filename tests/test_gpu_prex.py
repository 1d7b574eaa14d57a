"""PREX on the GPU (Sec. 5.1): with CUFZ_CF_PREX, an input whose program
qualifies runs only its corner threads, and its verdict (violation or not)
is the full grid's, the oracle's; its records are records of the full run.
Inputs that do not qualify run the full grid, bit-exact with the oracle."""
import numpy as np
import pytest

from paper_2601_01048_gb300 import gen

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


def n_corners(inp):
    g = [int(v) for v in inp["grid"]] + [int(v) for v in inp["block"]]
    return int(np.prod([2 if v > 1 else 1 for v in g]))


@pytest.mark.parametrize("path", [0, 64])
def test_prex_verdicts(B, orc, path):
    progs = gen.affine_programs()[:6] + [gen.c1_program()] + gen.c2_programs()[:1]
    aff = gen.affine_inputs(36, seed=61, max_blocks=24, max_threads=96)
    aff["program_id"] %= 6
    c1 = gen.c1_inputs(8, seed=62)
    c1["program_id"] = 6
    c2 = gen.c2_inputs(progs[7:8], per_program=4, seed=63, max_grid=2)
    c2["program_id"] = 7
    ins = np.concatenate([aff, c1, c2])
    eligible = [B.cufz_prex_check(progs[int(x["program_id"])], x) for x in ins]
    assert all(eligible[:len(aff)]) and not any(eligible[len(aff):])
    with B.Engine(max_slots=128, record_cap=1 << 15, flags=B.CF_KEEP_BITMAPS | B.CF_PREX | path) as E:
        for p in progs:
            E.load(p)
        dres, drecs, dbms = E.run(ins)
    ores, orecs, obms = orc.run_batch(progs, ins, rec_cap=1 << 20, bitmaps=True)
    n_viol = 0
    for k in range(len(ins)):
        d, o = dres[k], ores[k]
        assert int(d["status"]) == int(o["status"]), k
        if eligible[k]:
            assert int(d["flags"]) & B.FL_PARTIAL
            assert int(d["n_threads"]) == n_corners(ins[k])
            assert int(d["n_violations"]) <= int(o["n_violations"])
            full = set(zip(*(orecs[k][f][:int(o["n_records"])].tolist() for f in KEYS)))
            assert set(zip(*(drecs[k][f].tolist() for f in KEYS))) <= full
            n_viol += int(o["status"]) == B.ST_VIOLATION
        else:
            assert not int(d["flags"]) & B.FL_PARTIAL
            for f in ("n_accesses", "n_violations", "first_key", "digest", "n_branch", "n_edges"):
                assert int(d[f]) == int(o[f]), (k, f)
            assert np.array_equal(dbms[k], obms[k])
    assert 0 < n_viol < len(aff)
