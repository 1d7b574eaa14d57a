"""PREX on the GPU (Sec. 5.1): with CUFZ_CF_PREX, an input with a plan
(cufz_prex_plan: the corner threads of an unguarded affine program, or the
guards' change points of a guarded 1D launch) runs only the planned threads.
Its verdict (violation or not) is the full grid's, the oracle's, and its
records are exactly the full run's records of the planned threads.  Inputs
without a plan run the full grid, bit-exact with the oracle."""
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


def planned_records(orecs, o, plan, T):
    """The oracle's full-run records of the planned threads, as key tuples."""
    r = orecs[: int(o["n_records"])]
    keep = np.isin(r["block_lin"].astype(np.int64) * T + r["thread_lin"], plan)
    return set(zip(*(r[f][keep].tolist() for f in KEYS)))


@pytest.mark.parametrize("path", [0, 64])
def test_prex_verdicts(B, orc, path):
    progs = gen.affine_programs()[:6] + [gen.c1_program()] + gen.c2_programs()[:1] + gen.c3_programs()
    aff = gen.affine_inputs(36, seed=61, max_blocks=24, max_threads=96)
    aff["program_id"] %= 6
    c1 = gen.c1_inputs(8, seed=62)
    c1["program_id"] = 6
    c2 = gen.c2_inputs(progs[7:8], per_program=4, seed=63, max_grid=2)
    c2["program_id"] = 7
    c3 = gen.c3_inputs(16, seed=64, max_blocks=64, max_threads=256)
    c3["program_id"] += 8
    ins = np.concatenate([aff, c1, c2, c3])
    progs_of = [progs[int(x["program_id"])] for x in ins]
    corner = [B.cufz_prex_check(p, x) for p, x in zip(progs_of, ins)]
    plans = [B.cufz_prex_plan(p, x) for p, x in zip(progs_of, ins)]
    n_aff, n_c1, n_c2 = len(aff), len(c1), len(c2)
    assert all(corner[:n_aff]) and not any(corner[n_aff:])
    guarded = list(range(n_aff, n_aff + n_c1)) + list(range(n_aff + n_c1 + n_c2, len(ins)))
    assert all(plans[k] is not None for k in guarded)          # guarded 1D: line plans
    assert all(plans[k] is None for k in range(n_aff + n_c1, n_aff + n_c1 + n_c2))  # 2D blocks
    with B.Engine(max_slots=128, record_cap=1 << 15, flags=B.CF_KEEP_BITMAPS | B.CF_PREX | path) as E:
        for p in progs:
            E.load(p)
        dres, drecs, dbms = E.run(ins)
    ores, orecs, obms = orc.run_batch(progs, ins, rec_cap=1 << 20, bitmaps=True)
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
