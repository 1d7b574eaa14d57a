"""Parity at the benchmark's full sizes, in the launch configuration it
times: the whole workload of configurations 2, 3 and 4 (8,192, 4,096 and
16,384 inputs, grids up to 256 x 256 blocks of 256 threads and up to 67 M
threads per input) admitted in one submit, so one persistent launch per
lane, with the per-program paths the autotuner picks, as bench.py runs it.

  - Sampled outputs: 48 inputs of the workload small enough for the oracle
    to run one by one (at most 2^15 test threads), spread evenly over the
    batch, equal the oracle bit for bit: status, counts, digest, first key,
    records (any record_cap of them when an input overflows) and bitmap.
  - Every input, at any size: the compiled and autotuned run equals a run of
    the bytecode interpreter alone (two independent engines) in status,
    flags, every count (the executed-op count n_ops, the roofline's largest
    term, included), digest, first key, record count and bitmap; and
    status, record count and OVERFLOW agree with the counts.  The sampled
    inputs' n_ops also equals the oracle's count on the pruned program."""
import hashlib
import sys
import os

import numpy as np
import pytest

from conftest import record_keys

pytestmark = pytest.mark.gpu

SMALL = 1 << 15
N_SAMPLED = 48
FIELDS = ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch", "n_threads",
          "n_edges", "n_records", "n_ops")


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_01048_gb300 import binding
    binding.lib()
    return binding


def bench_workload(name):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    return bench.workload(name, 0)


def threads_of(inputs):
    return (inputs["grid"].astype(np.int64).prod(axis=1) * inputs["block"].astype(np.int64).prod(axis=1))


def run_whole(B, progs, inputs, cap, compiled, keep):
    """The whole workload in one submit; returns results in input order, a
    digest of every input's bitmap, and records and bitmaps of the inputs in
    `keep`."""
    flags = B.CF_KEEP_BITMAPS | (B.CF_JIT if compiled else 0)
    n = len(inputs)
    res = np.zeros(n, B.RESULT_DTYPE)
    bm_digest = [None] * n
    kept = {}
    with B.Engine(max_slots=n, record_cap=cap, flags=flags, n_lanes=2) as E:
        for p in progs:
            E.load(p)
        if compiled:
            sample = np.concatenate([inputs[inputs["program_id"] == p][:8]
                                     for p in np.unique(inputs["program_id"])])
            B.cufz_autotune(E.ctx, sample)
        st, acc, first = B.cufz_submit_inputs(E.ctx, inputs)
        assert acc == n, (st, acc)
        got = 0
        while got < n:
            out = B.cufz_poll_results(E.ctx, n, 60_000_000)
            assert len(out), "no results within 60 s"
            for r in out:
                t = int(r["ticket"])
                i = t - first
                res[i] = r
                bm = B.cufz_get_bitmap(E.ctx, t)
                bm_digest[i] = hashlib.blake2b(bm.tobytes(), digest_size=16).digest()
                if i in keep:
                    kept[i] = (B.cufz_get_records(E.ctx, t, int(r["n_records"])), bm.copy())
                B.cufz_release(E.ctx, t)
            got += len(out)
    return res, bm_digest, kept


@pytest.mark.parametrize("name", ["c2", "c3", "c4"])
def test_full_size_workload(B, orc, name):
    _, progs, inputs, cap = bench_workload(name)
    nt = threads_of(inputs)
    small = np.flatnonzero(nt <= SMALL)
    assert len(small) >= N_SAMPLED
    small = small[np.unique(np.linspace(0, len(small) - 1, N_SAMPLED).astype(np.int64))]
    keep = set(small.tolist())
    dres, ddig, dkept = run_whole(B, progs, inputs, cap, compiled=True, keep=keep)
    ires, idig, _ = run_whole(B, progs, inputs, cap, compiled=False, keep=set())

    # every input: two engines, and the counts' own consistency
    for f in FIELDS:
        assert np.array_equal(dres[f], ires[f]), f
    mask = B.FL_BUDGET | B.FL_OVERFLOW | B.FL_NEW_COV
    assert np.array_equal(dres["flags"] & mask, ires["flags"] & mask)
    assert ddig == idig
    assert np.array_equal(dres["n_threads"].astype(np.int64), nt)
    assert np.array_equal(dres["status"] == B.ST_VIOLATION, dres["n_violations"] > 0)
    assert np.array_equal(dres["n_records"].astype(np.int64), np.minimum(dres["n_violations"], cap))
    assert np.array_equal((dres["flags"] & B.FL_OVERFLOW) != 0, dres["n_violations"] > cap)

    # sampled outputs: the oracle, input by input
    sub = inputs[small]
    ores, orecs, obms = orc.run_batch(progs, sub, rec_cap=1 << 18, bitmaps=True)
    pres, _, _ = orc.run_batch([B.cufz_prune_program(p)[0] for p in progs], sub)
    for j, i in enumerate(small.tolist()):
        d, o = dres[i], ores[j]
        for f in ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch",
                  "n_threads", "n_edges"):
            assert int(d[f]) == int(o[f]), (i, f)
        assert int(d["flags"]) & B.FL_BUDGET == int(o["flags"]) & B.FL_BUDGET, i
        assert int(d["n_ops"]) == int(pres[j]["n_ops"]), i
        recs, bm = dkept[i]
        assert np.array_equal(bm, obms[j]), i
        n_o = int(o["n_violations"])
        full = record_keys(orecs[j][: int(o["n_records"])])
        if n_o <= cap:
            assert record_keys(recs) == full, i
        else:
            assert len(recs) == cap, i
            if int(o["n_records"]) == n_o:                     # the oracle kept them all
                assert set(record_keys(recs)) <= set(full), i
