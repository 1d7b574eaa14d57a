"""Serving: inputs admitted while others run give the same result as when
each runs alone and as the oracle's (exact: statuses, counts, digests,
records, bitmaps, NEW_COV against the same empty epoch snapshot), and the
batches of the mix did overlap on the device."""
import numpy as np
import pytest

from paper_2601_01048_gb300 import gen
from conftest import record_keys

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_01048_gb300 import binding
    binding.lib()
    return binding




FIELDS = ("status", "flags", "n_accesses", "n_violations", "first_key", "digest", "n_branch",
          "n_threads", "n_records", "n_edges")


@pytest.mark.parametrize("path", [0, 64])
def test_alone_equals_in_mix(B, orc, path):
    from paper_2601_01048_gb300.serve import serve_open_loop

    progs = gen.c5_programs()
    corpus = gen.c5_corpus(progs, per_program=2, max_blocks=64)
    stream = gen.c5_stream(progs, corpus, 600, seed=99)
    arrivals = gen.poisson_arrivals(20000.0, 1.0, seed=3)[:600]
    stream = stream[: len(arrivals)]
    watch = list(range(0, len(stream), 37))
    cap = 1 << 14
    flags = B.CF_KEEP_BITMAPS | path
    with B.Engine(record_cap=cap, max_slots=128, n_lanes=4, flags=flags) as E:
        for p in progs:
            E.load(p)
        mix, lat, kept, wall = serve_open_loop(E, stream, arrivals, keep=set(watch))
        st = E.stats()
    assert np.all(np.isfinite(lat)) and st.batches > 1
    # the device intervals of the mix's batches (from their CUDA events)
    # intersect: batches admitted while others ran did run beside them
    assert st.overlapping_batch_pairs > 0 and st.max_concurrent_batches >= 2
    with B.Engine(record_cap=cap, max_slots=8, n_lanes=1, flags=flags) as A:
        for p in progs:
            A.load(p)
        for i in watch:
            alone, recs, bms = A.run(stream[i:i + 1])
            for f in FIELDS:
                assert int(alone[0][f]) == int(mix[i][f]), (i, f)
            assert np.array_equal(bms[0], kept[i][1]), i
            if int(alone[0]["n_violations"]) <= cap:
                assert record_keys(recs[0]) == record_keys(kept[i][0]), i
    # and every watched input of the mix equals the oracle
    sub = stream[watch]
    ores, orecs, obms = orc.run_batch(progs, sub, rec_cap=1 << 18, bitmaps=True)
    for j, i in enumerate(watch):
        for f in ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch",
                  "n_threads", "n_edges"):
            assert int(mix[i][f]) == int(ores[j][f]), (i, f)
        assert np.array_equal(kept[i][1], obms[j]), i
        n_o = int(ores[j]["n_violations"])
        if n_o <= cap:
            assert record_keys(kept[i][0]) == record_keys(orecs[j][:n_o]), i
