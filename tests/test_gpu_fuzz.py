"""A short fuzzing campaign on the GPU engine: the corpus grows with
new-coverage inputs, off-by-one bugs of the guarded 1D kernel are filed,
the device union equals the OR of the corpus's bitmaps as the oracle computes
them, and a resumed campaign rebuilds that union."""
import numpy as np
import pytest

from paper_2601_01048_gb300 import gen
from paper_2601_01048_gb300.fuzz import Campaign, EngineExecutor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_01048_gb300 import binding
    binding.lib()
    return binding


def test_campaign_on_the_engine(B, orc, tmp_path):
    prog = gen.c1_program()
    seeds = gen.c1_inputs(8, seed=71)
    with B.Engine(max_slots=256, record_cap=64, flags=B.CF_KEEP_BITMAPS) as E:
        E.load(prog)
        c = Campaign(EngineExecutor(E), [4], seeds, seed=5, batch=64)
        stats = [c.run_round() for _ in range(3)]
        assert sum(s.new_coverage for s in stats) == len(c.corpus) - len(seeds)
        assert len(c.buckets) > 0
        union = E.union()
        path = str(tmp_path / "campaign")
        c.checkpoint(path)
    _, _, obms = orc.run_batch([prog], c.corpus, rec_cap=0, bitmaps=True)
    assert np.array_equal(union, np.bitwise_or.reduce(obms, axis=0))
    with B.Engine(max_slots=256, record_cap=64, flags=B.CF_KEEP_BITMAPS) as E2:
        E2.load(prog)
        c2 = Campaign.resume(path, EngineExecutor(E2))
        assert np.array_equal(E2.union(), union) and c2.rounds == 3


def _workload():
    """Guarded 1D, branch-heavy and random programs (the random ones have
    loops, so a small back-edge budget makes hangs), seeds with small grids."""
    progs = gen.c3_programs()[:3] + gen.c4_programs()[:3] + [gen.c2_program(k) for k in (3, 5, 9)]
    seeds = gen.c5_corpus(progs, per_program=2, max_blocks=2)
    n_bufs = gen.program_bufs(progs)
    return progs, seeds, n_bufs


# A record area larger than any child's violations: a bucket's key comes
# from the child's stored records, and which records an overflowing child
# stores depends on the order its threads finish.
RECORD_CAP = 1 << 17


def _engine(B, progs):
    E = B.Engine(max_slots=256, record_cap=RECORD_CAP, iter_budget=40, flags=B.CF_JIT)
    for p in progs:
        E.load(p)
    return E


class _NoOverflow(EngineExecutor):
    """The engine executor, checking that no child's records overflowed."""

    def run(self, inputs):
        res, first = super().run(inputs)
        assert not (res["flags"] & 2).any(), "a child overflowed the record area"
        return res, first


def _same_campaign(host, dev):
    """The device campaign's corpus, buckets, hangs and counters equal the
    host campaign's."""
    inp, fav, picks = dev.corpus()
    assert np.array_equal(inp.view(np.uint8), host.corpus.view(np.uint8))
    assert np.array_equal(fav, host.favoured)
    assert np.array_equal(picks.astype(np.int64), host.picks)
    hb, db = host.buckets, dev.buckets()
    assert sorted(hb) == sorted(db)
    for k in hb:
        for f in ("hits", "round", "child"):
            assert hb[k][f] == db[k][f], (k, f)
        assert hb[k]["input"].tobytes() == db[k]["input"].tobytes(), k
    hh, dh = host.hangs, dev.hangs()
    assert [(h["round"], h["input"].tobytes()) for h in hh] == \
        [(h["round"], h["input"].tobytes()) for h in dh]
    s = dev.counters()
    assert (s.rounds, s.executed, s.violating, s.hang_execs, s.new_coverage) == \
        (host.rounds, host.executed, host.n_violating, host.n_hangs, host.n_new_coverage)
    assert s.corpus_dropped == host.corpus_dropped and s.limit_children == 0


def test_device_campaign_equals_host_campaign(B):
    """The campaign run on the device (selection, mutation, batch building,
    filing in kernels, one graph per round) reaches exactly the host
    campaign's state from the same seeds: corpus with favoured flags and pick
    counts, bug buckets with their first child and hits, unique hangs,
    counters, and the device union."""
    from paper_2601_01048_gb300.fuzz import DeviceCampaign

    progs, seeds, n_bufs = _workload()
    with _engine(B, progs) as E1:
        host = Campaign(_NoOverflow(E1), n_bufs, seeds, seed=0xC0DE, batch=192, corpus_cap=60)
        for _ in range(5):
            host.run_round()
        union_host = E1.union()
    assert host.n_new_coverage > 0 and host.buckets and host.n_hangs > 0
    assert host.corpus_dropped > 0                      # the cap is reached
    with _engine(B, progs) as E2:
        dev = DeviceCampaign(E2, seeds, seed=0xC0DE, batch=192, corpus_cap=60, bucket_cap=256)
        try:
            dev.run(2)
            dev.run(3)
            _same_campaign(host, dev)
            assert np.array_equal(E2.union(), union_host)
            st = dev.stats()
            assert st["rounds"] == 5 and st["execs_done"] == 5 * 192
        finally:
            dev.close()


def test_device_campaign_checkpoint_and_resume(B, tmp_path):
    """A device campaign checkpointed after 2 rounds and resumed on a fresh
    context continues exactly as the uninterrupted one; the host campaign
    resumes the device campaign's checkpoint to the same state too."""
    from paper_2601_01048_gb300.fuzz import DeviceCampaign

    progs, seeds, n_bufs = _workload()
    path = str(tmp_path / "dev")
    with _engine(B, progs) as E1:
        a = DeviceCampaign(E1, seeds, seed=77, batch=128, corpus_cap=200, bucket_cap=256,
                           n_bufs=n_bufs)
        try:
            a.run(2)
            a.checkpoint(path)
            a.run(3)
            a_corpus = a.corpus()
            a_buckets = a.buckets()
            a_hangs = a.hangs()
            a_cnt = a.counters()
            union_a = E1.union()
        finally:
            a.close()
    with _engine(B, progs) as E2:
        b = DeviceCampaign.resume(path, E2, bucket_cap=256)
        try:
            b.run(3)
            b_corpus = b.corpus()
            for x, y in zip(a_corpus, b_corpus):
                assert np.array_equal(np.asarray(x).view(np.uint8), np.asarray(y).view(np.uint8))
            assert b.buckets().keys() == a_buckets.keys()
            assert [h["input"].tobytes() for h in b.hangs()] == [h["input"].tobytes() for h in a_hangs]
            c = b.counters()
            assert (c.rounds, c.executed, c.violating, c.hang_execs, c.new_coverage) == \
                (a_cnt.rounds, a_cnt.executed, a_cnt.violating, a_cnt.hang_execs, a_cnt.new_coverage)
            assert np.array_equal(E2.union(), union_a)
        finally:
            b.close()
    with _engine(B, progs) as E3:
        h = Campaign.resume(path, _NoOverflow(E3))
        for _ in range(3):
            h.run_round()
        assert np.array_equal(h.corpus.view(np.uint8), a_corpus[0].view(np.uint8))
        assert sorted(h.buckets) == sorted(a_buckets)
        assert np.array_equal(E3.union(), union_a)


def test_device_campaign_on_every_program_kind(B):
    """Division, heap and block-serial barrier programs (whole test blocks
    per work item, the block-serial launch limits) in a device campaign:
    it reaches the host campaign's corpus, buckets, hangs, counters and
    union."""
    from paper_2601_01048_gb300.fuzz import DeviceCampaign

    progs = gen.div_programs(4) + gen.heap_programs(4) + gen.barrier_programs(4, live=True)
    seeds = np.concatenate([gen.div_inputs(8, n_programs=4, seed=91),
                            gen.heap_inputs(8, n_programs=4, seed=92),
                            gen.barrier_inputs(8, n_programs=4, seed=93)])
    seeds["program_id"][8:16] += 4
    seeds["program_id"][16:] += 8
    n_bufs = gen.program_bufs(progs)
    with _engine(B, progs) as E1:
        host = Campaign(_NoOverflow(E1), n_bufs, seeds, seed=0xB0B, batch=96, corpus_cap=100)
        for _ in range(4):
            host.run_round()
        union_host = E1.union()
    assert host.n_new_coverage > 0 and host.buckets
    with _engine(B, progs) as E2:
        dev = DeviceCampaign(E2, seeds, seed=0xB0B, batch=96, corpus_cap=100, bucket_cap=256)
        try:
            dev.run(4)
            _same_campaign(host, dev)
            assert np.array_equal(E2.union(), union_host)
        finally:
            dev.close()
