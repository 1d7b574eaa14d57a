"""The fuzzing campaign's host logic (queue, corpus, bug buckets,
checkpoints) against a fake executor with a deterministic coverage and bug
model; the engine behind the real executor is tested on the GPU elsewhere."""
import numpy as np

from paper_2601_01048_gb300 import binding as B
from paper_2601_01048_gb300 import gen
from paper_2601_01048_gb300.fuzz import Campaign

VIOL = np.dtype([("site", "<u2"), ("cls", "u1")])


class FakeExecutor:
    """Edges of an input: (program, arg0 // 64, len0 // 256); it violates
    when len0 < 100, at site arg1 & 3 with class 1 + (len0 & 1), and hits the
    back-edge budget when arg1 is a multiple of 5.  NEW_COV and the union
    follow the engine's rules (snapshot at each epoch)."""

    def __init__(self):
        self.union_set, self.snapshot = set(), set()
        self.log = []

    @staticmethod
    def edges(x):
        p = int(x["program_id"])
        return {(p, 0, int(x["args"][0]) // 64), (p, 1, int(x["buf_len"][0]) // 256)}

    def run(self, inputs):
        res = np.zeros(len(inputs), B.RESULT_DTYPE)
        first = []
        for k, x in enumerate(inputs):
            e = self.edges(x)
            if e - self.snapshot:
                res[k]["flags"] |= B.FL_NEW_COV
            self.union_set |= e
            if int(x["args"][1]) % 5 == 0:
                res[k]["flags"] |= B.FL_BUDGET
            bad = int(x["buf_len"][0]) < 100
            res[k]["status"] = B.ST_VIOLATION if bad else B.ST_OK
            if bad:
                r = np.zeros(1, VIOL)[0]
                r["site"], r["cls"] = int(x["args"][1]) & 3, 1 + (int(x["buf_len"][0]) & 1)
                first.append(r)
            else:
                first.append(None)
        self.log.append(len(inputs))
        return res, first

    def new_epoch(self):
        self.snapshot = set(self.union_set)

    def union(self):
        return self.union_set


def seeds(n=6):
    s = gen.make_inputs(n)
    for k in range(n):
        gen.set_input(s[k], k % 2, (4, 1, 1), (64, 1, 1), (k * 10, k), (1000 + k, 500, 500))
    return s


def test_corpus_grows_with_new_coverage_only_and_buckets_dedupe():
    ex = FakeExecutor()
    c = Campaign(ex, [3, 3], seeds(), seed=7, batch=32)
    assert ex.log == [6]                                       # the dry run
    total_new, buckets = 0, 0
    for _ in range(12):
        before = len(c.corpus)
        snapshot = set(ex.snapshot)                            # the union when the round starts
        st = c.run_round()
        assert st.executed == 32 and st.corpus_size == before + st.new_coverage
        # every entry the round added has an edge the union lacked at its start
        for x in c.corpus[before:]:
            assert ex.edges(x) - snapshot
        total_new += st.new_coverage
        buckets += st.new_buckets
    assert total_new > 0 and len(c.corpus) == 6 + total_new
    assert buckets == len(c.buckets) > 0
    assert sum(b["hits"] for b in c.buckets.values()) >= buckets
    # the union is the OR of the corpus's coverage
    cov = set()
    for x in c.corpus:
        cov |= ex.edges(x)
    assert cov == ex.union_set


def test_new_entries_are_picked_first():
    ex = FakeExecutor()
    c = Campaign(ex, [3, 3], seeds(), seed=3, batch=8)
    c.run_round()
    c.run_round()
    fav = np.flatnonzero(c.favoured)
    if len(fav):
        parents = c._parents()
        assert set(parents[: len(fav)].tolist()) == set(fav.tolist())


def test_checkpoint_resume_continues_exactly(tmp_path):
    a_ex = FakeExecutor()
    a = Campaign(a_ex, [3, 3], seeds(), seed=11, batch=16)
    for _ in range(4):
        a.run_round()
    path = str(tmp_path / "ckpt")
    a.checkpoint(path)
    union_at_ckpt = set(a_ex.union_set)
    after_a = [a.run_round() for _ in range(5)]

    b_ex = FakeExecutor()
    b = Campaign.resume(path, b_ex)
    assert b_ex.union_set == union_at_ckpt                    # rebuilt by running the corpus
    after_b = [b.run_round() for _ in range(5)]
    assert after_a == after_b
    assert np.array_equal(a.corpus, b.corpus) and a.rounds == b.rounds == 9
    assert [(h["round"], h["input"].tobytes()) for h in a.hangs] == \
        [(h["round"], h["input"].tobytes()) for h in b.hangs]
    assert a.n_hangs == b.n_hangs and b.seconds >= sum(r.seconds for r in after_b)
    assert {k: v["hits"] for k, v in a.buckets.items()} == {k: v["hits"] for k, v in b.buckets.items()}


def test_native_mutator_draws_like_the_generator_mutator():
    """cufz_mutate_inputs (the campaign's mutator) makes the same draws as
    gen.Mutator: the same records and the same generator state after them,
    over programs with 0 to 9 buffers and arguments and lengths at random;
    a program id without an entry is refused and changes nothing."""
    rng = gen.SplitMix64(7)
    n_bufs = [rng.below(10) for _ in range(20)]
    x = gen.make_inputs(3000)
    for k in range(len(x)):
        gen.set_input(x[k], rng.below(20), (rng.randint(1, 9), 1, 1), (32, 1, 1),
                      [rng.randint(-2**31, 2**31 - 1) for _ in range(4)],
                      [rng.randint(0, 1 << 40) for _ in range(9)])
    a, b = x.copy(), x.copy()
    m = gen.Mutator(0xF022)
    for k in range(len(a)):
        m.mutate(a[k], n_bufs[int(a[k]["program_id"])])
    state = B.cufz_mutate_inputs(b, n_bufs, 0xF022)
    assert state == m.rng.state
    assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
    assert (a != x).all()                                 # every record changed
    c = x[:4].copy()
    c[2]["program_id"] = 20
    try:
        B.cufz_mutate_inputs(c, n_bufs, 1)
        raise AssertionError("accepted a program id without a buffer count")
    except B.CufzError as e:
        assert e.status == B.E_INVALID_ARG
    assert np.array_equal(c[[0, 1, 3]], x[[0, 1, 3]])


def test_hangs_and_campaign_stats():
    """Budget stops are hangs; a hang that also reached new coverage is a
    unique hang and is kept (AFL's rule); stats() reports the paper's Table 2
    columns."""
    ex = FakeExecutor()
    c = Campaign(ex, [3, 3], seeds(), seed=5, batch=64)
    rounds = [c.run_round() for _ in range(10)]
    assert sum(r.hangs for r in rounds) == c.n_hangs > 0
    assert sum(r.new_hangs for r in rounds) == len(c.hangs) > 0
    assert all(r.new_hangs <= min(r.hangs, r.new_coverage) for r in rounds)
    for h in c.hangs:
        assert int(h["input"]["args"][1]) % 5 == 0
        assert any(h["input"].tobytes() == x.tobytes() for x in c.corpus)
    s = c.stats()
    assert s["execs_done"] == 640 and s["execs_per_sec"] > 0
    assert s["unique_crashes"] == len(c.buckets) and s["unique_hangs"] == len(c.hangs)
    assert s["corpus_count"] == len(c.corpus) and s["rounds"] == 10
    assert s["cycles_done"] == int(c.picks.min())


def test_command_line_reports_checkpoints_and_resumes(tmp_path, capsys):
    import contextlib
    import json

    from paper_2601_01048_gb300 import fuzz

    @contextlib.contextmanager
    def fake(programs, batch):
        assert len(programs) == 64 and batch == 32
        yield FakeExecutor()

    path = str(tmp_path / "campaign")
    fuzz.main(["--rounds", "4", "--batch", "32", "--report", "2", "--checkpoint", path],
              executor_factory=fake)
    lines = [json.loads(x) for x in capsys.readouterr().out.splitlines()]
    assert [x["rounds"] for x in lines] == [2, 4] and lines[-1]["execs_done"] == 128
    fuzz.main(["--resume", path + ".npz", "--rounds", "3", "--batch", "32", "--report", "5"],
              executor_factory=fake)
    last = json.loads(capsys.readouterr().out.splitlines()[-1])
    assert last["rounds"] == 7 and last["execs_done"] == 224


def test_child_streams_draw_like_the_generator_mutator():
    """cufz_mutate_children mutates child j of round r with gen.Mutator's
    draws from the state child_stream(seed, r, j): the stream of each child
    is its own, so the device campaign's kernel gives the same children."""
    rng = gen.SplitMix64(17)
    n_bufs = [rng.below(10) for _ in range(12)]
    x = gen.make_inputs(700)
    for k in range(len(x)):
        gen.set_input(x[k], rng.below(12), (rng.randint(1, 9), 1, 1), (32, 1, 1),
                      [rng.randint(-2**31, 2**31 - 1) for _ in range(4)],
                      [rng.randint(0, 1 << 40) for _ in range(9)])
    for seed, rnd in ((0xF022, 0), (0xF022, 5), (2**64 - 3, 2**31 + 7)):
        a, b = x.copy(), x.copy()
        for j in range(len(a)):
            m = gen.Mutator(0)
            m.rng.state = gen.child_stream(seed, rnd, j)
            m.mutate(a[j], n_bufs[int(a[j]["program_id"])])
        B.cufz_mutate_children(b, n_bufs, seed, rnd)
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
        assert (a != x).all()
    # streams differ between rounds and children
    a, b = x[:64].copy(), x[:64].copy()
    B.cufz_mutate_children(a, n_bufs, 1, 0)
    B.cufz_mutate_children(b, n_bufs, 1, 1)
    assert (a != b).any()


def test_corpus_and_hang_caps():
    """Entries with new coverage beyond corpus_cap, and unique hangs beyond
    hang_cap, are counted as dropped; the round is otherwise the same as
    without caps (same children, same order)."""
    ex_a, ex_b = FakeExecutor(), FakeExecutor()
    a = Campaign(ex_a, [3, 3], seeds(), seed=9, batch=64)
    b = Campaign(ex_b, [3, 3], seeds(), seed=9, batch=64, corpus_cap=9, hang_cap=1)
    a.run_round()
    b.run_round()
    assert len(a.corpus) > 9 and len(a.hangs) > 1          # the caps matter here
    assert np.array_equal(b.corpus, a.corpus[:9])
    assert b.corpus_dropped == len(a.corpus) - 9
    assert len(b.hangs) == 1 and b.hangs[0]["input"].tobytes() == a.hangs[0]["input"].tobytes()
    assert b.hangs_dropped == len(a.hangs) - 1
    assert b.n_hangs == a.n_hangs and b.n_new_coverage == a.n_new_coverage
    s = b.stats()
    assert s["corpus_count"] == 9 and s["corpus_dropped"] == b.corpus_dropped


def test_campaign_config_limits():
    """cufz_campaign_bytes sizes valid configurations and gives 0 for
    invalid ones (batch 1..8192, corpus 1..16384, bucket table a power of
    two in 16..2^20, hang cap 1..2^20, item capacity up to 2^24); creating a
    campaign without a context is refused before anything runs."""
    def cfg(**kw):
        base = dict(batch=1024, corpus_cap=4096, bucket_cap=1024, hang_cap=256, item_threads=0,
                    max_items=0, seed=1)
        base.update(kw)
        return B.cufz_campaign_config(**base)

    small = B.cufz_campaign_bytes(cfg())
    assert small > 0 and small % 256 == 0
    assert B.cufz_campaign_bytes(cfg(corpus_cap=16384)) > small
    assert B.cufz_campaign_bytes(cfg(batch=8192)) > small
    for bad in (dict(batch=0), dict(batch=8193), dict(corpus_cap=0), dict(corpus_cap=16385),
                dict(bucket_cap=1000), dict(bucket_cap=8), dict(hang_cap=0),
                dict(max_items=(1 << 24) + 1)):
        assert B.cufz_campaign_bytes(cfg(**bad)) == 0, bad
    try:
        B.cufz_campaign_create(None, cfg(), 0, small, seeds(2))
        raise AssertionError("created a campaign without a context")
    except B.CufzError as e:
        assert e.status == B.E_INVALID_ARG


def test_first_record_is_the_least_key():
    """A bucket's key comes from the stored record of least (block, thread,
    ordinal), whatever order the records were stored in."""
    from paper_2601_01048_gb300.fuzz import first_record

    recs = np.zeros(5, B.VIOLATION_DTYPE)
    keys = [(3, 0, 1), (1, 7, 4), (1, 2, 9), (1, 2, 3), (2, 0, 0)]
    for r, (b, t, o) in zip(recs, keys):
        r["block_lin"], r["thread_lin"], r["ordinal"], r["site"] = b, t, o, 100 * b + 10 * t + o
    rng = gen.SplitMix64(5)
    for _ in range(8):
        perm = [int(v) for v in np.argsort([rng.next() for _ in range(5)])]
        f = first_record(recs[perm])
        assert (int(f["block_lin"]), int(f["thread_lin"]), int(f["ordinal"])) == (1, 2, 3)
        assert int(f["site"]) == 123
    assert first_record(recs[:0]) is None and first_record(None) is None
