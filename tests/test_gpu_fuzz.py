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
