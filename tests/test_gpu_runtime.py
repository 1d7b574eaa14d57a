"""Runtime behaviour on the GPU: admission by free slots (a prefix is
accepted, BUSY otherwise), slots reused after release, error codes for
unknown tickets and programs, host-completed statuses, bounded waits."""
import numpy as np
import pytest

from paper_2601_01048_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_01048_gb300 import binding
    binding.lib()
    return binding


def test_admission_busy_and_reuse(B, orc):
    prog = gen.c1_program()
    inputs = gen.c1_inputs(40, seed=4)
    ores, _, _ = orc.run_batch([prog], inputs, rec_cap=0)
    with B.Engine(max_slots=8, record_cap=1024, n_lanes=2) as E:
        E.load(prog)
        st, acc, first = B.cufz_submit_inputs(E.ctx, inputs)
        assert st == B.E_BUSY and acc == 8                       # a prefix, then BUSY
        st2, acc2, _ = B.cufz_submit_inputs(E.ctx, inputs[acc:])
        assert st2 == B.E_BUSY and acc2 == 0                     # nothing released yet
        B.cufz_sync(E.ctx, -1)
        done = B.cufz_poll_results(E.ctx, 64, 0)
        assert len(done) == 8
        assert B.cufz_submit_inputs(E.ctx, inputs[acc:])[0] == B.E_BUSY   # held until release
        for r in done:
            B.cufz_release(E.ctx, int(r["ticket"]))
        with pytest.raises(B.CufzError) as ei:
            B.cufz_release(E.ctx, int(done[0]["ticket"]))        # released twice
        assert ei.value.status == B.E_NOT_FOUND
        res, _, _ = E.run(inputs[acc:], records=False, bitmaps=False)
        assert np.array_equal(res["n_accesses"], ores["n_accesses"][acc:])
        assert np.array_equal(res["digest"], ores["digest"][acc:])
        for r in done:
            i = int(r["ticket"]) - first
            assert int(r["digest"]) == int(ores[i]["digest"])


def test_errors_and_host_completed_inputs(B):
    prog = gen.c1_program()
    ins = gen.make_inputs(3)
    gen.set_input(ins[0], 0, (0, 1, 1), (32, 1, 1), (), (4,))      # invalid launch
    gen.set_input(ins[1], 5, (1, 1, 1), (32, 1, 1), (), (4,))      # no such program
    gen.set_input(ins[2], 0, (1, 1, 1), (32, 1, 1), (0, 32), (128, 128, 128, 0))
    with B.Engine(max_slots=4) as E:
        with pytest.raises(B.CufzError) as ei:
            B.cufz_load_program(E.ctx, prog[:-3])
        assert ei.value.status == B.E_INVALID_PROGRAM
        E.load(prog)
        res, recs, bms = E.run(ins)
        assert [int(r["status"]) for r in res] == [B.ST_INVALID_CONFIG, B.ST_BAD_PROGRAM, B.ST_OK]
        assert not bms[0].any() and len(recs[0]) == 0
        with pytest.raises(B.CufzError) as ei:
            B.cufz_get_bitmap(E.ctx, 10 ** 9)
        assert ei.value.status == B.E_NOT_FOUND
        assert len(B.cufz_poll_results(E.ctx, 8, 1000)) == 0          # bounded, nothing pending
        B.cufz_sync(E.ctx, 1000)
