"""The allocation-free entry point (cufz_run_noalloc) gives the same results
as a context does for the same inputs.

It exists for callers that cannot allocate device memory (code running under
CUDA graph capture, plugins whose framework owns all device memory, services
with a fixed device footprint): its scratch is a fixed array inside the
library, shared by every call, so two calls in a row must not see each
other's leftovers.  This file is collected last on purpose."""
import numpy as np
import pytest
from conftest import record_keys

pytestmark = pytest.mark.gpu

FIELDS = ("status", "n_accesses", "n_violations", "first_key", "digest", "n_branch",
          "n_threads", "n_records", "n_edges")




def test_noalloc_matches_context_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_01048_gb300 import binding as B
    from paper_2601_01048_gb300 import gen

    progs = [gen.c1_program(), gen.c2_program(5)]
    a = gen.c1_inputs(40, seed=123)
    a = a[np.argmax(a["args"][:, 0] < 0)]                      # an input with violations
    b = gen.c2_inputs([progs[1]], per_program=1, seed=77, max_grid=1)[0]
    b["program_id"] = 1
    inputs = np.array([a, b], dtype=gen.INPUT_DTYPE)
    cap = 1 << 14

    with B.Engine(record_cap=cap, max_slots=8) as E:              # the existing entry points
        for p in progs:
            E.load(p)
        ref, ref_recs, ref_bms = E.run(inputs)

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    records = torch.empty(cap * 32, dtype=torch.uint8, device=dev)
    bitmap = torch.empty(65536, dtype=torch.uint8, device=dev)
    result = torch.empty(96, dtype=torch.uint8, device=dev)
    for k in (0, 1, 0):                                           # calls in a row
        records.fill_(0xAB)
        bitmap.fill_(0xCD)
        torch.cuda.synchronize(dev)
        B.cufz_run_noalloc(progs[int(inputs[k]["program_id"])], inputs[k], records.data_ptr(), cap,
                           bitmap.data_ptr(), result.data_ptr(), stream=stream)
        res = np.frombuffer(result.cpu().numpy().tobytes(), dtype=B.RESULT_DTYPE)[0]
        for f in FIELDS:
            assert int(res[f]) == int(ref[k][f]), (k, f)
        assert int(res["flags"]) == int(ref[k]["flags"]), k
        assert int(res["user_tag"]) == int(ref[k]["user_tag"])
        n = int(res["n_records"])
        recs = np.frombuffer(records.cpu().numpy().tobytes(), dtype=B.VIOLATION_DTYPE)[:n]
        assert int(ref[k]["n_violations"]) <= cap          # record sets are unique then
        assert record_keys(recs) == record_keys(ref_recs[k])
        assert np.array_equal(bitmap.cpu().numpy(), ref_bms[k])
    assert int(ref[0]["n_violations"]) > 0 and int(ref[1]["n_edges"]) > 0
