import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_collection_modifyitems(config, items):
    """The PREX, division-fault, heap-fault and barrier tests, then the
    full-size workload tests, run after the established parity tests (the
    first four cover the newest device and runtime code, the full-size ones
    take the longest).  The allocation-free entry point's tests come last of
    all, so a run that stops at its first failure has run every other test
    before them."""
    late = ("test_gpu_prex", "test_gpu_divfault", "test_gpu_heap", "test_gpu_barrier",
            "test_gpu_fullsize", "test_zz_no_alloc")
    items.sort(key=lambda item: next((k + 1 for k, f in enumerate(late) if f in item.nodeid), 0))


def golden(name):
    rows = []
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle
    oracle.lib()
    return oracle


RECORD_KEYS = ("block_lin", "thread_lin", "ordinal", "site", "buf", "kind", "width", "space", "cls",
               "byte_off")


def record_keys(recs):
    """A record array (engine or oracle) as the sorted list of its records'
    identifying fields, for comparing record sets."""
    if recs is None or len(recs) == 0:
        return []
    return sorted(zip(*(recs[c].tolist() for c in RECORD_KEYS)))



def checks_of(res):
    """Oracle results as bytes with the executed-op count cleared: every
    field pruning must leave unchanged (pruning removes ops, never checks,
    branches or their outcomes)."""
    r = res.copy()
    r["n_ops"] = 0
    return r.tobytes()
