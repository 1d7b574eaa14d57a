"""The open-loop serving driver's host logic on the CPU, against a fake
engine with a fixed number of slots and a fixed service time: every input
is submitted once and completes, a BUSY submit leaves the rest for later,
latency counts from the scheduled arrival (a backlog shows in it), held
results are read before their slot is released, and a stuck engine ends in
E_TIMEOUT."""
import time

import numpy as np
import pytest

from paper_2601_01048_gb300 import binding as B
from paper_2601_01048_gb300 import gen, serve


class FakeEngine:
    """Admits up to `slots` inputs; each completes `service_s` after it was
    admitted (never, if service_s is None)."""

    def __init__(self, slots, service_s, auto_release=False):
        import types
        self.ctx = object()
        self.cfg = types.SimpleNamespace(flags=B.CF_AUTO_RELEASE if auto_release else 0)
        self.slots, self.service_s = slots, service_s
        self.next_ticket = 1
        self.running = {}       # ticket -> (due time, user_tag)
        self.polled = set()     # polled, not yet released
        self.submitted = []     # user tags in submit order
        self.busy_returns = 0

    def submit(self, ctx, inputs):
        assert ctx is self.ctx
        room = self.slots - len(self.running) - len(self.polled)
        acc = max(0, min(room, len(inputs)))
        first = self.next_ticket
        now = time.perf_counter()
        for k in range(acc):
            due = float("inf") if self.service_s is None else now + self.service_s
            self.running[self.next_ticket] = (due, int(inputs[k]["user_tag"]))
            self.submitted.append(int(inputs[k]["user_tag"]))
            self.next_ticket += 1
        if acc < len(inputs):
            self.busy_returns += 1
        return (B.E_BUSY if acc < len(inputs) else B.OK), acc, first

    def poll(self, ctx, max_n, timeout_ms):
        now = time.perf_counter()
        done = sorted(t for t, (due, _) in self.running.items() if due <= now)[:max_n]
        out = np.zeros(len(done), B.RESULT_DTYPE)
        for r, t in zip(out, done):
            r["ticket"], r["user_tag"], r["n_records"] = t, self.running.pop(t)[1], 2
            if not self.cfg.flags & B.CF_AUTO_RELEASE:
                self.polled.add(t)                            # else released by the poll
        return out

    def _held(self, t):
        assert t in self.polled, f"ticket {t} read after release or before completion"

    def records(self, ctx, t, n):
        self._held(t)
        return np.zeros(n, B.VIOLATION_DTYPE)

    def bitmap(self, ctx, t):
        self._held(t)
        return np.full(65536, t % 251, np.uint8)

    def release(self, ctx, t):
        self._held(t)
        self.polled.discard(t)


@pytest.fixture
def fake(monkeypatch):
    def make(slots, service_s, auto_release=False):
        f = FakeEngine(slots, service_s, auto_release)
        monkeypatch.setattr(B, "cufz_submit_inputs", f.submit)
        monkeypatch.setattr(B, "cufz_poll_results", f.poll)
        monkeypatch.setattr(B, "cufz_get_records", f.records)
        monkeypatch.setattr(B, "cufz_get_bitmap", f.bitmap)
        monkeypatch.setattr(B, "cufz_release", f.release)
        return f
    return make


def inputs(n):
    x = gen.c1_inputs(n, seed=5)
    x["user_tag"] = np.arange(100, 100 + n)
    return x


def test_every_input_once_in_input_order(fake):
    f = fake(slots=3, service_s=0.002)
    x = inputs(20)
    arrivals = np.linspace(0.0, 0.01, 20)
    res, lat, kept, wall = serve.serve_open_loop(f, x, arrivals, keep={4, 11})
    assert f.submitted == list(range(100, 120))              # each once, in arrival order
    assert f.busy_returns > 0                               # the slot limit was hit
    assert res["user_tag"].tolist() == list(range(100, 120))  # results in input order
    assert np.all(lat >= 0.002 - 1e-4) and not np.isnan(lat).any()
    assert sorted(kept) == [4, 11]
    for i, (recs, bm) in kept.items():
        assert len(recs) == 2 and bm[0] == int(res[i]["ticket"]) % 251
    assert not f.running and not f.polled                   # everything released
    assert wall >= arrivals[-1]


def test_latency_counts_from_arrival(fake):
    """Ten inputs due at once on a one-slot engine: the k-th waits for the k
    before it, and its latency says so (about (k + 1) service times)."""
    f = fake(slots=1, service_s=0.004)
    res, lat, _, _ = serve.serve_open_loop(f, inputs(10), np.zeros(10))
    assert np.all(np.diff(lat) > 0)
    assert lat[-1] >= 10 * 0.004 - 1e-3


def test_stuck_engine_times_out(fake):
    f = fake(slots=4, service_s=None)
    t0 = time.perf_counter()
    with pytest.raises(B.CufzError) as ei:
        serve.serve_open_loop(f, inputs(3), np.zeros(3), timeout_s=0.2)
    assert ei.value.status == B.E_TIMEOUT and time.perf_counter() - t0 < 5


def test_auto_release_context(fake):
    """A context that releases results when they are polled: every input
    completes, in input order, and the loop releases nothing itself (a
    release of an auto-released ticket would be a read after release)."""
    f = fake(slots=4, service_s=0.001, auto_release=True)
    x = inputs(40)
    res, lat, kept, _ = serve.serve_open_loop(f, x, np.linspace(0.0, 0.02, 40))
    assert res["user_tag"].tolist() == list(range(100, 140)) and not kept
    assert not np.isnan(lat).any() and not f.running and not f.polled
