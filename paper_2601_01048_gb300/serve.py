"""Open-loop serving driver over one engine context.

Fuzz inputs arrive at given times (a Poisson process in the benchmark); each
is submitted as soon as it is due and a slot is free, so inputs that arrive
while earlier ones are still on the GPU join the device queue of the next
batch (batches of successive submits overlap on the device through the
context's pipeline lanes).  Latency is measured from the scheduled arrival,
not from the submit, so a backlog shows up in the percentiles instead of
being hidden (no coordinated omission).
"""
from __future__ import annotations

import time

import numpy as np

from . import binding as B
from .gen import INPUT_DTYPE


def serve_open_loop(engine: "B.Engine", inputs: np.ndarray, arrivals_s: np.ndarray,
                    keep: set | None = None, timeout_s: float = 300.0, poll_max: int = 8192):
    """Runs `inputs` (arrival times `arrivals_s`, seconds from start, sorted)
    through `engine`.  Results of inputs whose index is in `keep` are held
    (records and bitmaps fetched, then released); others are released as
    soon as they are polled.  Returns (results in input order, latency in
    seconds per input, {index: (records, bitmap)} for `keep`, wall seconds)."""
    inputs = np.ascontiguousarray(inputs, dtype=INPUT_DTYPE)
    n = len(inputs)
    keep = keep or set()
    results = np.zeros(n, B.RESULT_DTYPE)
    latency = np.full(n, np.nan)
    kept = {}
    ticket_idx: dict[int, int] = {}
    pos = 0
    done = 0
    t0 = time.perf_counter()
    deadline = t0 + timeout_s
    while done < n:
        now = time.perf_counter() - t0
        due = int(np.searchsorted(arrivals_s, now, side="right"))
        if pos < due:
            st, acc, first = B.cufz_submit_inputs(engine.ctx, inputs[pos:due])
            for k in range(acc):
                ticket_idx[first + k] = pos + k
            pos += acc
        out = B.cufz_poll_results(engine.ctx, poll_max, 0)
        if len(out):
            t_done = time.perf_counter() - t0
            for r in out:
                t = int(r["ticket"])
                i = ticket_idx.pop(t)
                results[i] = r
                latency[i] = t_done - arrivals_s[i]
                if i in keep:
                    recs = B.cufz_get_records(engine.ctx, t, int(r["n_records"]))
                    bm = B.cufz_get_bitmap(engine.ctx, t)
                    kept[i] = (recs, bm)
                B.cufz_release(engine.ctx, t)
            done += len(out)
        elif pos >= due:
            # nothing to submit or collect: wait a little (next arrival or 50 us)
            nxt = arrivals_s[pos] - (time.perf_counter() - t0) if pos < n else 5e-5
            time.sleep(min(max(nxt, 0.0), 5e-5))
        if time.perf_counter() > deadline:
            raise B.CufzError(B.E_TIMEOUT, "serve_open_loop")
    return results, latency, kept, time.perf_counter() - t0
