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
    soon as they are polled (by the context itself when it was created with
    CUFZ_CF_AUTO_RELEASE and nothing is kept).  Returns (results in input
    order, latency in seconds per input, {index: (records, bitmap)} for
    `keep`, wall seconds).

    The per-result host work is done on whole poll batches: tickets are
    handed out in submission order, one per input, so an input's index is
    its ticket minus the first ticket of the stream."""
    inputs = np.ascontiguousarray(inputs, dtype=INPUT_DTYPE)
    n = len(inputs)
    keep = keep or set()
    cfg = getattr(engine, "cfg", None)
    auto = bool(getattr(cfg, "flags", 0) & B.CF_AUTO_RELEASE) and not keep
    results = np.zeros(n, B.RESULT_DTYPE)
    latency = np.full(n, np.nan)
    kept = {}
    t_first = None
    pos = 0
    done = 0
    t0 = time.perf_counter()
    deadline = t0 + timeout_s
    while done < n:
        now = time.perf_counter() - t0
        due = int(np.searchsorted(arrivals_s, now, side="right"))
        if pos < due:
            st, acc, first = B.cufz_submit_inputs(engine.ctx, inputs[pos:due])
            if acc:
                if t_first is None:
                    t_first = first - pos
                elif first - pos != t_first:
                    raise B.CufzError(B.E_INVALID_ARG, "serve_open_loop: tickets out of order")
            pos += acc
        out = B.cufz_poll_results(engine.ctx, poll_max, 0)
        if len(out):
            t_done = time.perf_counter() - t0
            idx = out["ticket"].astype(np.int64) - t_first
            results[idx] = out
            latency[idx] = t_done - arrivals_s[idx]
            if not auto:
                for t, i in zip(out["ticket"].tolist(), idx.tolist()):
                    if i in keep:
                        recs = B.cufz_get_records(engine.ctx, t, int(results[i]["n_records"]))
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
