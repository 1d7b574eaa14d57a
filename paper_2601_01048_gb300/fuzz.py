"""Coverage-guided fuzzing campaign over one engine context.

The paper drives its translated kernels with AFL++ (Sec. 4, Fig. 2): a
mutated input is kept when it reaches coverage the campaign has not seen
(Sec. 2.1, AFL's bucketed edge bitmap), and inputs that trip the memory
checker are the bug reports.  Two forms share one set of rules:

  - Campaign keeps the queue, the corpus and the bug buckets on the host and
    runs each round's children as one device batch through the engine;
  - DeviceCampaign keeps them in device memory and runs every step of a
    round in kernels (cufz_campaign_*: selection, mutation, batch building,
    the engine, filing), a CUDA graph per round, with no host round trip.

The rules of a round:

  - it takes `batch` parents from the corpus, favoured entries first (those
    that brought new coverage and were not picked since), least picked
    first, then the lowest index, round robin;
  - child j of round r is a copy of its parent mutated from its own
    SplitMix64 stream (bit flips, +-1..35, boundary values on the scalar
    arguments and buffer lengths: cufz_mutate_children), so the children of
    a round can be mutated in parallel;
  - a child whose result carries CUFZ_FL_NEW_COV (a bucket bit the union
    lacked when the round started) joins the corpus as a favoured entry, in
    child order, while the corpus has room (corpus_cap);
  - a violating child is filed under (program, site, class) of its first
    stored violation record (least block, thread and ordinal), so repeated
    reports of one bug collapse into one bucket; the bucket keeps its first
    child (round, index) and counts its hits;
  - a child that hit the back-edge budget (CUFZ_FL_BUDGET, the analog of the
    paper's hang timeout, Sec. 7.1) is a hang; as in AFL, a hang is unique,
    and kept, when it also reached new coverage;
  - the round ends with a new coverage epoch, so the next round's NEW_COV is
    measured against everything seen so far.

A campaign starts by running its seed corpus once (AFL's dry run), so the
union is at every moment the OR of the corpus's bitmaps: every input that
added a bucket bit is in the corpus (while corpus_cap is not reached).
`checkpoint` writes the corpus, the bug buckets, the unique hangs and the
counters to one .npz file; `resume` reads it and runs the corpus once, which
rebuilds the device union, after which the campaign continues exactly as it
would have without the interruption.  `stats()` reports the columns of the
paper's Table 2: executions and executions per second, unique crashes (bug
buckets), unique hangs, queue cycles and the corpus size.
"""
from __future__ import annotations

import contextlib
import dataclasses
import time

import numpy as np

from . import binding as B
from .gen import INPUT_DTYPE


@dataclasses.dataclass
class RoundStats:
    executed: int
    new_coverage: int
    violating: int
    new_buckets: int
    corpus_size: int
    hangs: int = 0
    new_hangs: int = 0
    seconds: float = dataclasses.field(default=0.0, compare=False)


NO_SITE, NO_CLS = 0xFFFF, 0xFF  # bucket key parts of a violation with no stored record


def first_record(recs):
    """The stored violation record of least (block, thread, ordinal), or
    None."""
    if recs is None or not len(recs):
        return None
    k = np.lexsort((recs["ordinal"], recs["thread_lin"], recs["block_lin"]))
    return recs[k[0]]


class EngineExecutor:
    """The campaign's view of an engine context (binding.Engine): run a batch
    and report each input's result and first violation record; advance the
    coverage epoch; read the union."""

    def __init__(self, engine):
        self.engine = engine

    def run(self, inputs: np.ndarray):
        res, recs, _ = self.engine.run(inputs, records=True, bitmaps=False)
        return res, [first_record(r) for r in recs]

    def new_epoch(self) -> None:
        self.engine.new_epoch()

    def union(self) -> np.ndarray:
        return self.engine.union()


class Campaign:
    """A campaign over programs already loaded in the executor's context.
    n_bufs[p] is program p's buffer count (the mutator touches only the
    lengths of buffers the program has)."""

    NEW_COV = 4   # CUFZ_FL_NEW_COV
    BUDGET = 1    # CUFZ_FL_BUDGET
    VIOLATION = 1  # CUFZ_ST_VIOLATION

    def __init__(self, executor, n_bufs: list[int], seeds: np.ndarray, seed: int = 0xF022,
                 batch: int = 1024, corpus_cap: int = 16384, hang_cap: int = 4096):
        self.ex = executor
        self.n_bufs = list(n_bufs)
        self.batch = int(batch)
        self.seed = int(seed) & (2**64 - 1)
        self.corpus_cap = int(corpus_cap)
        self.hang_cap = int(hang_cap)
        self.corpus = np.ascontiguousarray(seeds, dtype=INPUT_DTYPE).copy()
        if not len(self.corpus):
            raise ValueError("a campaign needs at least one seed input")
        if len(self.corpus) > self.corpus_cap:
            raise ValueError("more seeds than corpus_cap")
        self.favoured = np.ones(len(self.corpus), dtype=bool)
        self.picks = np.zeros(len(self.corpus), dtype=np.int64)
        # (program, site, class) -> {"input", "hits", "round", "child"}
        self.buckets: dict[tuple[int, int, int], dict] = {}
        self.hangs: list[dict] = []   # unique hangs: {"input", "round"}
        self.n_hangs = 0              # executions that hit the budget
        self.n_violating = 0
        self.n_new_coverage = 0
        self.corpus_dropped = 0
        self.hangs_dropped = 0
        self.rounds = 0
        self.executed = 0
        self.seconds = 0.0
        # the dry run: the seeds' coverage becomes the union's starting point
        self.ex.run(self.corpus)
        self.ex.new_epoch()

    # ------------------------------------------------------------ rounds
    def _parents(self) -> np.ndarray:
        """Indices of this round's parents: favoured entries (least picked
        first), then the rest of the corpus round-robin by pick count."""
        n = len(self.corpus)
        order = np.lexsort((np.arange(n), self.picks, ~self.favoured))
        reps = -(-self.batch // n)
        return np.tile(order, reps)[: self.batch]

    def run_round(self) -> RoundStats:
        t0 = time.perf_counter()
        parents = self._parents()
        kids = self.corpus[parents].copy()
        # child j's own mutation stream (the device campaign's draws)
        B.cufz_mutate_children(kids, self.n_bufs, self.seed, self.rounds)
        np.add.at(self.picks, parents, 1)
        self.favoured[parents] = False
        res, first = self.ex.run(kids)
        self.executed += len(kids)
        new_cov = (res["flags"] & self.NEW_COV) != 0
        violating = res["status"] == self.VIOLATION
        new_buckets = 0
        for k in np.flatnonzero(violating):
            rec = first[k]
            key = (int(kids[k]["program_id"]),
                   int(rec["site"]) if rec is not None else NO_SITE,
                   int(rec["cls"]) if rec is not None else NO_CLS)
            b = self.buckets.get(key)
            if b is None:
                self.buckets[key] = {"input": kids[k].copy(), "hits": 1, "round": self.rounds,
                                     "child": int(k)}
                new_buckets += 1
            else:
                b["hits"] += 1
        hang = (res["flags"] & self.BUDGET) != 0
        new_hang = hang & new_cov
        for k in np.flatnonzero(new_hang):
            if len(self.hangs) < self.hang_cap:
                self.hangs.append({"input": kids[k].copy(), "round": self.rounds})
            else:
                self.hangs_dropped += 1
        self.n_hangs += int(hang.sum())
        self.n_violating += int(violating.sum())
        self.n_new_coverage += int(new_cov.sum())
        if new_cov.any():
            add = kids[new_cov]
            room = max(self.corpus_cap - len(self.corpus), 0)
            self.corpus_dropped += max(len(add) - room, 0)
            add = add[:room]
            self.corpus = np.concatenate([self.corpus, add])
            self.favoured = np.concatenate([self.favoured, np.ones(len(add), bool)])
            self.picks = np.concatenate([self.picks, np.zeros(len(add), np.int64)])
        self.ex.new_epoch()
        self.rounds += 1
        dt = time.perf_counter() - t0
        self.seconds += dt
        return RoundStats(len(kids), int(new_cov.sum()), int(violating.sum()), new_buckets,
                          len(self.corpus), int(hang.sum()), int(new_hang.sum()), dt)

    def stats(self) -> dict:
        """The campaign so far in the terms of the paper's Table 2."""
        return {"execs_done": self.executed,
                "execs_per_sec": self.executed / self.seconds if self.seconds > 0 else 0.0,
                "unique_crashes": len(self.buckets),
                "unique_hangs": len(self.hangs),
                "hang_execs": self.n_hangs,
                "cycles_done": int(self.picks.min()) if len(self.picks) else 0,
                "corpus_count": len(self.corpus),
                "corpus_dropped": self.corpus_dropped,
                "rounds": self.rounds}

    # ------------------------------------------------------ checkpoints
    def _state(self) -> dict:
        keys = sorted(self.buckets)
        return {"corpus": self.corpus, "favoured": self.favoured, "picks": self.picks,
                "bucket_keys": np.array(keys, dtype=np.int64).reshape(-1, 3),
                "bucket_inputs": np.array([self.buckets[k]["input"] for k in keys], dtype=INPUT_DTYPE),
                "bucket_hits": np.array([self.buckets[k]["hits"] for k in keys], dtype=np.int64),
                "bucket_rounds": np.array([self.buckets[k]["round"] for k in keys], dtype=np.int64),
                "bucket_children": np.array([self.buckets[k]["child"] for k in keys], dtype=np.int64),
                "hang_inputs": np.array([h["input"] for h in self.hangs], dtype=INPUT_DTYPE),
                "hang_rounds": np.array([h["round"] for h in self.hangs], dtype=np.int64),
                "counters": np.array([self.seed, self.rounds, self.executed, self.batch,
                                      self.n_hangs, self.n_violating, self.n_new_coverage,
                                      self.corpus_dropped, self.hangs_dropped, self.corpus_cap,
                                      self.hang_cap], dtype=np.uint64),
                "seconds": np.array([self.seconds], dtype=np.float64),
                "n_bufs": np.array(self.n_bufs, dtype=np.int64)}

    def checkpoint(self, path: str) -> None:
        np.savez(path, **self._state())

    @classmethod
    def resume(cls, path: str, executor) -> "Campaign":
        """A campaign restored from `checkpoint`; constructing it runs the
        saved corpus once, which rebuilds the executor's union."""
        z = np.load(path if path.endswith(".npz") else path + ".npz")
        k = [int(v) for v in z["counters"]]
        c = cls(executor, [int(v) for v in z["n_bufs"]], z["corpus"], seed=k[0], batch=k[3],
                corpus_cap=k[9], hang_cap=k[10])
        c.favoured = z["favoured"].astype(bool)
        c.picks = z["picks"].astype(np.int64)
        c.rounds, c.executed, c.n_hangs, c.n_violating, c.n_new_coverage = k[1], k[2], k[4], k[5], k[6]
        c.corpus_dropped, c.hangs_dropped = k[7], k[8]
        c.seconds = float(z["seconds"][0])
        c.hangs = [{"input": inp.copy(), "round": rnd}
                   for inp, rnd in zip(z["hang_inputs"], z["hang_rounds"].tolist())]
        for key, inp, hits, rnd, ch in zip(z["bucket_keys"].tolist(), z["bucket_inputs"],
                                           z["bucket_hits"].tolist(), z["bucket_rounds"].tolist(),
                                           z["bucket_children"].tolist()):
            c.buckets[tuple(key)] = {"input": inp.copy(), "hits": hits, "round": rnd, "child": ch}
        return c


class DeviceCampaign:
    """The campaign with its queue, corpus, buckets and hangs in device
    memory (a torch tensor on the engine's device) and every step of a round
    in kernels: run(k) enqueues k rounds, one CUDA graph launch each, and
    returns.  The engine must be compiled-path (CF_JIT); while the campaign
    lives, its programs stay as they are."""

    def __init__(self, engine, seeds: np.ndarray, seed: int = 0xF022, batch: int = 1024,
                 corpus_cap: int = 16384, bucket_cap: int = 4096, hang_cap: int = 4096,
                 item_threads: int = 0, max_items: int = 0, n_bufs: list[int] | None = None):
        """n_bufs (each program's buffer count) is kept for checkpoints, which
        the host campaign can then resume."""
        import torch

        self.engine = engine
        self.n_bufs = list(n_bufs) if n_bufs is not None else None
        self.cfg = B.cufz_campaign_config(batch=batch, corpus_cap=corpus_cap, bucket_cap=bucket_cap,
                                          hang_cap=hang_cap, item_threads=item_threads,
                                          max_items=max_items, seed=int(seed) & (2**64 - 1))
        n = B.cufz_campaign_bytes(self.cfg)
        if not n:
            raise B.CufzError(B.E_INVALID_ARG, "DeviceCampaign")
        self.mem = torch.empty(n, dtype=torch.uint8, device=f"cuda:{engine.device}")
        self.camp = B.cufz_campaign_create(engine.ctx, self.cfg, self.mem.data_ptr(), n, seeds)
        self.seconds = 0.0
        self._t = None

    def run(self, rounds: int = 1) -> None:
        if self._t is None:
            self._t = time.perf_counter()
        B.cufz_campaign_run(self.camp, rounds)

    def sync(self) -> None:
        B.cufz_campaign_sync(self.camp)
        if self._t is not None:
            self.seconds += time.perf_counter() - self._t
            self._t = None

    def counters(self) -> B.cufz_campaign_stats:
        self.sync()
        return B.cufz_campaign_get_stats(self.camp)

    def stats(self) -> dict:
        s = self.counters()
        return {"execs_done": int(s.executed),
                "execs_per_sec": s.executed / self.seconds if self.seconds > 0 else 0.0,
                "unique_crashes": int(s.buckets), "unique_hangs": int(s.hangs),
                "hang_execs": int(s.hang_execs), "cycles_done": int(s.cycles_done),
                "corpus_count": int(s.corpus), "corpus_dropped": int(s.corpus_dropped),
                "rounds": int(s.rounds)}

    def corpus(self):
        """(inputs, favoured, picks) in entry order."""
        self.sync()
        return B.cufz_campaign_corpus(self.camp)

    def buckets(self) -> dict:
        """{(program, site, class): {"input", "hits", "round", "child"}}."""
        self.sync()
        out = {}
        for b in B.cufz_campaign_buckets(self.camp):
            k = int(b["key"])
            key = (k >> 32, (k >> 8) & 0xFFFF, k & 0xFF)
            f = int(b["first"])
            out[key] = {"input": b["input"].copy(), "hits": int(b["hits"]), "round": f >> 32,
                        "child": f & 0xFFFFFFFF}
        return out

    def hangs(self) -> list[dict]:
        self.sync()
        inp, rounds = B.cufz_campaign_hangs(self.camp)
        return [{"input": x.copy(), "round": int(r)} for x, r in zip(inp, rounds)]

    def checkpoint(self, path: str) -> None:
        """The same .npz layout as Campaign.checkpoint (either resumes the
        other's file)."""
        s = self.counters()
        inp, fav, picks = B.cufz_campaign_corpus(self.camp)
        bk = self.buckets()
        hg = self.hangs()
        keys = sorted(bk)
        n_bufs = self.n_bufs
        np.savez(path, corpus=inp, favoured=fav, picks=picks.astype(np.int64),
                 bucket_keys=np.array(keys, dtype=np.int64).reshape(-1, 3),
                 bucket_inputs=np.array([bk[k]["input"] for k in keys], dtype=INPUT_DTYPE),
                 bucket_hits=np.array([bk[k]["hits"] for k in keys], dtype=np.int64),
                 bucket_rounds=np.array([bk[k]["round"] for k in keys], dtype=np.int64),
                 bucket_children=np.array([bk[k]["child"] for k in keys], dtype=np.int64),
                 hang_inputs=np.array([h["input"] for h in hg], dtype=INPUT_DTYPE),
                 hang_rounds=np.array([h["round"] for h in hg], dtype=np.int64),
                 counters=np.array([self.cfg.seed, s.rounds, s.executed, self.cfg.batch,
                                    s.hang_execs, s.violating, s.new_coverage, s.corpus_dropped,
                                    s.hangs_dropped, self.cfg.corpus_cap, self.cfg.hang_cap],
                                   dtype=np.uint64),
                 seconds=np.array([self.seconds], dtype=np.float64),
                 n_bufs=np.array(n_bufs if n_bufs is not None else [], dtype=np.int64))

    @classmethod
    def resume(cls, path: str, engine, bucket_cap: int = 4096, item_threads: int = 0,
               max_items: int = 0) -> "DeviceCampaign":
        """A campaign restored from a checkpoint: created with the saved
        corpus as its seeds (the dry run rebuilds the union), then given the
        saved favoured flags, pick counts, buckets, hangs and counters."""
        z = np.load(path if path.endswith(".npz") else path + ".npz")
        k = [int(v) for v in z["counters"]]
        c = cls(engine, z["corpus"], seed=k[0], batch=k[3], corpus_cap=k[9],
                bucket_cap=bucket_cap, hang_cap=k[10], item_threads=item_threads,
                max_items=max_items)
        keys = z["bucket_keys"].reshape(-1, 3)
        bk = np.zeros(len(keys), B.BUCKET_DTYPE)
        for i, (p, site, cls_) in enumerate(keys.tolist()):
            bk[i]["key"] = (p << 32) | (site << 8) | cls_
            bk[i]["first"] = (int(z["bucket_rounds"][i]) << 32) | int(z["bucket_children"][i])
            bk[i]["hits"] = int(z["bucket_hits"][i])
            bk[i]["input"] = z["bucket_inputs"][i]
        cnt = B.cufz_campaign_stats(rounds=k[1], executed=k[2], violating=k[5], hang_execs=k[4],
                                    new_coverage=k[6], corpus_dropped=k[7], hangs_dropped=k[8])
        B.cufz_campaign_restore(c.camp, z["favoured"], z["picks"], bk, z["hang_inputs"],
                                z["hang_rounds"], cnt)
        c.seconds = float(z["seconds"][0])
        c.n_bufs = [int(v) for v in z["n_bufs"]] if len(z["n_bufs"]) else None
        return c

    def close(self) -> None:
        if getattr(self, "camp", None):
            B.cufz_campaign_destroy(self.camp)
            self.camp = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ command line
@contextlib.contextmanager
def _engine_executor(programs: list[bytes], batch: int):
    """An engine context holding `programs`, for a campaign of `batch`
    inputs per round (compiled path; per-input bitmaps are not kept, the
    device union is)."""
    with B.Engine(max_slots=batch, record_cap=64, flags=B.CF_JIT) as engine:
        for p in programs:
            engine.load(p)
        yield EngineExecutor(engine)


def main(argv=None, executor_factory=None) -> int:
    """python -m paper_2601_01048_gb300.fuzz: a campaign over program files
    (--program, repeatable; default the serving workload's 64 programs) from
    a seed corpus of their shapes, printing stats() as one JSON line every
    --report rounds and writing --checkpoint then; --resume continues a
    saved campaign."""
    import argparse
    import json

    from . import bytecode as bc
    from .gen import c5_corpus, c5_programs

    ap = argparse.ArgumentParser(prog="python -m paper_2601_01048_gb300.fuzz")
    ap.add_argument("--program", action="append", default=[], help="program file (repeatable)")
    ap.add_argument("--rounds", type=int, default=100)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--seed", type=lambda s: int(s, 0), default=0xF022)
    ap.add_argument("--report", type=int, default=10, help="rounds between stats lines")
    ap.add_argument("--checkpoint", default=None)
    ap.add_argument("--resume", default=None)
    ap.add_argument("--device", action="store_true",
                    help="queue, corpus and rounds on the device (DeviceCampaign)")
    args = ap.parse_args(argv)
    progs = [open(p, "rb").read() for p in args.program] or c5_programs()
    n_bufs = [bc.decode_header(p)["n_bufs"] for p in progs]
    make = executor_factory or _engine_executor
    with make(progs, args.batch) as ex:
        if args.device:
            if args.resume:
                c = DeviceCampaign.resume(args.resume, ex.engine)
            else:
                c = DeviceCampaign(ex.engine, c5_corpus(progs), seed=args.seed, batch=args.batch,
                                   n_bufs=n_bufs)
            c.n_bufs = n_bufs
            done = 0
            try:
                while done < args.rounds:
                    k = min(max(args.report, 1), args.rounds - done)
                    c.run(k)
                    done += k
                    print(json.dumps(c.stats()), flush=True)
                    if args.checkpoint:
                        c.checkpoint(args.checkpoint)
            finally:
                c.close()
            return 0
        if args.resume:
            c = Campaign.resume(args.resume, ex)
        else:
            c = Campaign(ex, n_bufs, c5_corpus(progs), seed=args.seed, batch=args.batch)
        for r in range(args.rounds):
            c.run_round()
            if (r + 1) % max(args.report, 1) == 0 or r + 1 == args.rounds:
                print(json.dumps(c.stats()), flush=True)
                if args.checkpoint:
                    c.checkpoint(args.checkpoint)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
