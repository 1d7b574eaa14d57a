"""Coverage-guided fuzzing campaign over one engine context.

The paper drives its translated kernels with AFL++ (Sec. 4, Fig. 2): a
mutated input is kept when it reaches coverage the campaign has not seen
(Sec. 2.1, AFL's bucketed edge bitmap), and inputs that trip the memory
checker are the bug reports.  Here the queue, the corpus and the bug buckets
live on the host, and every execution (checks, coverage, the union of
bitmaps) runs on the device through the engine:

  - each round takes `batch` parents from the corpus, favoured entries first
    (those that brought new coverage and were picked least often), mutates
    copies of them (bit flips, +-1..35, boundary values on the scalar
    arguments and buffer lengths: cufz_mutate_inputs, the library's native
    form of gen.Mutator) and runs them as one batch;
  - an input whose result carries CUFZ_FL_NEW_COV (a bucket bit the union
    lacked when the round started) joins the corpus as a favoured entry;
  - a violating input is filed under (program, first record's site, class),
    so repeated reports of one bug collapse into one bucket;
  - an input that hit the back-edge budget (CUFZ_FL_BUDGET, the analog of
    the paper's hang timeout, Sec. 7.1) is a hang; as in AFL, a hang is
    unique, and kept, when it also reached new coverage;
  - the round ends with cufz_new_epoch, so the next round's NEW_COV is
    measured against everything seen so far.

A campaign starts by running its seed corpus once (AFL's dry run), so the
union is at every moment the OR of the corpus's bitmaps: every input that
added a bucket bit is in the corpus.  `checkpoint` writes the corpus, the bug
buckets, the unique hangs and the random state to one .npz file;
`Campaign.resume` reads it and runs the corpus once, which rebuilds the
device union, after which the campaign continues exactly as it would have
without the interruption.  `stats()` reports the columns of the paper's
Table 2: executions and executions per second, unique crashes (bug
buckets), unique hangs, queue cycles and the corpus size.
"""
from __future__ import annotations

import contextlib
import dataclasses
import time

import numpy as np

from . import binding as B
from .gen import INPUT_DTYPE, Mutator, SplitMix64


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


class EngineExecutor:
    """The campaign's view of an engine context (binding.Engine): run a batch
    and report each input's result and first violation record; advance the
    coverage epoch; read the union."""

    def __init__(self, engine):
        self.engine = engine

    def run(self, inputs: np.ndarray):
        res, recs, _ = self.engine.run(inputs, records=True, bitmaps=False)
        first = [r[0] if r is not None and len(r) else None for r in recs]
        return res, first

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
                 batch: int = 1024):
        self.ex = executor
        self.n_bufs = list(n_bufs)
        self.batch = int(batch)
        self.rng = SplitMix64(seed)
        self.mutator = Mutator(self.rng.next())
        self.corpus = np.ascontiguousarray(seeds, dtype=INPUT_DTYPE).copy()
        if not len(self.corpus):
            raise ValueError("a campaign needs at least one seed input")
        self.favoured = np.ones(len(self.corpus), dtype=bool)
        self.picks = np.zeros(len(self.corpus), dtype=np.int64)
        self.buckets: dict[tuple[int, int, int], dict] = {}
        self.hangs: list[dict] = []   # unique hangs: {"input", "round"}
        self.n_hangs = 0              # executions that hit the budget
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
        # the library's mutator: the same draws as gen.Mutator, natively
        self.mutator.rng.state = B.cufz_mutate_inputs(kids, self.n_bufs, self.mutator.rng.state)
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
                   int(rec["site"]) if rec is not None else -1,
                   int(rec["cls"]) if rec is not None else -1)
            b = self.buckets.get(key)
            if b is None:
                self.buckets[key] = {"input": kids[k].copy(), "hits": 1, "round": self.rounds}
                new_buckets += 1
            else:
                b["hits"] += 1
        hang = (res["flags"] & self.BUDGET) != 0
        new_hang = hang & new_cov
        for k in np.flatnonzero(new_hang):
            self.hangs.append({"input": kids[k].copy(), "round": self.rounds})
        self.n_hangs += int(hang.sum())
        if new_cov.any():
            self.corpus = np.concatenate([self.corpus, kids[new_cov]])
            self.favoured = np.concatenate([self.favoured, np.ones(int(new_cov.sum()), bool)])
            self.picks = np.concatenate([self.picks, np.zeros(int(new_cov.sum()), np.int64)])
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
                "rounds": self.rounds}

    # ------------------------------------------------------ checkpoints
    def checkpoint(self, path: str) -> None:
        keys = np.array(sorted(self.buckets), dtype=np.int64).reshape(-1, 3)
        np.savez(path, corpus=self.corpus, favoured=self.favoured, picks=self.picks,
                 bucket_keys=keys,
                 bucket_inputs=np.array([self.buckets[tuple(k)]["input"] for k in keys.tolist()],
                                        dtype=INPUT_DTYPE),
                 bucket_hits=np.array([self.buckets[tuple(k)]["hits"] for k in keys.tolist()],
                                      dtype=np.int64),
                 bucket_rounds=np.array([self.buckets[tuple(k)]["round"] for k in keys.tolist()],
                                        dtype=np.int64),
                 hang_inputs=np.array([h["input"] for h in self.hangs], dtype=INPUT_DTYPE),
                 hang_rounds=np.array([h["round"] for h in self.hangs], dtype=np.int64),
                 state=np.array([self.rng.state, self.mutator.rng.state, self.rounds,
                                 self.executed, self.batch, self.n_hangs], dtype=np.uint64),
                 seconds=np.array([self.seconds], dtype=np.float64),
                 n_bufs=np.array(self.n_bufs, dtype=np.int64))

    @classmethod
    def resume(cls, path: str, executor) -> "Campaign":
        """A campaign restored from `checkpoint`; constructing it runs the
        saved corpus once, which rebuilds the executor's union."""
        z = np.load(path if path.endswith(".npz") else path + ".npz")
        state = [int(v) for v in z["state"]]
        c = cls(executor, [int(v) for v in z["n_bufs"]], z["corpus"], batch=state[4])
        c.favoured = z["favoured"].astype(bool)
        c.picks = z["picks"].astype(np.int64)
        c.rng.state, c.mutator.rng.state = state[0], state[1]
        c.rounds, c.executed, c.n_hangs = state[2], state[3], state[5]
        c.seconds = float(z["seconds"][0])
        c.hangs = [{"input": inp.copy(), "round": rnd}
                   for inp, rnd in zip(z["hang_inputs"], z["hang_rounds"].tolist())]
        for k, inp, hits, rnd in zip(z["bucket_keys"].tolist(), z["bucket_inputs"],
                                     z["bucket_hits"].tolist(), z["bucket_rounds"].tolist()):
            c.buckets[tuple(k)] = {"input": inp.copy(), "hits": hits, "round": rnd}
        return c


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
    args = ap.parse_args(argv)
    progs = [open(p, "rb").read() for p in args.program] or c5_programs()
    make = executor_factory or _engine_executor
    with make(progs, args.batch) as ex:
        if args.resume:
            c = Campaign.resume(args.resume, ex)
        else:
            c = Campaign(ex, [bc.decode_header(p)["n_bufs"] for p in progs], c5_corpus(progs),
                         seed=args.seed, batch=args.batch)
        for r in range(args.rounds):
            c.run_round()
            if (r + 1) % max(args.report, 1) == 0 or r + 1 == args.rounds:
                print(json.dumps(c.stats()), flush=True)
                if args.checkpoint:
                    c.checkpoint(args.checkpoint)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
