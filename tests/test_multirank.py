"""The benchmark's multi-rank plumbing (one replica per rank, barrier,
max/sum over ranks, rank 0 reports) on two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    r, w, local, pg = bench.dist_init(None)
    assert (r, w) == (rank, world) and pg is not None
    bench.barrier(pg)
    dev = torch.device("cpu")
    mx = bench.allreduce_max(pg, float(rank + 1) * 10.0, dev)
    sm = bench.allreduce_sum(pg, float(rank + 1), dev)
    out.put((rank, mx, sm))
    pg.destroy_process_group()


def test_two_rank_max_and_sum():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 20.0, 3.0), (1, 20.0, 3.0)]


def _reference_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import contextlib
    import io
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    class A:
        steps, warmup, cpu_seconds, workload = 1, 0, 0.2, "c1"

    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(A, rank, world)
    out.put((rank, buf.getvalue()))


def test_reference_arm_reports_on_rank0_only():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_reference_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import json
    line = json.loads(got[0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2
    assert got[1].strip() == ""
