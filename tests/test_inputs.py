"""The seeded workloads match the input recipe the design notes state
(shapes, ranges, length distributions, program sizes), and are
deterministic in their seeds."""
import numpy as np

from paper_2601_01048_gb300 import bytecode as bc
from paper_2601_01048_gb300 import gen


def threads(x):
    return x["grid"].astype(np.int64).prod(axis=1) * x["block"].astype(np.int64).prod(axis=1)


def test_c1_recipe():
    x = gen.c1_inputs(1000)
    assert len(x) == 1000 and (x["program_id"] == 0).all()
    assert (x["grid"] == (64, 1, 1)).all() and (x["block"] == (128, 1, 1)).all()
    a0, a1 = x["args"][:, 0].astype(np.int64), x["args"][:, 1].astype(np.int64)
    assert a0.min() >= -4 and a0.max() <= 4 and a1.min() >= 0 and a1.max() <= 8192
    lens = x["buf_len"][:, :4].astype(np.int64)
    assert (lens % 4 == 0).all() and (x["buf_len"][:, 4:] == 0).all()
    e = lens // 4
    assert e.min() >= 0 and e.max() <= 8192
    off_by_one = (e == np.maximum(a1 - 1, 0)[:, None]) & (a1[:, None] > 0)
    assert 0.07 < off_by_one.mean() < 0.13                      # p = 0.1 per buffer


def test_c2_recipe():
    progs = gen.c2_programs()
    assert len(progs) == 32
    for p in progs:
        h = bc.decode_header(p)
        n_shared = bin(h["shared_mask"]).count("1")
        assert 20 <= h["n_ops"] <= 200 and 1 <= n_shared <= 3 and 2 <= h["n_bufs"] - n_shared <= 6
        loops = [o for o in bc.ops_of(p) if o[0] == bc.LOOP]
        assert len(loops) <= 2 and all(o[4] <= 64 for o in loops)
    x = gen.c2_inputs(progs)
    assert len(x) == 32 * 256 and (np.bincount(x["program_id"]) == 256).all()
    assert (x["block"] == (16, 16, 1)).all() and (x["grid"][:, 2] == 1).all()
    assert x["grid"][:, :2].min() >= 1 and x["grid"][:, :2].max() <= 256
    for k in range(0, len(x), 97):
        h = bc.decode_header(progs[int(x[k]["program_id"])])
        wmax = [1] * h["n_bufs"]
        for opc, _d, _a, b, imm in bc.ops_of(progs[int(x[k]["program_id"])]):
            if opc in (bc.LD, bc.ST):
                wmax[b] = max(wmax[b], imm)
        for b in range(h["n_bufs"]):
            ln = int(x[k]["buf_len"][b])
            if (h["shared_mask"] >> b) & 1:
                assert ln - 256 * wmax[b] in (-wmax[b], 0, wmax[b])
            else:
                assert 1 <= ln <= 16 << 20


def test_c3_c4_recipes():
    x = gen.c3_inputs(4096)
    assert len(x) == 4096 and x["program_id"].max() < 16
    nb, nt = x["grid"][:, 0].astype(np.int64), x["block"][:, 0].astype(np.int64)
    assert nb.min() >= 1 and nb.max() <= 65536 and nt.min() >= 32 and nt.max() <= 1024
    w = np.array(gen.C3_WIDTHS)[x["program_id"]]
    assert (x["buf_len"][:, :4] % w[:, None] == 0).all()
    assert 1e6 < threads(x).mean() < 3e6                            # ~1.7 M threads per input
    progs = gen.c4_programs()
    for p in progs:
        ifs = sum(1 for o in bc.ops_of(p) if o[0] == bc.IF)
        assert 32 <= ifs <= 64
    y = gen.c4_inputs(16384)
    assert len(y) == 16384 and (y["block"] == (256, 1, 1)).all()
    assert y["grid"][:, 0].min() >= 1 and y["grid"][:, 0].max() <= 1024
    assert (y["buf_len"][:, 0] == 4 * 4096).all()
    assert set(np.unique(y["buf_len"][:, 1] // 4).tolist()) <= {1023, 1024, 1025}


def test_prex_workload_recipes():
    x = gen.guard2d_inputs(4096)
    bx, by = x["block"][:, 0].astype(np.int64), x["block"][:, 1].astype(np.int64)
    assert set(zip(bx.tolist(), by.tolist())) <= {(8, 8), (16, 16), (32, 8), (32, 32)}
    gx, gy = x["grid"][:, 0].astype(np.int64), x["grid"][:, 1].astype(np.int64)
    assert gx.max() <= 256 and gy.max() <= 256 and gx.min() >= 1 and gy.min() >= 1
    rows, cols = x["args"][:, 0].astype(np.int64), x["args"][:, 1].astype(np.int64)
    assert (rows >= 1).all() and (rows <= gy * by).all() and (cols >= 1).all() and (cols <= gx * bx).all()
    w = np.array(gen.G2_WIDTHS)[x["program_id"]]
    short = (rows * cols)[:, None] - x["buf_len"][:, :3].astype(np.int64) // w[:, None]
    assert set(np.unique(short).tolist()) <= {0, 1} and 0.07 < (short == 1).mean() < 0.13
    a = gen.affine_inputs(4096)
    assert a["program_id"].max() < 16 and (a["grid"][:, 1:] == 1).all()


def test_generators_are_seeded():
    assert gen.c3_inputs(64, seed=5).tobytes() == gen.c3_inputs(64, seed=5).tobytes()
    assert gen.c3_inputs(64, seed=5).tobytes() != gen.c3_inputs(64, seed=6).tobytes()
    assert gen.c2_programs(4) == gen.c2_programs(4)
    progs = gen.c5_programs()
    assert len(progs) == 64 and len(gen.c5_corpus(progs)) == 256
