"""A second, deliberately naive evaluator of access-index programs, used only
to pin the C oracle on tiny grids (every block, every thread).

It is written independently of oracle/cufz_oracle.c: its own decoder (a
recursive parse into nested blocks), Python integers with explicit masking,
its own hash, classification and bucketing.  Both follow the same definition:
serial execution of every thread (Sec. 4.1, Listings 1-2), exact bounds
checks, AFL-style edges (Sec. 2.1).  A program with performed shared stores
runs each block as Python generators, one per thread, advanced in thread
order from one barrier to the next.
"""
from __future__ import annotations

import struct

M32 = 0xFFFFFFFF
M64 = (1 << 64) - 1


def s32(v):
    v &= M32
    return v - (1 << 32) if v >> 31 else v


def murmur_fmix32(h):
    h &= M32
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & M32
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & M32
    return h ^ (h >> 16)


def afl_class(n):
    for limit, cls in ((0, 0), (1, 1), (2, 2), (3, 4), (7, 8), (15, 16), (31, 32), (127, 64)):
        if n <= limit:
            return cls
    return 128


def parse(prog: bytes):
    magic, ver, n_ops, n_regs, n_bufs, n_sites, flags, shmask, _, seed = struct.unpack_from(
        "<IHHBBBBHHI", prog, 0)
    assert magic == 0x315A4643 and ver == 1
    loc = [struct.unpack_from("<HH", prog, 32 + 4 * s) for s in range(n_sites)]
    raw = [struct.unpack_from("<BBBBi", prog, 32 + 4 * n_sites + 8 * i) for i in range(n_ops)]
    counters = {"b": 0, "a": 0, "d": 0, "h": 0, "f": 0}
    pos = [0]

    def block(terminators):
        out = []
        while pos[0] < len(raw):
            opc, d, a, b, imm = raw[pos[0]]
            if opc in terminators:
                return out, opc
            pos[0] += 1
            if opc == 0x50:
                site = counters["b"]
                counters["b"] += 1
                then, t = block((0x51, 0x52))
                els = []
                if t == 0x51:
                    pos[0] += 1
                    els, t = block((0x52,))
                pos[0] += 1
                out.append(("if", a, site, then, els))
            elif opc == 0x53:
                site = counters["b"]
                counters["b"] += 1
                body, _ = block((0x54,))
                pos[0] += 1
                out.append(("loop", d, a, imm, site, body))
            elif opc in (0x40, 0x41):
                out.append(("mem", opc == 0x41, d, a, b, imm, counters["a"]))
                counters["a"] += 1
            elif opc in (0x05, 0x06):
                out.append(("div", opc == 0x06, d, a, b, counters["d"]))
                counters["d"] += 1
            elif opc == 0x07:
                out.append(("halloc", d, a, counters["h"]))
                counters["h"] += 1
            elif opc == 0x08:
                out.append(("hfree", a, counters["f"]))
                counters["f"] += 1
            elif opc in (0x42, 0x43):
                out.append(("hmem", opc == 0x43, d, a, b, imm, counters["a"]))
                counters["a"] += 1
            elif opc == 0x55:
                out.append(("bar",))
            else:
                out.append(("op", opc, d, a, b, imm))
        return out, None

    body, _ = block(())
    return dict(n_regs=n_regs, n_bufs=n_bufs, shmask=shmask, seed=seed, loc=loc, body=body,
                n_alloc=counters["h"], stores=bool(flags & 1))


def alu(opc, x, y):
    ux, uy = x & M32, y & M32
    sh = uy & 31
    f = {
        0x10: lambda: ux + uy, 0x11: lambda: ux - uy, 0x12: lambda: ux * uy,
        0x13: lambda: ux << sh, 0x14: lambda: s32(ux) >> sh, 0x15: lambda: ux >> sh,
        0x16: lambda: ux & uy, 0x17: lambda: ux | uy, 0x18: lambda: ux ^ uy,
        0x19: lambda: min(s32(ux), s32(uy)), 0x1A: lambda: max(s32(ux), s32(uy)),
        0x1B: lambda: int(s32(ux) < s32(uy)), 0x1C: lambda: int(s32(ux) <= s32(uy)),
        0x1D: lambda: int(ux == uy), 0x1E: lambda: int(ux != uy), 0x1F: lambda: int(ux < uy),
    }[opc]
    return s32(f())


def evaluate(prog: bytes, inp: dict, redzone=256, budget=4096):
    """inp: dict(grid=(x,y,z), block=(x,y,z), args=[4], lens=[...]).
    Returns dict(status, flags, records=[tuple], counts={e: n}, digest,
    n_accesses, n_violations, first_key, n_branch, n_ops, traces), where
    traces maps (block_lin, thread_lin) to the thread's accesses in order,
    as (site, index) pairs."""
    P = parse(prog)
    g, b = inp["grid"], inp["block"]
    if 0 in g or 0 in b or b[0] > 1024 or b[1] > 1024 or b[2] > 64 or b[0] * b[1] * b[2] > 1024 \
            or g[0] > 2**31 - 1 or g[1] > 65535 or g[2] > 65535:
        return dict(status=2, flags=0, records=[], counts={}, digest=0, n_accesses=0,
                    n_violations=0, first_key=M64, n_branch=0, n_ops=0, traces={})
    lens = list(inp["lens"]) + [0] * 9
    shm = P["shmask"]
    base = {}
    nxt = {0: redzone, 1: redzone}
    for k in range(P["n_bufs"]):
        sp = (shm >> k) & 1
        base[k] = nxt[sp]
        nxt[sp] = -(-(nxt[sp] + lens[k] + redzone) // 256) * 256
    # n_ops: executed ops that compute a value or make a non-access check
    # (IMM, MOV, SEL, ALU, DIV/REM, HALLOC, HFREE); SREG reads do not count
    st = dict(records=[], counts={}, digest=0, n_accesses=0, n_branch=0, n_ops=0,
              budget_hit=False, traces={})
    smem = {}  # (buffer, byte offset) -> byte: the current block's stored shared bytes

    def classify(buf, off, w):
        if -redzone <= off < 0:
            return 1
        if 0 <= off < lens[buf] + redzone:
            return 2
        addr = base[buf] + off
        for j in range(P["n_bufs"]):
            if j != buf and ((shm >> j) & 1) == ((shm >> buf) & 1) and lens[j] > 0:
                if addr < base[j] + lens[j] and addr + w > base[j]:
                    return 3
        return 4

    def run_thread(bl, tl, sregs):
        regs = [0] * max(P["n_regs"], 1)
        t = dict(ordinal=0, prev=0, back=0, stop=False,
                 h=(bl * 0x9E3779B1 + tl + 0x7F4A7C15) & M32)
        trace = st["traces"].setdefault((bl, tl), [])

        def edge(site, out):
            cur = P["loc"][site][out]
            e = (cur ^ t["prev"]) & 0xFFFF
            st["counts"][e] = st["counts"].get(e, 0) + 1
            t["prev"] = cur >> 1
            st["n_branch"] += 1

        def mem(is_st, d, a, buf, w, site):
            off = regs[a] * w
            bad = off < 0 or off + w > lens[buf]
            trace.append((site, regs[a]))
            k = ((site * 0xC2B2AE3D) & M32) | 3
            t["h"] = (t["h"] * k + regs[a]) & M32
            st["n_accesses"] += 1
            val = 0
            if bad:
                st["records"].append((bl, tl, t["ordinal"], site, buf, int(is_st), w,
                                      (shm >> buf) & 1, classify(buf, off, w), off))
            elif not is_st and not (shm >> buf) & 1:
                word = murmur_fmix32(P["seed"] ^ ((buf * 0x9E3779B9) & M32) ^ ((off >> 2) & M32))
                val = s32((word >> (8 * (off & 3))) & 0xFF) if w == 1 else s32(word)
            elif P["stores"] and (shm >> buf) & 1 and is_st:
                data = (regs[d] & M32).to_bytes(4, "little") + bytes(max(w - 4, 0))
                for k in range(w):
                    smem[(buf, off + k)] = data[k]
            elif P["stores"] and (shm >> buf) & 1:
                data = bytes(smem.get((buf, off + k), 0) for k in range(1 if w == 1 else 4))
                val = s32(int.from_bytes(data, "little"))
            t["ordinal"] += 1
            if not is_st:
                regs[d] = val

        def divide(is_rem, d, a, b, site):
            x, y = regs[a], regs[b]
            if y == 0:
                st["records"].append((bl, tl, t["ordinal"], site, 0, 2, 0, 0, 5, 0))
                val = 0
            else:
                q = abs(x) // abs(y)
                q = q if (x < 0) == (y < 0) else -q
                val = s32(x - y * q) if is_rem else s32(q)
            t["ordinal"] += 1
            regs[d] = val

        heap = {}  # allocation site -> [size, live]

        def block_of(h):
            return heap.get(h - 1) if 1 <= h <= P["n_alloc"] else None

        def hfree(a, site):
            h = regs[a]
            if h != 0:
                blk = block_of(h)
                if blk is None:
                    st["records"].append((bl, tl, t["ordinal"], site, 0, 3, 0, 2, 8, 0))
                elif not blk[1]:
                    st["records"].append((bl, tl, t["ordinal"], site, 0, 3, 0, 2, 7, 0))
                else:
                    blk[1] = False
            t["ordinal"] += 1

        def hmem(is_st, d, a, hreg, w, site):
            off = regs[a] * w
            trace.append((site, regs[a]))
            k = ((site * 0xC2B2AE3D) & M32) | 3
            t["h"] = (t["h"] * k + regs[a]) & M32
            st["n_accesses"] += 1
            h, blk, cls = regs[hreg], None, 0
            blk = block_of(h)
            if blk is None:
                cls = 4
            elif not blk[1]:
                cls = 6
            elif off < 0 or off + w > blk[0]:
                cls = 1 if -redzone <= off < 0 else 2 if 0 <= off < blk[0] + redzone else 4
            if cls:
                st["records"].append((bl, tl, t["ordinal"], site, h - 1 if blk is not None else 0,
                                      int(is_st), w, 2, cls, off))
            t["ordinal"] += 1
            if not is_st:
                regs[d] = 0

        def run(stmts):
            for s in stmts:
                if t["stop"]:
                    return
                kind = s[0]
                if kind == "op":
                    _, opc, d, a, bb, imm = s
                    if opc in (0x02, 0x03, 0x04) or 0x10 <= opc <= 0x1F or 0x30 <= opc <= 0x3F:
                        st["n_ops"] += 1
                    if opc == 0x01:
                        regs[d] = sregs[imm]
                    elif opc == 0x02:
                        regs[d] = imm
                    elif opc == 0x03:
                        regs[d] = regs[a]
                    elif opc == 0x04:
                        regs[d] = regs[bb] if regs[a] != 0 else regs[imm]
                    elif 0x10 <= opc <= 0x1F:
                        regs[d] = alu(opc, regs[a], regs[bb])
                    elif 0x30 <= opc <= 0x3F:
                        regs[d] = alu(opc - 0x20, regs[a], imm)
                elif kind == "mem":
                    _, is_st, d, a, buf, w, site = s
                    mem(is_st, d, a, buf, w, site)
                elif kind == "div":
                    _, is_rem, d, a, bb, site = s
                    divide(is_rem, d, a, bb, site)
                    st["n_ops"] += 1
                elif kind == "halloc":
                    _, d, a, site = s
                    st["n_ops"] += 1
                    if regs[a] >= 1:
                        heap[site] = [regs[a], True]
                        regs[d] = site + 1
                    else:
                        regs[d] = 0
                elif kind == "hfree":
                    hfree(s[1], s[2])
                    st["n_ops"] += 1
                elif kind == "hmem":
                    _, is_st, d, a, hreg, w, site = s
                    hmem(is_st, d, a, hreg, w, site)
                elif kind == "if":
                    _, a, site, then, els = s
                    taken = regs[a] != 0
                    edge(site, int(taken))
                    run(then if taken else els)
                else:
                    _, ctr, a, mx, site, body = s
                    trip = min(max(regs[a], 0), mx)
                    regs[ctr] = 0
                    while True:
                        edge(site, int(regs[ctr] < trip))
                        if regs[ctr] >= trip:
                            break
                        run(body)
                        if t["stop"]:
                            return
                        t["back"] += 1
                        if t["back"] > budget:
                            t["stop"] = True
                            st["budget_hit"] = True
                            return
                        regs[ctr] += 1

        for s in P["body"]:       # a barrier ends a phase: the next thread runs
            if s[0] == "bar":
                yield
            else:
                run([s])
        st["digest"] = (st["digest"] + (t["h"] ^ (t["h"] >> 16))) & M64

    args = [s32(v) for v in inp["args"]]
    for bz in range(g[2]):
        for by in range(g[1]):
            for bx in range(g[0]):
                bl = bx + by * g[0] + bz * g[0] * g[1]
                smem.clear()
                threads = []
                for tz in range(b[2]):
                    for ty in range(b[1]):
                        for tx in range(b[0]):
                            tl = tx + ty * b[0] + tz * b[0] * b[1]
                            sregs = [tx, ty, tz, b[0], b[1], b[2], bx, by, bz, g[0], g[1], g[2]] + args
                            threads.append(run_thread(bl, tl, [s32(v) for v in sregs]))
                if P["stores"]:       # phase by phase, every thread in order
                    for _ in range(1 + sum(1 for s in P["body"] if s[0] == "bar")):
                        for th in threads:
                            next(th, None)
                else:                 # each thread to its end (BAR does nothing)
                    for th in threads:
                        for _ in th:
                            pass
    recs = st["records"]
    fk = min(((r[0] << 32) | (r[1] << 22) | min(r[2], (1 << 22) - 1) for r in recs), default=M64)
    return dict(status=1 if recs else 0, flags=1 if st["budget_hit"] else 0, records=recs,
                counts=st["counts"], digest=st["digest"], n_accesses=st["n_accesses"],
                n_violations=len(recs), first_key=fk, n_branch=st["n_branch"],
                n_ops=st["n_ops"], traces=st["traces"])


def bitmap_of(counts: dict) -> dict:
    return {e: afl_class(n) for e, n in counts.items() if n}
