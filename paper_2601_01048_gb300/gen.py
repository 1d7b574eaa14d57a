"""Seeded synthetic workloads: programs, fuzz inputs and the input mutator.

Nothing here checks, prunes or counts anything; it only draws programs and
inputs.  Both the CPU oracle and the device engine consume what it makes.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then the variant-13 output mix.  Root seed 0xC0F5EED, one sub-seed per
workload.

The paper fuzzes HeteroMark, Rodinia and CUDA-SDK programs with AFL++
(Sec. 7, Table 2); those programs are not available here, so the workloads
below stand in for them with the same access shapes: affine guarded 1D
kernels (vecAdd-like, Listing 3), random 2D kernels with shared staging and
loops (matmul/fir-like), and branch-heavy data-dependent kernels (bfs/pr-like
indirect accesses, Sec. 7.4.1).
"""
from __future__ import annotations

import math

import numpy as np

from . import bytecode as bc
from .bytecode import Asm, Imm

ROOT_SEED = 0xC0F5EED
MASK64 = (1 << 64) - 1

# One fuzz input record, 128 bytes (the wire format of cufz_input).
INPUT_DTYPE = np.dtype([
    ("program_id", "<u4"), ("grid", "<u4", (3,)), ("block", "<u4", (3,)),
    ("args", "<i4", (4,)), ("pad", "<u4"), ("buf_len", "<u8", (9,)), ("user_tag", "<u8"),
])
assert INPUT_DTYPE.itemsize == 128


class SplitMix64:
    """SplitMix64 generator (Steele, Lea, Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def next32(self) -> int:
        return self.next() >> 32

    def below(self, n: int) -> int:
        """Uniform integer in [0, n) (n <= 2^32; multiply-shift, bias < 2^-32)."""
        return (self.next32() * n) >> 32

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] inclusive."""
        return lo + self.below(hi - lo + 1)

    def uniform(self) -> float:
        return (self.next() >> 11) * (1.0 / (1 << 53))

    def chance(self, p: float) -> bool:
        return self.uniform() < p

    def choice(self, seq):
        return seq[self.below(len(seq))]

    def loguniform_int(self, lo: int, hi: int) -> int:
        """Integer drawn log-uniformly from [lo, hi]."""
        v = int(math.exp(math.log(lo) + self.uniform() * (math.log(hi + 1) - math.log(lo))))
        return min(max(v, lo), hi)


def sub_seed(name: str, index: int = 0) -> int:
    h = ROOT_SEED
    for ch in name.encode():
        h = SplitMix64(h ^ ch).next()
    return SplitMix64(h ^ index).next()


def make_inputs(n: int) -> np.ndarray:
    return np.zeros(n, dtype=INPUT_DTYPE)


def set_input(rec, program_id: int, grid, block, args, lens, tag: int = 0) -> None:
    rec["program_id"] = program_id
    rec["grid"] = tuple(grid)
    rec["block"] = tuple(block)
    a = list(args) + [0] * (4 - len(args))
    rec["args"] = [((v + (1 << 31)) % (1 << 32)) - (1 << 31) for v in a]
    ln = list(lens) + [0] * (9 - len(lens))
    rec["buf_len"] = ln
    rec["user_tag"] = tag


# --------------------------------------------------------------------------
# hand-built programs from the paper's listings
# --------------------------------------------------------------------------

def vecadd_shared_program(block_size: int) -> bytes:
    """Listing 1: vecAdd staging a and b through shared arrays (7 accesses).

    Buffers: 0 a, 1 b, 2 c (global); 3 s_a, 4 s_b (shared, blockSize ints).
    The barrier has no counterpart here: stores are not performed, so it
    cannot change any access (Alg. 2, BarrierElimination).
    """
    A = Asm(n_bufs=5, shared_mask=0b11000, seed=0x5EC0ADD)
    tx = A.sreg(bc.TID_X)
    bx = A.sreg(bc.CTAID_X)
    idv = A.alu(bc.ADD, A.alu(bc.MUL, bx, Imm(block_size)), tx)
    va = A.ld(0, idv)
    A.st(3, tx, va)
    vb = A.ld(1, idv)
    A.st(4, tx, vb)
    sa = A.ld(3, tx)
    sb = A.ld(4, tx)
    A.st(2, idv, A.alu(bc.ADD, sa, sb))
    return A.build()


def guarded_plus1_program(block_size: int) -> bytes:
    """Listing 3: if (id < N) c[id+1] = a[id+1] + b[id+1]; N is arg0.

    Buffers 0 a, 1 b, 2 c (global).
    """
    A = Asm(n_bufs=3, seed=0x11573)
    tx = A.sreg(bc.TID_X)
    bx = A.sreg(bc.CTAID_X)
    n = A.sreg(bc.ARG0)
    idv = A.alu(bc.ADD, A.alu(bc.MUL, bx, Imm(block_size)), tx)
    A.if_(A.alu(bc.SETLT, idv, n))
    i1 = A.alu(bc.ADD, idv, Imm(1))
    va = A.ld(0, i1)
    vb = A.ld(1, i1)
    A.st(2, i1, A.alu(bc.ADD, va, vb))
    A.endif()
    return A.build()


# --------------------------------------------------------------------------
# config 1: the plain guarded 1D kernel
# --------------------------------------------------------------------------

def c1_family_program(offset: int = 0, width: int = 4, seed: int = 0xC1) -> bytes:
    """i = ctaid.x*ntid.x + tid.x + arg0 + offset; if (i < arg1) {
    x = A[i]; y = B[i]; C[i] = x + y }.  Buffer D (3) is allocated and never
    accessed, so a stray index can land in it.  All four buffers are global."""
    A = Asm(n_bufs=4, seed=seed)
    tx = A.sreg(bc.TID_X)
    bx = A.sreg(bc.CTAID_X)
    nx = A.sreg(bc.NTID_X)
    a0 = A.sreg(bc.ARG0)
    a1 = A.sreg(bc.ARG1)
    i = A.alu(bc.ADD, A.alu(bc.ADD, A.alu(bc.MUL, bx, nx), tx), a0)
    if offset:
        i = A.alu(bc.ADD, i, Imm(offset))
    A.if_(A.alu(bc.SETLT, i, a1))
    x = A.ld(0, i, width)
    y = A.ld(1, i, width)
    A.st(2, i, A.alu(bc.ADD, x, y), width)
    A.endif()
    return A.build()


def c1_program() -> bytes:
    return c1_family_program(0, 4, seed=0xC1)


def c1_inputs(n: int = 1000, seed: int | None = None, program_id: int = 0) -> np.ndarray:
    """Config 1: grid 64 x 128, arg0 ~ U[-4,4], arg1 ~ U[0,8192]; each buffer
    length (in 4-byte elements) is max(arg1-1, 0) with p=0.1 (off by one),
    U[0,8192] with p=0.1, else U[arg1, 8192]."""
    rng = SplitMix64(sub_seed("c1") if seed is None else seed)
    out = make_inputs(n)
    for k in range(n):
        a0 = rng.randint(-4, 4)
        a1 = rng.randint(0, 8192)
        lens = []
        for _b in range(4):
            u = rng.uniform()
            if u < 0.10:
                e = max(a1 - 1, 0)
            elif u < 0.20:
                e = rng.randint(0, 8192)
            else:
                e = rng.randint(a1, 8192)
            lens.append(4 * e)
        set_input(out[k], program_id, (64, 1, 1), (128, 1, 1), (a0, a1), lens, tag=k)
    return out


# --------------------------------------------------------------------------
# config 3: 16 C1-family programs, log-uniform grids and blocks
# --------------------------------------------------------------------------

C3_WIDTHS = (4, 4, 8, 1, 16, 4, 8, 4, 1, 4, 16, 8, 4, 4, 1, 4)


def c3_programs() -> list[bytes]:
    rng = SplitMix64(sub_seed("c3prog"))
    progs = []
    for p in range(16):
        off = rng.randint(-3, 3) if p else 0
        progs.append(c1_family_program(off, C3_WIDTHS[p], seed=rng.next32()))
    return progs


def c3_inputs(n: int = 4096, seed: int | None = None, max_blocks: int = 65536,
              min_threads: int = 32, max_threads: int = 1024) -> np.ndarray:
    rng = SplitMix64(sub_seed("c3") if seed is None else seed)
    out = make_inputs(n)
    for k in range(n):
        p = rng.below(16)
        w = C3_WIDTHS[p]
        nb = rng.loguniform_int(1, max_blocks)
        nt = rng.loguniform_int(min_threads, max_threads)
        total = nb * nt
        a0 = rng.randint(-4, 4)
        a1 = rng.randint(0, total)
        lens = []
        for _b in range(4):
            u = rng.uniform()
            if u < 0.10:
                e = max(a1 - 1, 0)
            elif u < 0.20:
                e = rng.randint(0, total)
            else:
                e = rng.randint(a1, total)
            lens.append(w * e)
        set_input(out[k], p, (nb, 1, 1), (nt, 1, 1), (a0, a1), lens, tag=k)
    return out


# --------------------------------------------------------------------------
# PREX workload: unguarded affine-access programs (Sec. 5.1's class, like the
# paper's vecadd/matmul/aes), launch shapes as configuration 3
# --------------------------------------------------------------------------

AFF_WIDTHS = (4, 8, 4, 1, 16, 4, 4, 8, 4, 1, 4, 16, 4, 8, 4, 4)


def affine_family_program(off: int, w: int, k_inner: int, seed: int) -> bytes:
    """i = ctaid.x * ntid.x + tid.x + arg0; loads A[i], B[i + off] (width w),
    a uniform loop over k < min(arg1, 8) reading C[i * k_inner + k], a store
    D[i]; no thread-dependent branch (the affine-access class)."""
    A = Asm(n_bufs=4, seed=seed)
    tx, bx, nx = A.sreg(bc.TID_X), A.sreg(bc.CTAID_X), A.sreg(bc.NTID_X)
    a0, a1 = A.sreg(bc.ARG0), A.sreg(bc.ARG1)
    i = A.alu(bc.ADD, A.alu(bc.ADD, A.alu(bc.MUL, bx, nx), tx), a0)
    A.ld(0, i, 4)
    A.ld(1, A.alu(bc.ADD, i, Imm(off)), w)
    k = A.loop(a1, 8)
    A.ld(2, A.alu(bc.ADD, A.alu(bc.MUL, i, Imm(k_inner)), k), 4)
    A.endloop()
    A.st(3, i, tx, 4)
    return A.build()


def affine_programs() -> list[bytes]:
    rng = SplitMix64(sub_seed("affprog"))
    return [affine_family_program(rng.randint(-2, 2), AFF_WIDTHS[p], rng.randint(1, 4),
                                  seed=rng.next32()) for p in range(16)]


def affine_inputs(n: int = 4096, seed: int | None = None, max_blocks: int = 65536,
                  min_threads: int = 32, max_threads: int = 1024) -> np.ndarray:
    """Configuration-3 shapes; each buffer sized for the grid, one in ten an
    element short (the off-by-one bug PREX must still find)."""
    rng = SplitMix64(sub_seed("aff") if seed is None else seed)
    progs_k = []
    rk = SplitMix64(sub_seed("affprog"))
    for p in range(16):
        rk.randint(-2, 2)
        progs_k.append(rk.randint(1, 4))
        rk.next32()
    out = make_inputs(n)
    for k in range(n):
        p = rng.below(16)
        nb = rng.loguniform_int(1, max_blocks)
        nt = rng.loguniform_int(min_threads, max_threads)
        total = nb * nt
        a0 = rng.randint(-1, 1)
        a1 = rng.randint(0, 8)
        ws = (4, AFF_WIDTHS[p], 4, 4)
        lens = []
        for b in range(4):
            e = total + 2 if b != 2 else total * progs_k[p] + 8
            if rng.uniform() < 0.10:
                e -= 3
            lens.append(ws[b] * e)
        set_input(out[k], p, (nb, 1, 1), (nt, 1, 1), (a0, a1), lens, tag=k)
    return out


# --------------------------------------------------------------------------
# guarded 2D workload: bounds-guarded matrix kernels (the guarded class of
# Sec. 5.1's Alg. 1 in two dimensions, like the paper's matmul)
# --------------------------------------------------------------------------

G2_WIDTHS = (4, 4, 8, 1, 16, 4, 8, 4, 4, 1, 4, 16, 8, 4, 4, 4)


def guard2d_family_program(off: int, w: int, seed: int) -> bytes:
    """row = ctaid.y * ntid.y + tid.y, col = ctaid.x * ntid.x + tid.x;
    if (row < arg0 && col < arg1) { A[row * arg1 + col]; B[row * arg1 + col
    + off]; C[row * arg1 + col] = ... } with accesses of width w."""
    A = Asm(n_bufs=3, seed=seed)
    row = A.alu(bc.ADD, A.alu(bc.MUL, A.sreg(bc.CTAID_Y), A.sreg(bc.NTID_Y)), A.sreg(bc.TID_Y))
    col = A.alu(bc.ADD, A.alu(bc.MUL, A.sreg(bc.CTAID_X), A.sreg(bc.NTID_X)), A.sreg(bc.TID_X))
    n, m = A.sreg(bc.ARG0), A.sreg(bc.ARG1)
    A.if_(A.alu(bc.AND, A.alu(bc.SETLT, row, n), A.alu(bc.SETLT, col, m)))
    i = A.alu(bc.ADD, A.alu(bc.MUL, row, m), col)
    x = A.ld(0, i, w)
    y = A.ld(1, A.alu(bc.ADD, i, Imm(off)), w)
    A.st(2, i, A.alu(bc.ADD, x, y), w)
    A.endif()
    return A.build()


def guard2d_programs() -> list[bytes]:
    rng = SplitMix64(sub_seed("g2prog"))
    return [guard2d_family_program(rng.randint(-2, 2) if p else 0, G2_WIDTHS[p], seed=rng.next32())
            for p in range(16)]


def guard2d_inputs(n: int = 4096, seed: int | None = None, max_grid: int = 256) -> np.ndarray:
    """Blocks 8x8, 16x16, 32x8 or 32x32; gx, gy log-uniform in [1, max_grid];
    rows and columns uniform up to the grid's extent (the guards cut inside
    the grid); each buffer holds rows x columns elements, one in ten an
    element short."""
    rng = SplitMix64(sub_seed("g2") if seed is None else seed)
    out = make_inputs(n)
    for k in range(n):
        p = rng.below(16)
        bx, by = rng.choice(((8, 8), (16, 16), (32, 8), (32, 32)))
        gx, gy = rng.loguniform_int(1, max_grid), rng.loguniform_int(1, max_grid)
        rows, cols = rng.randint(1, gy * by), rng.randint(1, gx * bx)
        lens = [G2_WIDTHS[p] * (rows * cols - (1 if rng.uniform() < 0.10 else 0)) for _ in range(3)]
        set_input(out[k], p, (gx, gy, 1), (bx, by, 1), (rows, cols), lens, tag=k)
    return out


# --------------------------------------------------------------------------
# division workload: signed DIV/REM whose divisors are zero for some threads
# or inputs (the divide-by-zero kernel error of Sec. 2.3)
# --------------------------------------------------------------------------

def div_program(index: int) -> bytes:
    """Random programs with signed divisions.  Divisors come from a
    coordinate minus an argument, a masked argument, a loaded byte, or a
    value plus a small constant: each is zero for some threads or inputs.
    Quotients and remainders feed access indices, branch conditions and a
    uniform loop."""
    rng = SplitMix64(sub_seed("divprog", index))
    A = Asm(n_bufs=3, seed=rng.next32())
    tx, ty, bx = A.sreg(bc.TID_X), A.sreg(bc.TID_Y), A.sreg(bc.CTAID_X)
    args = [A.sreg(bc.ARG0 + k) for k in range(4)]
    lin = A.alu(bc.ADD, A.alu(bc.MUL, bx, A.sreg(bc.NTID_X)), tx)
    coords = [tx, ty, lin]
    vals = coords + args

    def divisor():
        r = rng.below(4)
        if r == 0:
            return A.alu(bc.SUB, rng.choice(coords), rng.choice(args))
        if r == 1:
            return A.alu(bc.AND, rng.choice(args), Imm(rng.choice((1, 3, 7))))
        if r == 2:
            return A.ld(0, A.alu(bc.AND, lin, Imm(63)), 1)
        return A.alu(bc.ADD, rng.choice(vals), Imm(rng.randint(-2, 2)))

    def division():
        x = rng.choice(vals)
        q = A.div(x, divisor()) if rng.below(2) else A.rem(x, divisor())
        vals.append(q)
        return q

    def index():
        v = rng.choice(vals[-4:])
        return A.alu(bc.AND, v, Imm(rng.choice((63, 255, -1))))

    def body(depth):
        for _ in range(rng.randint(2, 5)):
            r = rng.below(6)
            if r <= 1 or depth >= 2:
                division()
            elif r == 2:
                A.ld(rng.choice((1, 2)), index(), rng.choice((1, 4)))
            elif r == 3:
                A.if_(A.alu(bc.SETLT, rng.choice(vals), rng.choice(vals)))
                body(depth + 1)
                A.endif()
            elif r == 4:
                k = A.loop(A.alu(bc.AND, args[3], Imm(3)), 4)
                q = A.div(A.alu(bc.ADD, k, rng.choice(vals)), divisor())
                A.ld(1, A.alu(bc.AND, q, Imm(127)), 1)
                A.endloop()
            else:
                A.st(2, index(), rng.choice(vals), 4)
        A.ld(1, index(), 4)

    body(0)
    return A.build()


def div_programs(n: int = 16) -> list[bytes]:
    return [div_program(i) for i in range(n)]


def div_inputs(n: int, n_programs: int = 16, seed: int | None = None,
               max_blocks: int = 8) -> np.ndarray:
    """Blocks of 16 x 4 threads, 1D grids up to max_blocks; arguments from
    {0, +-1, 2, 3, 5, 16, -7, INT_MIN}; buffer 0 (the divisor bytes) 0-512
    bytes, buffers 1 and 2 up to 4 KiB."""
    rng = SplitMix64(sub_seed("div") if seed is None else seed)
    out = make_inputs(n)
    for k in range(n):
        args = [rng.choice((0, 1, -1, 2, 3, 5, 16, -7, -(1 << 31))) for _ in range(4)]
        lens = [rng.randint(0, 512), rng.randint(0, 4096), rng.randint(0, 4096)]
        set_input(out[k], k % n_programs, (rng.randint(1, max_blocks), 1, 1), (16, 4, 1), args,
                  lens, tag=k)
    return out


# --------------------------------------------------------------------------
# heap workload: per-thread device-heap blocks, accessed, freed and misused
# (the temporal errors of Sec. 2.3: use after free, double free, invalid free)
# --------------------------------------------------------------------------

def heap_program(index: int) -> bytes:
    """Random programs over the device heap.  Sizes come from arguments,
    coordinates and constants (some <= 0: a NULL handle); handles are the
    allocations' results or fabricated (small constants, coordinates);
    blocks are loaded and stored at indices that may leave them, freed once,
    twice or never, used after free, under guards and in a uniform loop."""
    rng = SplitMix64(sub_seed("heapprog", index))
    A = Asm(n_bufs=1, seed=rng.next32())
    tx, bx = A.sreg(bc.TID_X), A.sreg(bc.CTAID_X)
    args = [A.sreg(bc.ARG0 + k) for k in range(4)]
    lin = A.alu(bc.ADD, A.alu(bc.MUL, bx, A.sreg(bc.NTID_X)), tx)
    handles = []

    def size():
        r = rng.below(4)
        if r == 0:
            return rng.choice(args)
        if r == 1:
            return A.alu(bc.ADD, tx, Imm(rng.randint(-2, 8)))
        if r == 2:
            return A.imm(rng.choice((1, 4, 16, 64, 0, -3)))
        return A.alu(bc.SUB, A.alu(bc.AND, rng.choice(args), Imm(63)), A.alu(bc.AND, lin, Imm(7)))

    def handle():
        if handles and rng.below(5):
            return rng.choice(handles)
        return A.imm(rng.randint(-1, 4)) if rng.below(2) else A.alu(bc.AND, lin, Imm(3))

    def index():
        r = rng.below(4)
        if r == 0:
            return tx
        if r == 1:
            return A.alu(bc.SUB, lin, rng.choice(args))
        if r == 2:
            return A.alu(bc.AND, rng.choice(args), Imm(31))
        return A.alu(bc.SUB, A.alu(bc.MUL, tx, Imm(4)), Imm(2))

    def body(depth):
        for _ in range(rng.randint(3, 7)):
            r = rng.below(8)
            if r <= 1 or not handles:
                handles.append(A.halloc(size()))
            elif r == 2:
                A.hld(handle(), index(), rng.choice((1, 4, 8)))
            elif r == 3:
                A.hst(handle(), index(), tx, rng.choice((1, 4)))
            elif r == 4:
                A.hfree(handle())
            elif r == 5 and depth < 2:
                A.if_(A.alu(bc.SETLT, tx, args[3]))
                body(depth + 1)
                A.endif()
            elif r == 6 and depth < 2:
                k = A.loop(A.alu(bc.AND, args[2], Imm(3)), 4)
                h = A.halloc(A.alu(bc.ADD, k, Imm(rng.randint(0, 4))))
                A.hst(h, A.alu(bc.SUB, k, Imm(1)), k, 1)
                if rng.below(2):
                    A.hfree(h)
                A.endloop()
            else:
                A.ld(0, index(), 4)

    body(0)
    return A.build()


def heap_programs(n: int = 16) -> list[bytes]:
    return [heap_program(i) for i in range(n)]


def heap_inputs(n: int, n_programs: int = 16, seed: int | None = None,
                max_blocks: int = 4) -> np.ndarray:
    """Blocks of 16 x 2 threads, 1D grids up to max_blocks; arguments from
    {0, +-1, 2, 3, 5, 8, 16, 40, -7}; buffer 0 up to 256 bytes."""
    rng = SplitMix64(sub_seed("heap") if seed is None else seed)
    out = make_inputs(n)
    for k in range(n):
        args = [rng.choice((0, 1, -1, 2, 3, 5, 8, 16, 40, -7)) for _ in range(4)]
        set_input(out[k], k % n_programs, (rng.randint(1, max_blocks), 1, 1), (16, 2, 1), args,
                  [rng.randint(0, 256)], tag=k)
    return out


# --------------------------------------------------------------------------
# barrier workload: performed shared stores ordered by barriers (the input
# of AXIPrune's BarrierElimination, Sec. 5.2)
# --------------------------------------------------------------------------

BAR_BLOCKS = ((8, 2, 1), (16, 1, 1), (4, 4, 1), (32, 1, 1))


def barrier_program(index: int, live: bool = False) -> bytes:
    """Random programs whose stores to shared buffers are performed, in 2-4
    phases split by barriers.  Buffers: 0 global (read), 1 global (written),
    2 shared int32 (a tile, one word per thread), 3 shared bytes.  Threads
    store loaded values, coordinates and arguments into the tiles at their
    own or a neighbour's slot, read other threads' slots after a barrier,
    and store what they read.  With `live`, some values read from a tile
    also become indices or branch conditions, so the barriers matter; without
    it, no value read from a tile reaches a check (BarrierElimination
    applies)."""
    rng = SplitMix64(sub_seed("barprog", 2 * index + (1 if live else 0)))
    A = Asm(n_bufs=4, shared_mask=0b1100, seed=rng.next32(), shared_stores=True)
    tx, ty, ntx = A.sreg(bc.TID_X), A.sreg(bc.TID_Y), A.sreg(bc.NTID_X)
    args = [A.sreg(bc.ARG0 + k) for k in range(4)]
    t = A.alu(bc.ADD, A.alu(bc.MUL, ty, ntx), tx)
    T = A.alu(bc.MUL, ntx, A.sreg(bc.NTID_Y))
    gid = A.alu(bc.ADD, A.alu(bc.MUL, A.sreg(bc.CTAID_X), T), t)
    read = []            # values read from the tiles so far

    def slot():
        r = rng.below(6)
        if r == 0:
            return t
        if r == 1:
            return A.alu(bc.ADD, t, Imm(1))
        if r == 2:
            return A.alu(bc.XOR, t, Imm(1))
        if r == 3:
            return A.alu(bc.SUB, A.alu(bc.SUB, T, Imm(1)), t)
        if r == 4:
            return A.alu(bc.ADD, t, rng.choice(args))
        return A.alu(bc.AND, A.alu(bc.MUL, t, Imm(rng.choice((2, 3, 5)))), Imm(31))

    def value():
        r = rng.below(5)
        if r == 0:
            return A.ld(0, gid, rng.choice((1, 4)))
        if r == 1:
            return A.alu(bc.MUL, t, Imm(rng.randint(1, 4)))
        if r == 2 and read:
            return A.alu(bc.ADD, rng.choice(read), Imm(rng.randint(-2, 2)))
        return A.alu(bc.ADD, rng.choice(args), t)

    def use(v):
        """A value read from a tile: stored on, or (live) a check."""
        if live and rng.below(2):
            if rng.below(2):
                A.ld(rng.choice((0, 1)), A.alu(bc.SUB, v, rng.choice(args)), 4)
            else:
                A.if_(A.alu(bc.SETLT, v, rng.choice(args)))
                A.ld(0, t, 4)
                A.endif()
        elif rng.below(2):
            A.st(1, gid, A.alu(bc.XOR, v, t), 4)
        else:
            read.append(v)

    def statement(depth):
        r = rng.below(7)
        if r <= 1:
            A.st(2, slot(), value(), 4)
        elif r == 2:
            A.st(3, slot(), value(), 1)
        elif r == 3:
            use(A.ld(2, slot(), 4))
        elif r == 4:
            use(A.ld(3, slot(), 1))
        elif r == 5 and depth == 0:
            A.if_(A.alu(bc.SETLT, t, rng.choice(args)))
            statement(1)
            A.endif()
        elif depth == 0:
            k = A.loop(A.alu(bc.AND, rng.choice(args), Imm(3)), 3)
            A.st(2, A.alu(bc.ADD, t, k), A.alu(bc.MUL, k, t), 4)
            A.endloop()
        else:
            A.st(1, gid, t, 4)

    for phase in range(rng.randint(2, 4)):
        if phase:
            A.bar()
        for _ in range(rng.randint(2, 5)):
            statement(0)
    if live:             # at least one read value is a check
        A.bar()
        A.ld(1, A.alu(bc.SUB, A.ld(2, A.alu(bc.XOR, t, Imm(1)), 4), args[0]), 4)
    return A.build()


def barrier_programs(n: int = 16, live: bool = False) -> list[bytes]:
    return [barrier_program(i, live) for i in range(n)]


def barrier_inputs(n: int, n_programs: int = 16, seed: int | None = None,
                   max_blocks: int = 3) -> np.ndarray:
    """Blocks from BAR_BLOCKS, 1D grids up to max_blocks; arguments from
    {0, +-1, 2, 3, 5, 8, 16}; global buffers up to 256 bytes; the int32
    tile one word per thread (+-1 word), the byte tile one byte per thread
    (+-1)."""
    rng = SplitMix64(sub_seed("barrier") if seed is None else seed)
    out = make_inputs(n)
    for k in range(n):
        blk = rng.choice(BAR_BLOCKS)
        T = blk[0] * blk[1] * blk[2]
        args = [rng.choice((0, 1, -1, 2, 3, 5, 8, 16)) for _ in range(4)]
        lens = [rng.randint(0, 256), rng.randint(0, 256), 4 * (T + rng.randint(-1, 1)),
                T + rng.randint(-1, 1)]
        set_input(out[k], k % n_programs, (rng.randint(1, max_blocks), 1, 1), blk, args, lens,
                  tag=k)
    return out


# --------------------------------------------------------------------------
# config 2: random 2D programs with shared buffers and loops
# --------------------------------------------------------------------------

_C2_ALU = (bc.ADD, bc.MUL, bc.SHL, bc.AND, bc.MIN, bc.MAX, bc.SUB, bc.XOR, bc.SHR, bc.OR)


def c2_program(index: int) -> bytes:
    """One seeded random access program: 20-200 ops over thread/block ids and
    four scalar args; at most two non-nested loops (trip <= 64); 2-6 global
    and 1-3 shared buffers with per-buffer widths from {1,4,8,16}."""
    rng = SplitMix64(sub_seed("c2prog", index))
    n_glob = rng.randint(2, 6)
    n_sh = rng.randint(1, 3)
    n_bufs = n_glob + n_sh
    shared_mask = ((1 << n_sh) - 1) << n_glob
    widths = [rng.choice(bc.WIDTHS) for _ in range(n_bufs)]
    target = rng.randint(20, 200)
    A = Asm(n_bufs, shared_mask, seed=rng.next32())

    tx, ty = A.sreg(bc.TID_X), A.sreg(bc.TID_Y)
    bx, by = A.sreg(bc.CTAID_X), A.sreg(bc.CTAID_Y)
    nx = A.sreg(bc.NTID_X)
    gxn = A.sreg(bc.NCTAID_X)
    args = [A.sreg(bc.ARG0 + k) for k in range(4)]
    gx = A.alu(bc.ADD, A.alu(bc.MUL, bx, nx), tx)
    ny = A.sreg(bc.NTID_Y)
    gy = A.alu(bc.ADD, A.alu(bc.MUL, by, ny), ty)
    row = A.alu(bc.MUL, gxn, nx)
    lin = A.alu(bc.ADD, A.alu(bc.MUL, gy, row), gx)
    tlin = A.alu(bc.ADD, A.alu(bc.MUL, ty, nx), tx)
    idx_pool = [gx, gy, lin, lin, lin, tlin]
    val_pool = [tx, ty, bx, by] + args
    loops = [0]

    def small_imm():
        return Imm(rng.choice((1, 2, 3, 4, 7, 8, 15, 16, 31, 32, 255, -1, -4)))

    def pick_val():
        return rng.choice(val_pool + idx_pool)

    def math_stmt():
        op = rng.choice(_C2_ALU)
        a = pick_val()
        if rng.chance(0.5):
            b = small_imm()
            if op in (bc.SHL, bc.SHR):
                b = Imm(rng.randint(0, 4))
        else:
            b = pick_val()
        v = A.alu(op, a, b)
        (idx_pool if rng.chance(0.3) else val_pool).append(v)

    def index_expr(buf, ctr=None):
        shared = (shared_mask >> buf) & 1
        base = tlin if shared else rng.choice(idx_pool)
        kind = rng.below(6)
        if kind == 0:
            idx = A.alu(bc.ADD, base, rng.choice(args))
        elif kind == 1:
            idx = A.alu(bc.ADD, base, Imm(rng.randint(-2, 2)))
        elif kind == 2:
            idx = A.alu(bc.MIN, base, rng.choice(args))
        elif kind == 3:
            idx = A.alu(bc.AND, base, rng.choice(args + [A.imm(rng.choice((255, 1023, 65535)))]))
        elif kind == 4:
            idx = A.alu(bc.SUB, base, A.alu(bc.AND, rng.choice(args), Imm(7)))
        else:
            idx = base
        if ctr is not None:
            idx = A.alu(bc.ADD, idx, A.alu(bc.MUL, ctr, Imm(rng.choice((1, 16, 256)))))
        return idx

    def access_stmt(ctr=None):
        buf = rng.below(n_bufs)
        idx = index_expr(buf, ctr)
        w = widths[buf]
        if rng.chance(0.6):
            v = A.ld(buf, idx, w)
            val_pool.append(v)
        else:
            A.st(buf, idx, pick_val(), w)

    def if_stmt(depth, in_loop):
        c = A.alu(rng.choice((bc.SETLT, bc.SETNE, bc.SETLE, bc.SETEQ)), pick_val(),
                  rng.choice(args + [pick_val()]))
        A.if_(c)
        block(depth + 1, in_loop, rng.randint(1, 4))
        if rng.chance(0.3):
            A.else_()
            block(depth + 1, in_loop, rng.randint(1, 3))
        A.endif()

    def loop_stmt(depth):
        loops[0] += 1
        n = rng.choice(args + [A.imm(rng.randint(0, 64))])
        ctr = A.loop(n, rng.randint(1, 64))
        for _ in range(rng.randint(1, 3)):
            if rng.chance(0.6):
                access_stmt(ctr)
            else:
                math_stmt()
        A.endloop()

    def block(depth, in_loop, count):
        for _ in range(count):
            if len(A.ops) >= target - 2 * (A.depth + 1):
                return
            r = rng.uniform()
            if r < 0.35:
                math_stmt()
            elif r < 0.75:
                access_stmt()
            elif r < 0.9 and depth < 3:
                if_stmt(depth, in_loop)
            elif not in_loop and loops[0] < 2 and depth < 2:
                loop_stmt(depth)
            else:
                access_stmt()

    while len(A.ops) < target - 2:
        block(0, False, 1)
    return A.build()


def c2_programs(n: int = 32) -> list[bytes]:
    return [c2_program(i) for i in range(n)]


_INTERESTING_ARGS = (0, -1, 1)


def interesting_arg(rng: SplitMix64) -> int:
    k = rng.randint(0, 30)
    base = 1 << k
    return rng.choice((0, -1, 1, base, base + 1, base - 1, -base))


def c2_inputs(programs: list[bytes], per_program: int = 256, seed: int | None = None,
              max_grid: int = 256) -> np.ndarray:
    """Per program: 2D grids with gx, gy log-uniform in [1, 256] of 16x16
    blocks; args uniform int32 (p=0.5) or from {0,-1,1,2^k,2^k+-1,-2^k};
    global lengths log-uniform in [1 B, 16 MiB]; shared lengths B*w + d,
    d in {-w, 0, +w}."""
    rng = SplitMix64(sub_seed("c2") if seed is None else seed)
    out = make_inputs(len(programs) * per_program)
    k = 0
    for p, prog in enumerate(programs):
        h = bc.decode_header(prog)
        # the per-buffer element width: the widest access to each buffer
        wmax = [1] * h["n_bufs"]
        for opc, _d, _a, b, imm in bc.ops_of(prog):
            if opc in (bc.LD, bc.ST):
                wmax[b] = max(wmax[b], imm)
        for _j in range(per_program):
            gx = rng.loguniform_int(1, max_grid)
            gy = rng.loguniform_int(1, max_grid)
            args = [(rng.next32() - (1 << 31)) if rng.chance(0.5) else interesting_arg(rng)
                    for _ in range(4)]
            lens = []
            for b in range(h["n_bufs"]):
                if (h["shared_mask"] >> b) & 1:
                    w = wmax[b]
                    lens.append(max(256 * w + rng.choice((-w, 0, w)), 0))
                else:
                    lens.append(rng.loguniform_int(1, 16 << 20))
            set_input(out[k], p, (gx, gy, 1), (16, 16, 1), args, lens, tag=k)
            k += 1
    return out


# --------------------------------------------------------------------------
# config 4: branch-heavy programs with data-dependent conditions
# --------------------------------------------------------------------------

def c4_program(index: int, n_sites_max: int = 64) -> bytes:
    """Up to 64 branch sites whose conditions read the args and int32 values
    loaded from a seeded global table (buffer 0), nested at most 4 deep;
    buffers 1 and 2 are outputs written under the branches.  Temporaries
    cycle through a small register pool, as compiled code reuses registers."""
    rng = SplitMix64(sub_seed("c4prog", index))
    A = Asm(n_bufs=3, seed=rng.next32())
    tx = A.sreg(bc.TID_X)
    bx = A.sreg(bc.CTAID_X)
    nx = A.sreg(bc.NTID_X)
    args = [A.sreg(bc.ARG0 + k) for k in range(4)]
    i = A.alu(bc.ADD, A.alu(bc.MUL, bx, nx), tx)
    tmask = A.alu(bc.AND, i, Imm(4095))
    v = A.ld(0, tmask, 4)
    vals = [v, i, tx]
    vslots = [A.new_reg() for _ in range(6)]
    temps = [A.new_reg() for _ in range(8)]
    tnext = [0]
    n_target = rng.randint(max(n_sites_max // 2, 1), n_sites_max)
    sites = [0]

    def tmp():
        t = temps[tnext[0] % len(temps)]
        tnext[0] += 1
        return t

    def cond():
        r = rng.below(5)
        x = rng.choice(vals)
        if r == 0:
            m = A.alu(bc.AND, x, Imm(1 << rng.randint(0, 30)), dst=tmp())
            return A.alu(bc.SETNE, m, A.imm(0, dst=tmp()), dst=tmp())
        if r == 1:
            return A.alu(bc.SETLT, x, rng.choice(args), dst=tmp())
        if r == 2:
            m = rng.choice((3, 7, 15))
            p = A.alu(bc.AND, x, Imm(m), dst=tmp())
            q = A.alu(bc.AND, rng.choice(args), Imm(m), dst=tmp())
            return A.alu(bc.SETEQ, p, q, dst=tmp())
        if r == 3:
            p = A.alu(bc.SHRU, x, Imm(rng.randint(1, 28)), dst=tmp())
            return A.alu(bc.SETLE, p, rng.choice(args), dst=tmp())
        p = A.alu(bc.ADD, rng.choice(args), Imm(rng.randint(0, 1 << 20)), dst=tmp())
        return A.alu(bc.SETLTU, x, p, dst=tmp())

    def body(depth):
        while sites[0] < n_target:
            sites[0] += 1
            A.if_(cond())
            if rng.chance(0.5):
                a = A.alu(bc.ADD, rng.choice(vals), rng.choice(args), dst=tmp())
                a = A.alu(bc.AND, a, Imm(4095), dst=tmp())
                slot = rng.below(len(vslots))
                nv = A.ld(0, a, 4, dst=vslots[slot])
                if nv not in vals:
                    vals.append(nv)
            if rng.chance(0.3):
                A.st(1, A.alu(bc.AND, i, Imm(1023), dst=tmp()), rng.choice(vals), 4)
            if depth < 4 and rng.chance(0.45):
                body(depth + 1)
            if rng.chance(0.3):
                A.else_()
                A.st(2, A.alu(bc.ADD, tmask, rng.choice(args), dst=tmp()), rng.choice(vals), 4)
            A.endif()
            if depth > 0 and rng.chance(0.5):
                return

    body(0)
    return A.build()


def c4_programs(n: int = 16) -> list[bytes]:
    return [c4_program(i) for i in range(n)]


def c4_inputs(n: int = 16384, n_programs: int = 16, seed: int | None = None,
              max_blocks: int = 1024) -> np.ndarray:
    rng = SplitMix64(sub_seed("c4") if seed is None else seed)
    out = make_inputs(n)
    for k in range(n):
        p = k % n_programs
        nb = rng.loguniform_int(1, max_blocks)
        args = [(rng.next32() - (1 << 31)) if rng.chance(0.3) else
                (interesting_arg(rng) if rng.chance(0.5) else rng.randint(0, 1 << 16))
                for _ in range(4)]
        lens = [4 * 4096, 4 * rng.choice((1024, 1023, 1025)), 4 * rng.loguniform_int(1, 1 << 20)]
        set_input(out[k], p, (nb, 1, 1), (256, 1, 1), args, lens, tag=k)
    return out


# --------------------------------------------------------------------------
# config 5: serving mix and the mutator
# --------------------------------------------------------------------------

_INTERESTING_LENS = (0, 1, 2, 3, 4, 7, 8, 15, 16, 17, 31, 32, 63, 64, 100, 127, 128, 129,
                     255, 256, 511, 512, 1000, 1023, 1024, 4095, 4096, 65535, 65536)


class Mutator:
    """Seeded mutator over scalar args and buffer lengths: single bit flips,
    add/subtract 1..35, and substitution from a small set of boundary
    values.  Grid and block shapes are left alone."""

    def __init__(self, seed: int):
        self.rng = SplitMix64(seed)

    def mutate(self, rec, n_bufs: int) -> None:
        rng = self.rng
        n_fields = 4 + max(n_bufs, 0)
        for _ in range(1 + rng.below(3)):
            f = rng.below(n_fields)
            kind = rng.below(3)
            if f < 4:
                v = int(rec["args"][f])
                if kind == 0:
                    v ^= 1 << rng.below(32)
                elif kind == 1:
                    d = rng.randint(1, 35)
                    v = v + d if rng.chance(0.5) else v - d
                else:
                    v = interesting_arg(rng)
                rec["args"][f] = ((v + (1 << 31)) % (1 << 32)) - (1 << 31)
            else:
                b = f - 4
                v = int(rec["buf_len"][b])
                if kind == 0:
                    v ^= 1 << rng.below(24)
                elif kind == 1:
                    d = rng.randint(1, 35)
                    v = v + d if rng.chance(0.5) else max(v - d, 0)
                else:
                    v = rng.choice(_INTERESTING_LENS)
                rec["buf_len"][b] = v


def child_stream(seed: int, round_: int, j: int) -> int:
    """SplitMix64 state of child j's mutation stream in round `round_` of a
    campaign (one stream per child)."""
    return (seed + (((round_ << 32) | j) * 0xD1B54A32D192ED03)) & MASK64


def c5_programs() -> list[bytes]:
    """64 resident programs: 16 of config 3's family, 32 random (config 2
    generator with fresh seeds), 16 branch-heavy (config 4 generator)."""
    progs = c3_programs()
    progs += [c2_program(1000 + i) for i in range(32)]
    progs += [c4_program(1000 + i) for i in range(16)]
    return progs


def c5_corpus(programs: list[bytes], per_program: int = 4, seed: int | None = None,
              max_blocks: int = 4096) -> np.ndarray:
    """Seed corpus: per program a few inputs with total blocks log-uniform in
    [1, 4096] and block sizes log-uniform in [32, 1024] (2D programs use
    16 x 16 blocks and a near-square grid)."""
    rng = SplitMix64(sub_seed("c5corpus") if seed is None else seed)
    out = make_inputs(len(programs) * per_program)
    k = 0
    for p, prog in enumerate(programs):
        h = bc.decode_header(prog)
        two_d = any(o[0] == bc.SREG and o[4] == bc.TID_Y for o in bc.ops_of(prog))
        wmax = [1] * h["n_bufs"]
        for opc, _d, _a, b, imm in bc.ops_of(prog):
            if opc in (bc.LD, bc.ST):
                wmax[b] = max(wmax[b], imm)
        for _j in range(per_program):
            nb = rng.loguniform_int(1, max_blocks)
            if two_d:
                gx = max(int(math.sqrt(nb)), 1)
                grid, block = (gx, max(nb // gx, 1), 1), (16, 16, 1)
            else:
                grid, block = (nb, 1, 1), (rng.loguniform_int(32, 1024), 1, 1)
            total = grid[0] * grid[1] * block[0] * block[1]
            args = [rng.randint(-4, 4), rng.randint(0, total), rng.randint(0, 1 << 16),
                    interesting_arg(rng)]
            lens = []
            for b in range(h["n_bufs"]):
                if (h["shared_mask"] >> b) & 1:
                    lens.append(block[0] * block[1] * wmax[b])
                else:
                    lens.append(wmax[b] * rng.randint(max(total - 2, 0), total + 2))
            set_input(out[k], p, grid, block, args, lens, tag=k)
            k += 1
    return out


def program_bufs(programs: list[bytes]) -> list[int]:
    return [bc.decode_header(p)["n_bufs"] for p in programs]


def c5_stream(programs: list[bytes], corpus: np.ndarray, n: int, seed: int | None = None) -> np.ndarray:
    """n mutated inputs: each takes a uniformly chosen corpus entry and
    applies 1-3 mutations."""
    rng = SplitMix64(sub_seed("c5pick") if seed is None else seed)
    mut = Mutator(sub_seed("c5mut") if seed is None else seed ^ 0x5A5A)
    nb = program_bufs(programs)
    out = make_inputs(n)
    for k in range(n):
        src = corpus[rng.below(len(corpus))]
        out[k] = src
        mut.mutate(out[k], nb[int(src["program_id"])])
        out[k]["user_tag"] = k
    return out


def poisson_arrivals(rate: float, duration_s: float, seed: int) -> np.ndarray:
    """Open-loop arrival times (seconds) of a Poisson process."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    while True:
        u = max(rng.uniform(), 1e-300)
        t += -math.log(u) / rate
        if t >= duration_s:
            break
        out.append(t)
    return np.asarray(out, dtype=np.float64)


def total_threads(inputs: np.ndarray) -> np.ndarray:
    g = inputs["grid"].astype(np.float64)
    b = inputs["block"].astype(np.float64)
    return g.prod(axis=1) * b.prod(axis=1)
