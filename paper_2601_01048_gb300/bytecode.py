"""Wire format of a kernel-under-test program, and an assembler for it.

A program is the integer *access-index program* of one CUDA kernel: the
instructions that compute memory-access indices and branch conditions from
threadIdx/blockIdx/blockDim/gridDim and scalar arguments, the loads and
stores of a given width to numbered buffers, and structured control flow
(IF/ELSE/ENDIF, bounded LOOP/ENDLOOP).  It is what the paper's kernel
translator keeps of a kernel when only memory behaviour matters (Sec. 5,
"does not require output equivalence"; Alg. 2 keeps exactly the operations
used as an index or in a branch).

This module only *encodes*: it holds none of the checking, coverage or
pruning arithmetic.  Both the CPU oracle and the device loader decode the
bytes with decoders of their own.

Layout (little endian):

    header, 32 bytes
      u32 magic   = 0x315A4643 ("CFZ1")
      u16 version = 1
      u16 n_ops               (1 .. 2048)
      u8  n_regs              virtual i32 registers r0 .. r(n_regs-1)
      u8  n_bufs              buffers 0 .. n_bufs-1, at most 9
      u8  n_sites             number of IF + LOOP ops (branch sites)
      u8  reserved (0)
      u16 shared_mask         bit k set: buffer k lives in block-shared space
      u16 reserved (0)
      u32 seed                content seed of the global buffers
      u32 reserved[3] (0)
    LOC table, n_sites x 2 x u16   LOC[s][0] (not taken / exit), LOC[s][1]
    ops, n_ops x 8 bytes           u8 opcode, u8 dst, u8 a, u8 b, i32 imm

Total size is exactly 32 + 4*n_sites + 8*n_ops bytes.

Opcodes and the fields they use (unused fields must be 0):

    SREG  dst, imm=id          id: 0-2 tid.xyz, 3-5 ntid.xyz, 6-8 ctaid.xyz,
                               9-11 nctaid.xyz, 12-15 arg0..arg3
    IMM   dst, imm             dst = imm
    MOV   dst, a               dst = a
    SEL   dst, a, b, imm=y     dst = a != 0 ? b : y   (y is a register, 0..255)
    DIV   dst, a, b            dst = a / b, signed, truncating (0x05)
    REM   dst, a, b            dst = a % b, signed, truncating (0x06); for both a
                               zero divisor is a fault (result 0), and
                               INT_MIN / -1 = INT_MIN, INT_MIN % -1 = 0
    HALLOC dst, a              heap block of a bytes (0x07): dst = its handle
                               (allocation site + 1), or 0 when a <= 0
    HFREE a                    free the block of handle a (0x08); 0 is a no-op
    HLD   dst, a=idx, b=handle, imm=width   heap load (0x42), reads 0
    HST   dst=value, a=idx, b=handle, imm=width   heap store (0x43)
    ALU   dst, a, b            opcode 0x10-0x1F, register b
    ALUI  dst, a, imm          opcode 0x30-0x3F, immediate b
    LD    dst, a=idx, b=buf, imm=width in {1,4,8,16}
    ST    dst=value, a=idx, b=buf, imm=width
    IF    a=cond
    ELSE, ENDIF
    LOOP  dst=ctr, a=n, imm=max_trip (0..65535)
    ENDLOOP
    BAR                        block-wide barrier (0x55), top level only

Header byte 11 holds flags; bit 0 (PF_SHARED_STORES) makes stores to shared
buffers performed: each block's shared buffers start as zero bytes, an
in-bounds ST writes the value's little-endian bytes (width 1: the low byte;
widths 8 and 16: the four bytes, then zeros) and an in-bounds LD reads them
(width 1: the byte, zero-extended; wider: the int32 of the first four
bytes).  The BARs split the program into phases that a block runs for all
of its threads, in thread order, one phase after another.  Without the flag
stores are never performed, shared loads read 0 and BAR does nothing.

The k-th LD/ST in program order is access site k; the k-th IF/LOOP is branch
site k; the k-th DIV/REM is division site k.  HLD/HST share the access
sites with LD/ST; the k-th HALLOC is allocation site k, the k-th HFREE free
site k.
"""
from __future__ import annotations

import struct
from dataclasses import dataclass

MAGIC = 0x315A4643
VERSION = 1
HEADER_BYTES = 32
OP_BYTES = 8
MAX_OPS = 2048
MAX_BUFS = 9
MAX_DEPTH = 16

# opcodes
NOP = 0x00
SREG = 0x01
IMM = 0x02
MOV = 0x03
SEL = 0x04
DIV = 0x05
REM = 0x06
HALLOC = 0x07
HFREE = 0x08
ADD, SUB, MUL, SHL, SHR, SHRU, AND, OR, XOR, MIN, MAX, SETLT, SETLE, SETEQ, SETNE, SETLTU = range(0x10, 0x20)
IMM_FORM = 0x20
LD = 0x40
ST = 0x41
HLD = 0x42
HST = 0x43
IF = 0x50
ELSE = 0x51
ENDIF = 0x52
LOOP = 0x53
ENDLOOP = 0x54
BAR = 0x55

# header byte 11: program flags
PF_SHARED_STORES = 1   # stores to shared buffers are performed; BARs order them

ALU_NAMES = {
    ADD: "add", SUB: "sub", MUL: "mul", SHL: "shl", SHR: "shr", SHRU: "shru",
    AND: "and", OR: "or", XOR: "xor", MIN: "min", MAX: "max", SETLT: "setlt",
    SETLE: "setle", SETEQ: "seteq", SETNE: "setne", SETLTU: "setltu",
}

# special registers
TID_X, TID_Y, TID_Z, NTID_X, NTID_Y, NTID_Z = range(6)
CTAID_X, CTAID_Y, CTAID_Z, NCTAID_X, NCTAID_Y, NCTAID_Z = range(6, 12)
ARG0, ARG1, ARG2, ARG3 = range(12, 16)

WIDTHS = (1, 4, 8, 16)


@dataclass(frozen=True)
class Imm:
    """An immediate operand for the ALU immediate forms."""
    value: int


def _i32(v: int) -> int:
    v &= 0xFFFFFFFF
    return v - (1 << 32) if v & 0x80000000 else v


class Asm:
    """Builds a program op by op with structured control flow.

    Registers are allocated fresh for every result (SSA-like), so a generated
    program never reads a register before writing it unless asked to via
    :meth:`raw`.
    """

    def __init__(self, n_bufs: int, shared_mask: int = 0, seed: int = 0,
                 shared_stores: bool = False):
        if not 0 <= n_bufs <= MAX_BUFS:
            raise ValueError("n_bufs out of range")
        self.n_bufs = n_bufs
        self.shared_mask = shared_mask
        self.flags = PF_SHARED_STORES if shared_stores else 0
        self.seed = seed & 0xFFFFFFFF
        self.ops: list[tuple[int, int, int, int, int]] = []
        self.n_regs = 0
        self._stack: list[str] = []
        self.n_sites = 0
        self.n_access = 0

    # -- registers -------------------------------------------------------
    def new_reg(self) -> int:
        r = self.n_regs
        if r >= 255:
            raise ValueError("out of registers")
        self.n_regs += 1
        return r

    def raw(self, opc: int, dst: int = 0, a: int = 0, b: int = 0, imm: int = 0) -> None:
        """Append one op verbatim (used by tests to build odd programs)."""
        self.ops.append((opc, dst, a, b, _i32(imm)))

    # -- value ops ----------------------------------------------------------
    def _dst(self, dst):
        return self.new_reg() if dst is None else dst

    def sreg(self, sid: int, dst: int | None = None) -> int:
        d = self._dst(dst)
        self.raw(SREG, d, 0, 0, sid)
        return d

    def imm(self, value: int, dst: int | None = None) -> int:
        d = self._dst(dst)
        self.raw(IMM, d, 0, 0, value)
        return d

    def mov(self, a: int, dst: int | None = None) -> int:
        d = self._dst(dst)
        self.raw(MOV, d, a)
        return d

    def alu(self, op: int, a: int, b, dst: int | None = None) -> int:
        d = self._dst(dst)
        if isinstance(b, Imm):
            self.raw(op | IMM_FORM, d, a, 0, b.value)
        else:
            self.raw(op, d, a, b, 0)
        return d

    def div(self, a: int, b: int, dst: int | None = None) -> int:
        d = self._dst(dst)
        self.raw(DIV, d, a, b)
        return d

    def rem(self, a: int, b: int, dst: int | None = None) -> int:
        d = self._dst(dst)
        self.raw(REM, d, a, b)
        return d

    def halloc(self, size: int, dst: int | None = None) -> int:
        d = self._dst(dst)
        self.raw(HALLOC, d, size)
        return d

    def hfree(self, handle: int) -> None:
        self.raw(HFREE, 0, handle)

    def hld(self, handle: int, idx: int, width: int = 4, dst: int | None = None) -> int:
        d = self._dst(dst)
        self.raw(HLD, d, idx, handle, width)
        self.n_access += 1
        return d

    def hst(self, handle: int, idx: int, val: int, width: int = 4) -> None:
        self.raw(HST, val, idx, handle, width)
        self.n_access += 1

    def sel(self, c: int, x: int, y: int, dst: int | None = None) -> int:
        d = self._dst(dst)
        self.raw(SEL, d, c, x, y)
        return d

    # -- memory ---------------------------------------------------------------
    def ld(self, buf: int, idx: int, width: int = 4, dst: int | None = None) -> int:
        d = self._dst(dst)
        self.raw(LD, d, idx, buf, width)
        self.n_access += 1
        return d

    def st(self, buf: int, idx: int, val: int, width: int = 4) -> None:
        self.raw(ST, val, idx, buf, width)
        self.n_access += 1

    # -- control --------------------------------------------------------------
    def if_(self, cond: int) -> None:
        self.raw(IF, 0, cond)
        self._stack.append("if")
        self.n_sites += 1

    def else_(self) -> None:
        if not self._stack or self._stack[-1] != "if":
            raise ValueError("ELSE outside IF")
        self._stack[-1] = "else"
        self.raw(ELSE)

    def endif(self) -> None:
        if not self._stack or self._stack[-1] not in ("if", "else"):
            raise ValueError("ENDIF outside IF")
        self._stack.pop()
        self.raw(ENDIF)

    def loop(self, n: int, max_trip: int) -> int:
        ctr = self.new_reg()
        self.raw(LOOP, ctr, n, 0, max_trip)
        self._stack.append("loop")
        self.n_sites += 1
        return ctr

    def endloop(self) -> None:
        if not self._stack or self._stack[-1] != "loop":
            raise ValueError("ENDLOOP outside LOOP")
        self._stack.pop()
        self.raw(ENDLOOP)

    def bar(self) -> None:
        if self._stack:
            raise ValueError("BAR inside IF/LOOP")
        self.raw(BAR)

    @property
    def depth(self) -> int:
        return len(self._stack)

    # -- encoding -----------------------------------------------------------
    def build(self, loc: list[tuple[int, int]] | None = None) -> bytes:
        if self._stack:
            raise ValueError("unterminated IF/LOOP")
        n_sites = sum(1 for o in self.ops if o[0] in (IF, LOOP))
        if loc is None:
            loc = default_loc(self.seed, n_sites)
        if len(loc) != n_sites:
            raise ValueError("LOC table size does not match the branch sites")
        return encode(self.ops, max(self.n_regs, 1), self.n_bufs, self.shared_mask,
                      self.seed, loc, self.flags)


def default_loc(seed: int, n_sites: int) -> list[tuple[int, int]]:
    """Per-site random 16-bit locations, drawn from the program seed."""
    from .gen import SplitMix64  # local import: gen imports this module

    rng = SplitMix64(seed ^ 0x10C0C0FFEE)
    return [((rng.next() >> 48) & 0xFFFF, (rng.next() >> 48) & 0xFFFF) for _ in range(n_sites)]


def encode(ops, n_regs: int, n_bufs: int, shared_mask: int, seed: int,
           loc: list[tuple[int, int]], flags: int = 0) -> bytes:
    out = bytearray()
    out += struct.pack("<IHHBBBBHHIIII", MAGIC, VERSION, len(ops), n_regs, n_bufs,
                       len(loc), flags, shared_mask, 0, seed & 0xFFFFFFFF, 0, 0, 0)
    assert len(out) == HEADER_BYTES
    for l0, l1 in loc:
        out += struct.pack("<HH", l0 & 0xFFFF, l1 & 0xFFFF)
    for opc, dst, a, b, imm in ops:
        out += struct.pack("<BBBBi", opc, dst, a, b, _i32(imm))
    return bytes(out)


def decode_header(prog: bytes) -> dict:
    (magic, version, n_ops, n_regs, n_bufs, n_sites, flags, shared_mask, _r1, seed,
     _r2, _r3, _r4) = struct.unpack_from("<IHHBBBBHHIIII", prog, 0)
    return dict(magic=magic, version=version, n_ops=n_ops, n_regs=n_regs, n_bufs=n_bufs,
                n_sites=n_sites, shared_mask=shared_mask, seed=seed, flags=flags)


def ops_of(prog: bytes) -> list[tuple[int, int, int, int, int]]:
    h = decode_header(prog)
    off = HEADER_BYTES + 4 * h["n_sites"]
    return [struct.unpack_from("<BBBBi", prog, off + OP_BYTES * i) for i in range(h["n_ops"])]


def loc_of(prog: bytes) -> list[tuple[int, int]]:
    h = decode_header(prog)
    return [struct.unpack_from("<HH", prog, HEADER_BYTES + 4 * s) for s in range(h["n_sites"])]


def disasm(prog: bytes) -> str:
    lines = []
    for pc, (opc, dst, a, b, imm) in enumerate(ops_of(prog)):
        base = opc & ~IMM_FORM if 0x30 <= opc <= 0x3F else opc
        if base in ALU_NAMES:
            rhs = f"#{imm}" if opc & IMM_FORM else f"r{b}"
            lines.append(f"{pc:4d}  r{dst} = {ALU_NAMES[base]} r{a}, {rhs}")
        elif opc == SREG:
            lines.append(f"{pc:4d}  r{dst} = sreg {imm}")
        elif opc == IMM:
            lines.append(f"{pc:4d}  r{dst} = #{imm}")
        elif opc == MOV:
            lines.append(f"{pc:4d}  r{dst} = r{a}")
        elif opc == SEL:
            lines.append(f"{pc:4d}  r{dst} = r{a} ? r{b} : r{imm}")
        elif opc in (DIV, REM):
            lines.append(f"{pc:4d}  r{dst} = {'div' if opc == DIV else 'rem'} r{a}, r{b}")
        elif opc == HALLOC:
            lines.append(f"{pc:4d}  r{dst} = halloc r{a}")
        elif opc == HFREE:
            lines.append(f"{pc:4d}  hfree r{a}")
        elif opc == HLD:
            lines.append(f"{pc:4d}  r{dst} = hld.w{imm} heap[r{b}][r{a}]")
        elif opc == HST:
            lines.append(f"{pc:4d}  hst.w{imm} heap[r{b}][r{a}] = r{dst}")
        elif opc == LD:
            lines.append(f"{pc:4d}  r{dst} = ld.w{imm} buf{b}[r{a}]")
        elif opc == ST:
            lines.append(f"{pc:4d}  st.w{imm} buf{b}[r{a}] = r{dst}")
        elif opc == IF:
            lines.append(f"{pc:4d}  if r{a}")
        elif opc == LOOP:
            lines.append(f"{pc:4d}  loop r{dst} < clamp(r{a}, 0, {imm})")
        elif opc == BAR:
            lines.append(f"{pc:4d}  bar")
        elif opc in (ELSE, ENDIF, ENDLOOP):
            lines.append(f"{pc:4d}  {({ELSE: 'else', ENDIF: 'endif', ENDLOOP: 'endloop'})[opc]}")
        else:
            lines.append(f"{pc:4d}  op{opc:#x} {dst} {a} {b} {imm}")
    return "\n".join(lines)
