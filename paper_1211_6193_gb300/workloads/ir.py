"""Encoding of the simulated-kernel IR, a small assembler, and the program container.

The paper interprets CUDA-C source directly (Sec. 3, "Threads and memory"): every
thread of a grid runs the kernel body, reading ``threadIdx``/``blockIdx``/``blockDim``
(Sec. 3, list of supported features), touching global and per-block shared memory
(Sec. 3, "Threads and memory") and meeting at ``__syncthreads()`` (Sec. 3, "Barrier
synchronization").  This project runs the same kind of program written in a small
int32 register IR instead of C.  This module only *encodes* programs; it contains
no interpretation logic.  Both the CUDA library and the CPU oracle decode the same
byte layout, each with its own independently written decoder.

Instruction word (8 bytes, little endian)::

    uint32 op_d_a_b = op | d << 8 | a << 16 | b << 24
    int32  imm

``op`` bits 0..5 hold the opcode, bit 7 (``BIMM``) says that the second ALU operand
is ``imm`` instead of register ``b``.  Registers are ``r0..r15``; ``RZ`` (255) reads
as zero and drops writes.  Word addresses everywhere (global arena and shared array
are int32 words).

Opcodes and operand use::

    MOV d, B             d = B
    ADD..SNE d, a, B     d = a OP B          (B = reg b, or imm when BIMM)
    S2R d, #sreg         d = TID | BID | BDIM | GDIM | WARPSIZE
    LDG d, [a + imm]     global load          STG [a + imm], b   global store
    LDS d, [a + imm]     shared load          STS [a + imm], b   shared store
    ATOMS [a + imm], b   shared atomic add, no return value
    BRA #t   BRZ a, #t   BRNZ a, #t           absolute targets (program pc)
    BAR                  __syncthreads()
    EXIT                 thread exits; running past the last instruction also exits
    BARAND d, a          __syncthreads_and(a): d = 1 if a != 0 in every thread released
    BAROR d, a           __syncthreads_or(a):  d = 1 if a != 0 in some thread released
    BARPOPC d, a         __syncthreads_count(a): d = number of released threads with a != 0
                         (Sec. 3 feature list; threads released from a plain BAR count as 0)
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Sequence, Tuple, Union

import numpy as np

# ---------------------------------------------------------------- opcode table
MOV, ADD, SUB, MUL, DIV, REM, AND, OR, XOR, SHL, SHR, MIN, MAX, SLT, SLE, SEQ, SNE = range(1, 18)
S2R, LDG, STG, LDS, STS, ATOMS, BRA, BRZ, BRNZ, BAR, EXIT = range(18, 29)
BARAND, BAROR, BARPOPC = range(29, 32)
BAR_OPS = (BAR, BARAND, BAROR, BARPOPC)
BIMM = 0x80
RZ_INDEX = 0xFF
NREGS = 16

ALU_OPS = (MOV, ADD, SUB, MUL, DIV, REM, AND, OR, XOR, SHL, SHR, MIN, MAX, SLT, SLE, SEQ, SNE)
OP_NAMES = {
    MOV: "MOV", ADD: "ADD", SUB: "SUB", MUL: "MUL", DIV: "DIV", REM: "REM", AND: "AND",
    OR: "OR", XOR: "XOR", SHL: "SHL", SHR: "SHR", MIN: "MIN", MAX: "MAX", SLT: "SLT",
    SLE: "SLE", SEQ: "SEQ", SNE: "SNE", S2R: "S2R", LDG: "LDG", STG: "STG", LDS: "LDS",
    STS: "STS", ATOMS: "ATOMS", BRA: "BRA", BRZ: "BRZ", BRNZ: "BRNZ", BAR: "BAR", EXIT: "EXIT",
    BARAND: "BARAND", BAROR: "BAROR", BARPOPC: "BARPOPC",
}

# special registers read by S2R (the built-in symbols of Sec. 3; 1-D only)
TID, BID, BDIM, GDIM, WARPSIZE = range(5)

INSTR_DTYPE = np.dtype([("op_d_a_b", "<u4"), ("imm", "<i4")])

# limits shared by every consumer of the format
MAX_CODE = 4096          # pcs fit in 12 bits
MAX_BLOCK_DIM = 1024     # tids fit in 10 bits
MAX_SHMEM_WORDS = 12288  # 48 KB of simulated shared memory per block
MAX_PARAMS = 4


class Reg(int):
    """A register operand (distinguishes registers from immediates in the assembler)."""

    def __repr__(self) -> str:  # pragma: no cover - debugging aid
        return "RZ" if self == RZ_INDEX else f"r{int(self)}"


R = [Reg(i) for i in range(NREGS)]
(r0, r1, r2, r3, r4, r5, r6, r7, r8, r9, r10, r11, r12, r13, r14, r15) = R
RZ = Reg(RZ_INDEX)

Operand = Union[Reg, int]


def encode(op: int, d: int = 0, a: int = 0, b: int = 0, imm: int = 0) -> Tuple[int, int]:
    """Pack one instruction into its two 32-bit words."""
    for f in (op, d, a, b):
        if not 0 <= f <= 0xFF:
            raise ValueError(f"field out of range: {f}")
    imm = int(imm)
    if not -(1 << 31) <= imm < (1 << 31):
        raise ValueError(f"immediate out of int32 range: {imm}")
    return (op | d << 8 | a << 16 | b << 24), imm


class Asm:
    """Tiny label-resolving assembler producing an ``INSTR_DTYPE`` array.

    Registers are ``Reg`` instances (``r0``..``r15``, ``RZ``); plain ints are
    immediates.  Branch targets are label names, resolved at ``assemble()``.
    """

    def __init__(self) -> None:
        self.code: List[List] = []  # [op, d, a, b, imm-or-label]
        self.labels: Dict[str, int] = {}

    # -- bookkeeping
    @property
    def pc(self) -> int:
        return len(self.code)

    def label(self, name: str) -> "Asm":
        if name in self.labels:
            raise ValueError(f"duplicate label {name}")
        self.labels[name] = self.pc
        return self

    def _emit(self, op, d=0, a=0, b=0, imm=0) -> "Asm":
        self.code.append([op, int(d), int(a), int(b), imm])
        return self

    # -- ALU
    def alu(self, op: int, d: Reg, a: Reg, b: Operand) -> "Asm":
        if op not in ALU_OPS:
            raise ValueError("not an ALU op")
        if isinstance(b, Reg):
            return self._emit(op, d, a, b, 0)
        return self._emit(op | BIMM, d, a, 0, int(b))

    def mov(self, d: Reg, b: Operand) -> "Asm":
        return self.alu(MOV, d, RZ, b)

    def __getattr__(self, name: str):
        # add/sub/mul/... helpers: asm.add(d, a, b)
        ops = {"add": ADD, "sub": SUB, "mul": MUL, "div": DIV, "rem": REM, "and_": AND,
               "or_": OR, "xor": XOR, "shl": SHL, "shr": SHR, "min_": MIN, "max_": MAX,
               "slt": SLT, "sle": SLE, "seq": SEQ, "sne": SNE}
        if name in ops:
            op = ops[name]
            return lambda d, a, b: self.alu(op, d, a, b)
        raise AttributeError(name)

    # -- special registers, memory
    def s2r(self, d: Reg, sreg: int) -> "Asm":
        return self._emit(S2R, d, 0, 0, sreg)

    def ldg(self, d: Reg, a: Reg, off: int = 0) -> "Asm":
        return self._emit(LDG, d, a, 0, off)

    def stg(self, a: Reg, b: Reg, off: int = 0) -> "Asm":
        return self._emit(STG, 0, a, b, off)

    def lds(self, d: Reg, a: Reg, off: int = 0) -> "Asm":
        return self._emit(LDS, d, a, 0, off)

    def sts(self, a: Reg, b: Reg, off: int = 0) -> "Asm":
        return self._emit(STS, 0, a, b, off)

    def atoms(self, a: Reg, b: Reg, off: int = 0) -> "Asm":
        return self._emit(ATOMS, 0, a, b, off)

    # -- control
    def bra(self, target: str) -> "Asm":
        return self._emit(BRA, 0, 0, 0, target)

    def brz(self, a: Reg, target: str) -> "Asm":
        return self._emit(BRZ, 0, a, 0, target)

    def brnz(self, a: Reg, target: str) -> "Asm":
        return self._emit(BRNZ, 0, a, 0, target)

    def bar(self) -> "Asm":
        return self._emit(BAR)

    def bar_and(self, d: Reg, a: Reg) -> "Asm":
        return self._emit(BARAND, d, a)

    def bar_or(self, d: Reg, a: Reg) -> "Asm":
        return self._emit(BAROR, d, a)

    def bar_count(self, d: Reg, a: Reg) -> "Asm":
        return self._emit(BARPOPC, d, a)

    def exit(self) -> "Asm":
        return self._emit(EXIT)

    def assemble(self) -> np.ndarray:
        out = np.zeros(len(self.code), dtype=INSTR_DTYPE)
        for i, (op, d, a, b, imm) in enumerate(self.code):
            if isinstance(imm, str):
                if imm not in self.labels:
                    raise ValueError(f"undefined label {imm}")
                imm = self.labels[imm]
            w, im = encode(op, d, a, b, imm)
            out[i] = (w, im)
        return out


def decode_fields(code: np.ndarray):
    """Split an INSTR_DTYPE array into (op, d, a, b, imm) integer arrays (for tooling)."""
    w = code["op_d_a_b"].astype(np.uint32)
    return (w & 0xFF, (w >> 8) & 0xFF, (w >> 16) & 0xFF, (w >> 24) & 0xFF,
            code["imm"].astype(np.int32))


def disassemble(code: np.ndarray) -> List[str]:
    """Human-readable listing (debugging and docs)."""
    lines = []
    ops, ds, as_, bs, imms = decode_fields(code)
    rn = lambda x: "RZ" if x == RZ_INDEX else f"r{x}"
    for pc in range(len(code)):
        op, d, a, b, imm = int(ops[pc]), int(ds[pc]), int(as_[pc]), int(bs[pc]), int(imms[pc])
        base = op & 0x3F
        name = OP_NAMES.get(base, f"?{op}")
        if base in ALU_OPS:
            B = f"#{imm}" if op & BIMM else rn(b)
            s = f"{name} {rn(d)}, {B}" if base == MOV else f"{name} {rn(d)}, {rn(a)}, {B}"
        elif base == S2R:
            s = f"S2R {rn(d)}, {['TID', 'BID', 'BDIM', 'GDIM', 'WARPSIZE'][imm] if 0 <= imm < 5 else imm}"
        elif base in (LDG, LDS):
            s = f"{name} {rn(d)}, [{rn(a)}{imm:+d}]"
        elif base in (STG, STS, ATOMS):
            s = f"{name} [{rn(a)}{imm:+d}], {rn(b)}"
        elif base == BRA:
            s = f"BRA ->{imm}"
        elif base in (BRZ, BRNZ):
            s = f"{name} {rn(a)}, ->{imm}"
        elif base in (BARAND, BAROR, BARPOPC):
            s = f"{name} {rn(d)}, {rn(a)}"
        else:
            s = name
        lines.append(f"{pc:3d} {s}")
    return lines


@dataclass
class Launch:
    """One ``kernel<<<grid, block_dim, shmem, stream>>>(params...)`` call (Sec. 2, kernel
    configuration).  Launches of one stream run in order; launches of different streams may
    run in parallel; ``wait`` >= 0 makes the launch also wait for an event recorded right after
    launch ``wait`` of the same program (an earlier one), as ``cudaStreamWaitEvent`` would
    (Sec. 3, streams and events).  The defaults put every launch in one stream."""

    kernel: int
    grid: int
    block_dim: int
    shmem_words: int
    params: Tuple[int, ...] = ()
    stream: int = 0
    wait: int = -1
    # run only blocks [block_begin, block_begin + block_count) of the grid (a process's share
    # of a launch split across processes); 0 = every block.  Block indices keep the grid's
    # numbering.
    block_begin: int = 0
    block_count: int = 0


@dataclass
class Program:
    """A simulated CUDA program: code, kernels, launch list and initial global arena.

    Launches run in stream order over the one global arena, with the implicit grid-wide
    synchronisation between kernel calls of a stream (Sec. 2).
    """

    code: np.ndarray
    kernel_entry: List[int]
    launches: List[Launch]
    global_init: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    def __post_init__(self) -> None:
        self.code = np.ascontiguousarray(self.code, dtype=INSTR_DTYPE)
        self.global_init = np.ascontiguousarray(self.global_init, dtype=np.int32)

    @property
    def ncode(self) -> int:
        return int(len(self.code))

    def total_threads(self) -> int:
        return sum(l.grid * l.block_dim for l in self.launches)
