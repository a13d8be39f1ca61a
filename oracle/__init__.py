"""CPU oracle for the SIMT race/barrier checker (ctypes wrapper around simt_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``.  The library package never imports this module.

``run(programs, ...)`` executes every program with the canonical round-lockstep
schedule and returns the final global arenas, per-program status bits and the
canonically sorted report records ``(kind, prog, launch, block, epoch, a, b, c)``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "simt_oracle.c")
_HDR = os.path.join(_HERE, "simt_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

# report kinds / status bits (same numbers as simt_oracle.h)
RACE, DIVERGENCE, DEADLOCK, STEP_LIMIT, ERR_OOB_SHARED, ERR_OOB_GLOBAL, ERR_DIV0, ERR_UNINIT_SHARED = range(1, 9)
GLOBAL_RACE, GLOBAL_BLOCKS, GLOBAL_LAUNCHES = 9, 10, 11      # with check_global
CLS_WW, CLS_WR, CLS_WA, CLS_AR = 1, 2, 4, 8
ST_DEADLOCK, ST_STEP_LIMIT = 1, 2

REPORT_DTYPE = np.dtype([(n, "<u4") for n in ("kind", "prog", "launch", "block", "epoch", "a", "b", "c")])


class _Instr(C.Structure):
    _fields_ = [("op_d_a_b", C.c_uint32), ("imm", C.c_int32)]


class _Launch(C.Structure):
    _fields_ = [("kernel", C.c_uint32), ("grid", C.c_uint32), ("block_dim", C.c_uint32),
                ("shmem_words", C.c_uint32), ("nparams", C.c_uint32), ("params", C.c_int32 * 4),
                ("stream", C.c_uint32), ("wait", C.c_uint32), ("block_begin", C.c_uint32),
                ("block_count", C.c_uint32)]


class _Program(C.Structure):
    _fields_ = [("code", C.c_void_p), ("ncode", C.c_uint32),
                ("kernel_entry", C.c_void_p), ("nkernels", C.c_uint32),
                ("launches", C.c_void_p), ("nlaunches", C.c_uint32),
                ("arena", C.c_void_p), ("arena_words", C.c_uint64)]


class _Opts(C.Structure):
    _fields_ = [("round_budget", C.c_uint32), ("check_races", C.c_uint32), ("schedule", C.c_uint32),
                ("nthreads", C.c_uint32), ("check_interblock", C.c_uint32), ("max_blocks", C.c_uint32),
                ("check_uninit", C.c_uint32), ("check_streams", C.c_uint32), ("check_global", C.c_uint32)]


class _Result(C.Structure):
    _fields_ = [("reports", C.c_void_p), ("nreports", C.c_uint64), ("status", C.POINTER(C.c_uint32)),
                ("thread_instrs", C.c_uint64), ("shared_accesses", C.c_uint64), ("rounds", C.c_uint64),
                ("interblock_conflicts", C.c_uint64), ("stream_conflicts", C.c_uint64)]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (plain gcc, no GPU code)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC,
                               "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.orc_run.argtypes = [C.c_void_p, C.c_uint32, C.POINTER(_Opts), C.POINTER(_Result)]
            lib.orc_run.restype = C.c_int
            lib.orc_free.argtypes = [C.POINTER(_Result)]
            lib.orc_last_error.restype = C.c_char_p
            _lib = lib
    return _lib


@dataclass
class OracleResult:
    arenas: List[np.ndarray]
    status: np.ndarray
    reports: np.ndarray          # REPORT_DTYPE, canonical order
    thread_instrs: int
    shared_accesses: int
    rounds: int
    interblock_conflicts: int    # check_interblock: global words two blocks of a launch touch, one writing
    stream_conflicts: int = 0    # check_streams: global words two unordered launches share, one writing

    def report_tuples(self):
        return [tuple(int(x) for x in r) for r in self.reports]


def run(programs: Sequence, round_budget: int = 0, check_races: bool = True, schedule: str = "lockstep",
        nthreads: int = 1, check_interblock: bool = False, max_blocks: int = 0,
        check_uninit: bool = False, check_streams: bool = False, check_global: bool = False) -> OracleResult:
    """Run ``programs`` (``workloads.ir.Program``) through the oracle."""
    lib = _load()
    keep = []
    arenas = []
    progs = (_Program * max(1, len(programs)))()
    for i, p in enumerate(programs):
        code = np.ascontiguousarray(p.code)
        entries = np.ascontiguousarray(np.asarray(p.kernel_entry, dtype=np.uint32))
        ls = (_Launch * max(1, len(p.launches)))()
        for j, l in enumerate(p.launches):
            ls[j].kernel, ls[j].grid, ls[j].block_dim = l.kernel, l.grid, l.block_dim
            ls[j].shmem_words, ls[j].nparams = l.shmem_words, len(l.params)
            for k, v in enumerate(l.params):
                ls[j].params[k] = int(v)
            ls[j].stream, ls[j].wait = getattr(l, "stream", 0), getattr(l, "wait", -1) + 1
            ls[j].block_begin, ls[j].block_count = getattr(l, "block_begin", 0), getattr(l, "block_count", 0)
        arena = np.array(p.global_init, dtype=np.int32, copy=True)
        arenas.append(arena)
        keep += [code, entries, ls]
        progs[i].code, progs[i].ncode = code.ctypes.data, len(code)
        progs[i].kernel_entry, progs[i].nkernels = entries.ctypes.data, len(entries)
        progs[i].launches, progs[i].nlaunches = C.addressof(ls), len(p.launches)
        progs[i].arena, progs[i].arena_words = (arena.ctypes.data if arena.size else None), arena.size
    opts = _Opts(round_budget, int(check_races), {"lockstep": 0, "sequential": 1}[schedule], nthreads,
                 int(check_interblock), max_blocks, int(check_uninit), int(check_streams), int(check_global))
    res = _Result()
    rc = lib.orc_run(C.addressof(progs), len(programs), C.byref(opts), C.byref(res))
    if rc != 0:
        raise ValueError("oracle rejected the programs: " + lib.orc_last_error().decode())
    try:
        n = int(res.nreports)
        reps = np.zeros(n, dtype=REPORT_DTYPE)
        if n:
            C.memmove(reps.ctypes.data, res.reports, n * REPORT_DTYPE.itemsize)
        status = np.array([res.status[i] for i in range(len(programs))], dtype=np.uint32)
        out = OracleResult(arenas, status, reps, int(res.thread_instrs), int(res.shared_accesses),
                           int(res.rounds), int(res.interblock_conflicts), int(res.stream_conflicts))
    finally:
        lib.orc_free(C.byref(res))
    return out
