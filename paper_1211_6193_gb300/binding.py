"""Thin ctypes binding of libsimtcheck (include/simtcheck.h): same entry-point names,
argument marshalling only.  Every step of the check runs in the library's CUDA kernels;
there is no CPU fallback - loading fails loudly when the library is missing.

PyTorch provides device memory (a caching-allocator-backed ``sr_allocator``) and
streams (``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence

import numpy as np

from .workloads.ir import Program

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsimtcheck.so")

# return codes / constants (include/simtcheck.h)
SR_OK, SR_E_INVAL, SR_E_NOMEM, SR_E_CUDA, SR_E_TIMEOUT, SR_E_RANGE, SR_E_BOUNDS = 0, -1, -2, -3, -4, -5, -6
SR_ALL_PROGRAMS = 0xFFFFFFFF
MODE_PLAIN, MODE_BATCHED = 0, 1
RACE, DIVERGENCE, DEADLOCK, STEP_LIMIT, ERR_OOB_SHARED, ERR_OOB_GLOBAL, ERR_DIV0, ERR_UNINIT_SHARED = range(1, 9)
GLOBAL_RACE, GLOBAL_BLOCKS, GLOBAL_LAUNCHES = 9, 10, 11
ST_DEADLOCK, ST_STEP_LIMIT, ST_LOG_OVERFLOW, ST_INTERNAL, ST_BOUNDS = 1, 2, 4, 8, 16
REPORT_DTYPE = np.dtype([(n, "<u4") for n in ("kind", "prog", "launch", "block", "epoch", "a", "b", "c")])


class SimtCheckError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"simtcheck error {code}: {msg}")
        self.code = code


class sr_instr(C.Structure):
    _fields_ = [("op_d_a_b", C.c_uint32), ("imm", C.c_int32)]


class sr_launch(C.Structure):
    _fields_ = [("kernel", C.c_uint32), ("grid", C.c_uint32), ("block_dim", C.c_uint32),
                ("shmem_words", C.c_uint32), ("nparams", C.c_uint32), ("params", C.c_int32 * 4),
                ("stream", C.c_uint32), ("wait", C.c_uint32), ("block_begin", C.c_uint32),
                ("block_count", C.c_uint32)]


class sr_program(C.Structure):
    _fields_ = [("code", C.c_void_p), ("ncode", C.c_uint32), ("kernel_entry", C.c_void_p),
                ("nkernels", C.c_uint32), ("launches", C.c_void_p), ("nlaunches", C.c_uint32),
                ("global_init", C.c_void_p), ("global_words", C.c_uint64)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)


class sr_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("user", C.c_void_p)]


class sr_opts(C.Structure):
    _fields_ = [("check_races", C.c_uint32), ("round_budget", C.c_uint32), ("mode", C.c_uint32),
                ("ctas_per_sm", C.c_uint32), ("loop_log_records", C.c_uint32),
                ("interp_variant", C.c_uint32), ("use_graph", C.c_uint32), ("profile", C.c_uint32),
                ("spin_limit", C.c_uint32), ("log_budget_mb", C.c_uint32), ("report_cap", C.c_uint32),
                ("allocator", C.POINTER(sr_allocator)), ("check_variant", C.c_uint32),
                ("check_uninit", C.c_uint32), ("fused_check", C.c_uint32), ("check_global", C.c_uint32)]


class sr_stats(C.Structure):
    _fields_ = [("thread_instrs", C.c_uint64), ("shared_accesses", C.c_uint64), ("global_accesses", C.c_uint64),
                ("reports", C.c_uint64), ("log_bytes", C.c_uint64), ("blocks", C.c_uint64),
                ("ms_reset", C.c_float), ("ms_interp", C.c_float), ("ms_check", C.c_float),
                ("ms_compact", C.c_float), ("waves", C.c_uint32), ("kernels", C.c_uint32),
                ("ms_global", C.c_float), ("global_records", C.c_uint64), ("one_per_cta_blocks", C.c_uint64)]


EXPORTS = ["sr_create", "sr_destroy", "sr_validate_program", "load_programs", "run_and_check", "fetch_reports",
           "fetch_memory", "sr_batch_status", "sr_batch_stats", "sr_free_batch", "sr_last_error",
           "sr_check_program_noalloc"]
NOALLOC_SCRATCH_BYTES = 32 << 20

_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libsimtcheck.so (build it with ``paper_1211_6193_gb300.build.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"libsimtcheck.so not built ({path}); run paper_1211_6193_gb300.build.build()")
        lib = C.CDLL(path)
        vp, u32, u64 = C.c_void_p, C.c_uint32, C.c_uint64
        lib.sr_create.argtypes = [C.POINTER(vp), C.POINTER(sr_opts)]
        lib.sr_destroy.argtypes = [vp]
        lib.sr_destroy.restype = None
        lib.sr_validate_program.argtypes = [C.POINTER(sr_program), C.c_char_p, C.c_size_t]
        lib.load_programs.argtypes = [vp, C.POINTER(sr_program), u32, vp, C.POINTER(vp)]
        lib.run_and_check.argtypes = [vp, vp, vp]
        lib.fetch_reports.argtypes = [vp, vp, vp, u64, C.POINTER(u64)]
        lib.fetch_memory.argtypes = [vp, vp, u32, vp, u64, C.POINTER(u64)]
        lib.sr_batch_status.argtypes = [vp, vp, u32, C.POINTER(u32)]
        lib.sr_batch_stats.argtypes = [vp, vp, C.POINTER(sr_stats)]
        lib.sr_free_batch.argtypes = [vp, vp]
        lib.sr_free_batch.restype = None
        lib.sr_last_error.argtypes = [vp]
        lib.sr_last_error.restype = C.c_char_p
        lib.sr_check_program_noalloc.argtypes = [C.POINTER(sr_program), vp, vp, u64, C.POINTER(u64),
                                                 C.POINTER(u32), vp]
        for name in EXPORTS:
            if name not in ("sr_destroy", "sr_free_batch", "sr_last_error"):
                getattr(lib, name).restype = C.c_int
        _lib = lib
    return _lib


# ------------------------------------------------------------------ marshalling
class _Marshalled:
    """ctypes program descriptors plus the numpy buffers they point into."""

    def __init__(self, programs: Sequence[Program]):
        self.keep: list = []
        self.array = (sr_program * max(1, len(programs)))()
        for i, p in enumerate(programs):
            code = np.ascontiguousarray(p.code)
            entries = np.ascontiguousarray(np.asarray(p.kernel_entry, dtype=np.uint32))
            ls = (sr_launch * max(1, len(p.launches)))()
            for j, l in enumerate(p.launches):
                ls[j].kernel, ls[j].grid, ls[j].block_dim = l.kernel, l.grid, l.block_dim
                ls[j].shmem_words, ls[j].nparams = l.shmem_words, len(l.params)
                for k, v in enumerate(l.params):
                    ls[j].params[k] = int(v)
                ls[j].stream, ls[j].wait = l.stream, l.wait + 1
                ls[j].block_begin, ls[j].block_count = l.block_begin, l.block_count
            arena = np.ascontiguousarray(p.global_init, dtype=np.int32)
            self.keep += [code, entries, ls, arena]
            a = self.array[i]
            a.code, a.ncode = code.ctypes.data, len(code)
            a.kernel_entry, a.nkernels = entries.ctypes.data, len(entries)
            a.launches, a.nlaunches = C.addressof(ls), len(p.launches)
            a.global_init, a.global_words = (arena.ctypes.data if arena.size else None), arena.size


def host_empty(n: int, dtype, pinned: bool = False) -> np.ndarray:
    """Uninitialised host array; page-locked (from PyTorch's caching host allocator) when
    ``pinned``, so that device-to-host copies into it run at link speed.  The returned
    array keeps its page-locked block alive until the array and its views are gone."""
    dtype = np.dtype(dtype)
    if not pinned:
        return np.empty(n, dtype=dtype)
    import torch
    t = torch.empty(max(1, n * dtype.itemsize), dtype=torch.uint8, pin_memory=True)
    return t.numpy()[: n * dtype.itemsize].view(dtype)


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class TorchAllocator:
    """sr_allocator backed by PyTorch's caching allocator (uint8 tensors kept alive by pointer)."""

    def __init__(self):
        import torch
        self._torch = torch
        self.live: Dict[int, object] = {}
        self._alloc = ALLOC_FN(self._do_alloc)
        self._release = RELEASE_FN(self._do_release)
        self.struct = sr_allocator(self._alloc, self._release, None)

    def _do_alloc(self, user, nbytes, stream):
        torch = self._torch
        try:
            s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(s):
                t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        except Exception:  # allocation failure is reported to the library as NULL
            return None
        ptr = t.data_ptr()
        self.live[ptr] = t
        return ptr

    def _do_release(self, user, ptr, nbytes, stream):
        self.live.pop(int(ptr), None)


@dataclass
class Stats:
    thread_instrs: int
    shared_accesses: int
    global_accesses: int
    reports: int
    log_bytes: int
    blocks: int
    ms_reset: float
    ms_interp: float
    ms_check: float
    ms_compact: float
    waves: int
    kernels: int
    ms_global: float
    global_records: int
    one_per_cta_blocks: int


class Context:
    """An ``sr_ctx``: options + device; creates batches with the same-named entry points."""

    def __init__(self, check_races: bool = True, round_budget: int = 0, mode: str = "plain", ctas_per_sm: int = 0,
                 loop_log_records: int = 0, interp_variant: int = 0, use_graph: bool = False,
                 profile: bool = False, spin_limit: int = 0, log_budget_mb: int = 0, report_cap: int = 0,
                 torch_allocator: bool = True, check_variant: int = 0, check_uninit: bool = False,
                 fused_check: bool = False, check_global: bool = False):
        self.lib = load_library()
        self.allocator = TorchAllocator() if torch_allocator else None
        o = sr_opts()
        o.check_races, o.round_budget = int(check_races), round_budget
        o.mode = {"plain": MODE_PLAIN, "batched": MODE_BATCHED}[mode]
        o.ctas_per_sm, o.loop_log_records, o.interp_variant = ctas_per_sm, loop_log_records, interp_variant
        o.use_graph, o.profile, o.spin_limit = int(use_graph), int(profile), spin_limit
        o.log_budget_mb, o.report_cap = log_budget_mb, report_cap
        o.check_variant = check_variant
        o.check_uninit = int(check_uninit)
        o.fused_check = int(fused_check)
        o.check_global = int(check_global)
        if self.allocator is not None:
            o.allocator = C.pointer(self.allocator.struct)
        self.opts = o
        h = C.c_void_p()
        self._check(self.lib.sr_create(C.byref(h), C.byref(o)), ctx=None)
        self.handle = h

    def _check(self, rc: int, ctx="self"):
        if rc != SR_OK:
            h = None if ctx is None else self.handle
            raise SimtCheckError(rc, (self.lib.sr_last_error(h) or b"").decode())

    def close(self):
        if getattr(self, "handle", None):
            self.lib.sr_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --- entry points
    def load_programs(self, programs: Sequence[Program], stream=None) -> "Batch":
        m = _Marshalled(programs)
        b = C.c_void_p()
        self._check(self.lib.load_programs(self.handle, m.array, len(programs), _stream_handle(stream), C.byref(b)))
        return Batch(self, b, programs)

    def validate(self, program: Program) -> Optional[str]:
        m = _Marshalled([program])
        buf = C.create_string_buffer(256)
        rc = self.lib.sr_validate_program(m.array, buf, 256)
        return None if rc == SR_OK else buf.value.decode()


class Batch:
    """A loaded ``sr_batch``."""

    def __init__(self, ctx: Context, handle, programs: Sequence[Program]):
        self.ctx, self.handle = ctx, handle
        self.nprogs = len(programs)
        self.arena_words = [int(np.asarray(p.global_init).size) for p in programs]

    def run_and_check(self, stream=None) -> None:
        self.ctx._check(self.ctx.lib.run_and_check(self.ctx.handle, self.handle, _stream_handle(stream)))

    def fetch_reports(self, pinned: bool = False) -> np.ndarray:
        lib = self.ctx.lib
        n = C.c_uint64()
        self.ctx._check(lib.fetch_reports(self.ctx.handle, self.handle, None, 0, C.byref(n)))
        out = host_empty(int(n.value), REPORT_DTYPE, pinned)
        if n.value:
            self.ctx._check(lib.fetch_reports(self.ctx.handle, self.handle, out.ctypes.data, n.value, C.byref(n)))
        return out

    def fetch_memory(self, prog: int, out: Optional[np.ndarray] = None) -> np.ndarray:
        lib = self.ctx.lib
        n = C.c_uint64()
        self.ctx._check(lib.fetch_memory(self.ctx.handle, self.handle, prog, None, 0, C.byref(n)))
        if out is None:
            out = np.zeros(int(n.value), dtype=np.int32)
        self.ctx._check(lib.fetch_memory(self.ctx.handle, self.handle, prog, out.ctypes.data, out.size, C.byref(n)))
        return out

    def fetch_all_memory(self, pinned: bool = False) -> List[np.ndarray]:
        """Every program's final arena with one copy (views into one host buffer)."""
        lib = self.ctx.lib
        n = C.c_uint64()
        self.ctx._check(lib.fetch_memory(self.ctx.handle, self.handle, SR_ALL_PROGRAMS, None, 0, C.byref(n)))
        buf = host_empty(int(n.value), np.int32, pinned)
        self.ctx._check(lib.fetch_memory(self.ctx.handle, self.handle, SR_ALL_PROGRAMS,
                                         buf.ctypes.data if buf.size else None, buf.size, C.byref(n)))
        out, off = [], 0
        for w in self.arena_words:
            out.append(buf[off: off + w])
            off += (w + 3) & ~3
        return out

    def status(self, prog: int) -> int:
        st = C.c_uint32()
        self.ctx._check(self.ctx.lib.sr_batch_status(self.ctx.handle, self.handle, prog, C.byref(st)))
        return int(st.value)

    def all_status(self) -> np.ndarray:
        st = np.zeros(max(1, self.nprogs), dtype=np.uint32)
        self.ctx._check(self.ctx.lib.sr_batch_status(self.ctx.handle, self.handle, SR_ALL_PROGRAMS,
                                                     st.ctypes.data_as(C.POINTER(C.c_uint32))))
        return st[: self.nprogs]

    def stats(self) -> Stats:
        s = sr_stats()
        self.ctx._check(self.ctx.lib.sr_batch_stats(self.ctx.handle, self.handle, C.byref(s)))
        return Stats(*(getattr(s, f) for f, _ in sr_stats._fields_))

    def free(self):
        if self.handle:
            self.ctx.lib.sr_free_batch(self.ctx.handle, self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()


@dataclass
class CheckResult:
    arenas: List[np.ndarray]
    status: np.ndarray
    reports: np.ndarray
    stats: Stats

    def report_tuples(self):
        return [tuple(int(x) for x in r) for r in self.reports]


def check(programs: Sequence[Program], **opts) -> CheckResult:
    """Load, run and fetch everything for ``programs`` in one call."""
    with Context(**opts) as ctx, ctx.load_programs(programs) as b:
        b.run_and_check()
        reps = b.fetch_reports()
        arenas = [b.fetch_memory(i) for i in range(len(programs))]
        status = np.array([b.status(i) for i in range(len(programs))], dtype=np.uint32)
        return CheckResult(arenas, status, reps, b.stats())
