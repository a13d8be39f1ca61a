"""Continuous-batching serving loop over the checker.

Jobs (one simulated program each) arrive over time.  The server keeps up to
``max_inflight`` micro-batches on the GPU, each loaded and run on its own CUDA stream
(`load_programs` + `run_and_check`), so work of batches admitted at different times
overlaps on the device.  A waiting job is admitted as soon as a stream slot is free and
its predicted access-log bytes fit the remaining log budget; a finished batch (polled
with a CUDA event) is fetched, split back into per-job results, and freed, which
returns its budget.  Latency of a job = arrival -> its reports and arena on the host.

The log-byte prediction is the same static bound the library reserves (shared accesses on
the longest control path x blockDim + barrier/error record room, per block), computed
here from the IR so that admission needs no device call.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import binding
from .workloads import ir
from .workloads.ir import Program
from .workloads import families, rng


# ------------------------------------------------------------------ admission estimate
def _kernel_bound(code: np.ndarray, entry: int):
    """(cyclic, max shared accesses on a path, max barriers on a path, error-capable pcs)."""
    ops, _, _, _, imms = ir.decode_fields(code)
    n = len(code)
    succ = []
    for pc in range(n):
        b, t = int(ops[pc]) & 0x7F, int(imms[pc])
        if b == ir.EXIT:
            succ.append(())
        elif b == ir.BRA:
            succ.append((t,))
        elif b in (ir.BRZ, ir.BRNZ):
            succ.append((pc + 1, t))
        else:
            succ.append((pc + 1,))
    succ.append(())                                     # pc == n: implicit exit
    colour = [0] * (n + 1)
    acc = [0] * (n + 1)
    bar = [0] * (n + 1)
    errs = 0
    stack = [(entry, 0)]
    colour[entry] = 1
    while stack:
        pc, i = stack[-1]
        if i < len(succ[pc]):
            stack[-1] = (pc, i + 1)
            nx = succ[pc][i]
            if colour[nx] == 1:
                return True, 0, 0, 0
            if colour[nx] == 0:
                colour[nx] = 1
                stack.append((nx, 0))
            continue
        a = max((acc[s] for s in succ[pc]), default=0)
        br = max((bar[s] for s in succ[pc]), default=0)
        if pc < n:
            b = int(ops[pc]) & 0x7F
            a += b in (ir.LDS, ir.STS, ir.ATOMS)
            br += b in ir.BAR_OPS
            errs += b in (ir.LDS, ir.STS, ir.ATOMS, ir.LDG, ir.STG, ir.DIV, ir.REM)
        acc[pc], bar[pc], colour[pc] = a, br, 2
        stack.pop()
    return False, acc[entry], bar[entry], errs


def predicted_log_bytes(p: Program, loop_records: int = 65536) -> int:
    """Access-log bytes the library reserves for program ``p`` (all launches resident)."""
    total = 0
    bounds = {}
    for l in p.launches:
        if l.kernel not in bounds:
            bounds[l.kernel] = _kernel_bound(p.code, p.kernel_entry[l.kernel])
        cyc, acc, bars, errs = bounds[l.kernel]
        if cyc:
            recs, misc = loop_records, max(256, 4 * (1 + errs))
        else:
            recs, misc = acc * l.block_dim, (bars + 1) * (1 + errs) + 1
        cap = (recs + 2 * misc + 1) & ~1
        total += (l.block_count or l.grid) * cap * 8
    return total


# ------------------------------------------------------------------ jobs and results
@dataclass
class Job:
    jid: int
    program: Program
    arrival: float          # seconds from the start of the trace
    log_bytes: int = 0


@dataclass
class JobResult:
    reports: np.ndarray     # REPORT_DTYPE; `prog` is the job's position in its micro-batch
    arena: np.ndarray
    status: int
    arrival: float
    done: float

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class ServeStats:
    jobs: int
    seconds: float
    jobs_per_s: float
    p50_ms: float
    p99_ms: float
    shared_accesses: int
    accesses_per_s: float
    batches: int
    max_inflight_seen: int
    mean_batch_jobs: float
    peak_log_bytes: int
    host_load_s: float = 0.0       # host time in load_programs + run_and_check (enqueue)
    host_fetch_s: float = 0.0      # host time fetching and splitting finished batches
    mean_batch_gpu_ms: float = 0.0  # enqueue-to-completion time of a batch on its stream


def poisson_trace(rate: float, seconds: float, seed: int = 5) -> List[float]:
    """Arrival times of a Poisson process (exponential gaps from SplitMix64)."""
    R = rng.SplitMix64(seed)
    t, out = 0.0, []
    while True:
        t += -np.log(1.0 - R.uniform()) / rate
        if t >= seconds:
            return out
        out.append(t)


def job_pool(n: int, seed: int = 5, max_grid: int = 4096) -> List[Program]:
    """Distinct programs drawn from the batched-workload generator (sub-streams of seed)."""
    return families.batch(n_programs=n, seed=seed, max_grid=max_grid)


# ------------------------------------------------------------------ the server
@dataclass
class _Flight:
    jobs: List[Job]
    batch: "binding.Batch"
    stream: object
    event: object
    log_bytes: int
    start: object


class Server:
    def __init__(self, log_budget_bytes: int = 120 << 30, max_inflight: int = 4, max_batch_jobs: int = 512,
                 mode: str = "batched", **ctx_opts):
        import torch
        self.torch = torch
        self.budget = log_budget_bytes
        self.max_inflight = max_inflight
        self.max_batch_jobs = max_batch_jobs
        # one context: the server loop is the only host thread using it.  Device memory comes
        # from the context's stream-ordered pool by default: a micro-batch then costs no
        # Python allocator callbacks, which at two jobs per batch were a third of its host
        # time.  (ctx_opts: further binding.Context options, e.g. kernel shapes.)
        ctx_opts.setdefault("torch_allocator", False)
        self.ctx = binding.Context(mode=mode, log_budget_mb=max(1, log_budget_bytes >> 20), **ctx_opts)
        self.streams = [torch.cuda.Stream() for _ in range(max_inflight)]

    def close(self):
        self.ctx.close()

    def _finish(self, f: _Flight, t0: float, emit: Callable[[int, JobResult], None]):
        tf = time.perf_counter()
        self._gpu_ms.append(f.start.elapsed_time(f.event))
        # one page-locked copy each for the reports, the arenas and the status words
        reps = f.batch.fetch_reports(pinned=True)
        arenas = f.batch.fetch_all_memory(pinned=True)
        status = f.batch.all_status()
        self._accesses += f.batch.stats().shared_accesses
        now = time.perf_counter() - t0
        # reports are in canonical order, program first: one slice per job (its `prog`
        # field stays the job's position in the micro-batch)
        cut = np.searchsorted(reps["prog"], np.arange(len(f.jobs) + 1, dtype=np.uint32))
        for k, job in enumerate(f.jobs):
            emit(job.jid, JobResult(reps[cut[k]:cut[k + 1]], arenas[k], int(status[k]), job.arrival, now))
        f.batch.free()
        self._fetch_s += time.perf_counter() - tf

    def serve(self, jobs: Sequence[Job], on_result: Optional[Callable[[int, JobResult], None]] = None
              ) -> Tuple[Dict[int, JobResult], ServeStats]:
        """Serve the trace.  Each result goes to ``on_result(jid, result)`` when given (and
        is not kept; results hold page-locked host memory until they are dropped),
        otherwise into the returned dict."""
        jobs = sorted(jobs, key=lambda j: j.arrival)
        for j in jobs:
            if not j.log_bytes:
                j.log_bytes = predicted_log_bytes(j.program)
            if j.log_bytes > self.budget:
                raise ValueError(f"job {j.jid} needs {j.log_bytes} log bytes, over the whole budget")
        results: Dict[int, JobResult] = {}
        latencies: List[float] = []

        def emit(jid: int, r: JobResult):
            latencies.append(r.latency)
            if on_result is None:
                results[jid] = r
            else:
                on_result(jid, r)

        self._accesses = 0
        self._fetch_s = load_s = 0.0
        self._gpu_ms = []
        waiting: collections.deque = collections.deque()
        inflight: List[_Flight] = []
        free_streams = list(range(self.max_inflight))
        used = peak = 0
        nb, batch_sizes, max_fl = 0, [], 0
        nxt = 0
        t0 = time.perf_counter()
        while nxt < len(jobs) or waiting or inflight:
            now = time.perf_counter() - t0
            while nxt < len(jobs) and jobs[nxt].arrival <= now:
                waiting.append(jobs[nxt])
                nxt += 1
            # completed batches return their streams and log budget
            for f in [f for f in inflight if f.event.query()]:
                inflight.remove(f)
                self._finish(f, t0, emit)
                used -= f.log_bytes
                free_streams.append(self.streams.index(f.stream))
            # admit waiting jobs into a new micro-batch while a stream and budget are free
            while waiting and free_streams:
                take, bytes_ = [], 0
                while waiting and len(take) < self.max_batch_jobs and used + bytes_ + waiting[0].log_bytes <= self.budget:
                    j = waiting.popleft()
                    take.append(j)
                    bytes_ += j.log_bytes
                if not take:
                    break
                si = free_streams.pop()
                stream = self.streams[si]
                tl = time.perf_counter()
                start = self.torch.cuda.Event(enable_timing=True)
                start.record(stream)
                batch = self.ctx.load_programs([j.program for j in take], stream=stream)
                batch.run_and_check(stream=stream)
                ev = self.torch.cuda.Event(enable_timing=True)
                ev.record(stream)
                load_s += time.perf_counter() - tl
                inflight.append(_Flight(take, batch, stream, ev, bytes_, start))
                used += bytes_
                peak = max(peak, used)
                nb += 1
                batch_sizes.append(len(take))
                max_fl = max(max_fl, len(inflight))
            if not inflight and not waiting and nxt < len(jobs):
                time.sleep(max(0.0, min(0.01, jobs[nxt].arrival - (time.perf_counter() - t0))))
            elif inflight:
                time.sleep(0.0002)
        elapsed = time.perf_counter() - t0
        lat = np.array(latencies) * 1e3
        stats = ServeStats(len(lat), elapsed, len(lat) / elapsed if elapsed else 0.0,
                           float(np.percentile(lat, 50)) if len(lat) else 0.0,
                           float(np.percentile(lat, 99)) if len(lat) else 0.0, self._accesses,
                           self._accesses / elapsed if elapsed else 0.0, nb, max_fl,
                           float(np.mean(batch_sizes)) if batch_sizes else 0.0, peak, load_s, self._fetch_s,
                           float(np.mean(self._gpu_ms)) if self._gpu_ms else 0.0)
        return results, stats
