"""Continuous-batching serving loop over the checker.

Jobs (one simulated program each) arrive over time.  The server runs up to
``max_inflight`` workers, each a host thread with its own context and CUDA stream; a
worker takes one micro-batch of waiting jobs, loads it (`load_programs`), runs it
(`run_and_check`), fetches the reports and arenas into page-locked memory, splits them
back into per-job results and frees the batch, which returns its log budget.  The host
work of one batch (IR marshalling, validation, fetching) thus overlaps the kernels of the
others.  A waiting job is admitted as soon as a worker is free and its predicted
access-log bytes fit the remaining budget.  Latency of a job = arrival -> its reports and
arena on the host.

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
    host_load_s: float = 0.0       # worker time in load_programs + run_and_check, summed over workers
    host_fetch_s: float = 0.0      # worker time fetching, splitting and freeing, summed over workers
    mean_batch_gpu_ms: float = 0.0  # load-to-completion time of a batch on its stream (CUDA events)


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
class Server:
    """Continuous batching over ``max_inflight`` workers.  The admission loop (the caller's
    thread) moves arrived jobs to a waiting queue and, whenever a worker is free and the
    jobs' predicted log bytes fit the budget, hands the waiting jobs (up to max_batch_jobs)
    to that worker as one micro-batch; jobs that arrive meanwhile wait for the next free
    worker, so batches grow when the GPU is busy.  A worker is a host thread with its own
    context and CUDA stream (the library's contexts are single-threaded): it loads, runs,
    fetches and splits its micro-batch, so the host work of several batches overlaps and
    their kernels share the GPU."""

    def __init__(self, log_budget_bytes: int = 120 << 30, max_inflight: int = 4, max_batch_jobs: int = 512,
                 mode: str = "batched", **ctx_opts):
        import torch
        self.torch = torch
        self.budget = log_budget_bytes
        self.max_inflight = max_inflight
        self.max_batch_jobs = max_batch_jobs
        # Device memory comes from each context's stream-ordered pool by default: a micro-batch
        # then costs no Python allocator callbacks.  (ctx_opts: further binding.Context options,
        # e.g. kernel shapes.)
        ctx_opts.setdefault("torch_allocator", False)
        self.device = torch.cuda.current_device()
        self.ctxs = [binding.Context(mode=mode, log_budget_mb=max(1, log_budget_bytes >> 20), **ctx_opts)
                     for _ in range(max_inflight)]
        self.streams = [torch.cuda.Stream() for _ in range(max_inflight)]

    def close(self):
        for c in self.ctxs:
            c.close()

    def serve(self, jobs: Sequence[Job], on_result: Optional[Callable[[int, JobResult], None]] = None
              ) -> Tuple[Dict[int, JobResult], ServeStats]:
        """Serve the trace.  Each result goes to ``on_result(jid, result)`` when given (and
        is not kept; results hold page-locked host memory until they are dropped),
        otherwise into the returned dict.  Latency: arrival to the job's reports and arena
        on the host."""
        import queue
        import threading

        torch = self.torch
        jobs = sorted(jobs, key=lambda j: j.arrival)
        for j in jobs:
            if not j.log_bytes:
                j.log_bytes = predicted_log_bytes(j.program)
            if j.log_bytes > self.budget:
                raise ValueError(f"job {j.jid} needs {j.log_bytes} log bytes, over the whole budget")
        results: Dict[int, JobResult] = {}
        latencies: List[float] = []
        lock = threading.Condition()
        state = {"used": 0, "peak": 0, "free": list(range(self.max_inflight)), "accesses": 0, "load_s": 0.0,
                 "fetch_s": 0.0, "gpu_ms": [], "busy": 0, "max_busy": 0, "error": None}
        inbox = [queue.Queue() for _ in range(self.max_inflight)]
        t0 = time.perf_counter()

        def worker(wi: int):
            torch.cuda.set_device(self.device)
            ctx, stream = self.ctxs[wi], self.streams[wi]
            while True:
                take = inbox[wi].get()
                if take is None:
                    return
                try:
                    tl = time.perf_counter()
                    start = torch.cuda.Event(enable_timing=True)
                    start.record(stream)
                    batch = ctx.load_programs([j.program for j in take], stream=stream)
                    batch.run_and_check(stream=stream)
                    ev = torch.cuda.Event(enable_timing=True)
                    ev.record(stream)
                    tf = time.perf_counter()
                    # one page-locked copy each for the reports, the arenas and the status words
                    reps = batch.fetch_reports(pinned=True)
                    arenas = batch.fetch_all_memory(pinned=True)
                    status = batch.all_status()
                    acc = batch.stats().shared_accesses
                    now = time.perf_counter() - t0
                    # reports are in canonical order, program first: one slice per job (its
                    # `prog` field stays the job's position in the micro-batch)
                    cut = np.searchsorted(reps["prog"], np.arange(len(take) + 1, dtype=np.uint32))
                    out = [JobResult(reps[cut[k]:cut[k + 1]], arenas[k], int(status[k]), job.arrival, now)
                           for k, job in enumerate(take)]
                    batch.free()
                    gpu_ms = start.elapsed_time(ev)
                    te = time.perf_counter()
                    with lock:
                        for job, r in zip(take, out):
                            latencies.append(r.latency)
                            if on_result is None:
                                results[job.jid] = r
                            else:
                                on_result(job.jid, r)
                        state["accesses"] += acc
                        state["load_s"] += tf - tl
                        state["fetch_s"] += te - tf
                        state["gpu_ms"].append(gpu_ms)
                        state["used"] -= sum(j.log_bytes for j in take)
                        state["busy"] -= 1
                        state["free"].append(wi)
                        lock.notify_all()
                except Exception as e:                    # surfaced by serve() below
                    with lock:
                        state["error"] = e
                        state["busy"] -= 1
                        state["free"].append(wi)
                        lock.notify_all()

        threads = [threading.Thread(target=worker, args=(i,), daemon=True) for i in range(self.max_inflight)]
        for t in threads:
            t.start()
        waiting: collections.deque = collections.deque()
        nb, batch_sizes, nxt = 0, [], 0
        try:
            with lock:
                while nxt < len(jobs) or waiting or state["busy"]:
                    if state["error"] is not None:
                        raise state["error"]
                    now = time.perf_counter() - t0
                    while nxt < len(jobs) and jobs[nxt].arrival <= now:
                        waiting.append(jobs[nxt])
                        nxt += 1
                    dispatched = False
                    while waiting and state["free"]:
                        take, bytes_ = [], 0
                        while (waiting and len(take) < self.max_batch_jobs and
                               state["used"] + bytes_ + waiting[0].log_bytes <= self.budget):
                            j = waiting.popleft()
                            take.append(j)
                            bytes_ += j.log_bytes
                        if not take:
                            break
                        wi = state["free"].pop()
                        state["used"] += bytes_
                        state["peak"] = max(state["peak"], state["used"])
                        state["busy"] += 1
                        state["max_busy"] = max(state["max_busy"], state["busy"])
                        nb += 1
                        batch_sizes.append(len(take))
                        inbox[wi].put(take)
                        dispatched = True
                    if dispatched:
                        continue
                    # sleep until the next arrival or until a worker finishes
                    gap = jobs[nxt].arrival - (time.perf_counter() - t0) if nxt < len(jobs) else 0.01
                    lock.wait(timeout=max(0.0, min(0.01, gap)))
        finally:
            for q in inbox:
                q.put(None)
            for t in threads:
                t.join()
        elapsed = time.perf_counter() - t0
        lat = np.array(latencies) * 1e3
        stats = ServeStats(len(lat), elapsed, len(lat) / elapsed if elapsed else 0.0,
                           float(np.percentile(lat, 50)) if len(lat) else 0.0,
                           float(np.percentile(lat, 99)) if len(lat) else 0.0, state["accesses"],
                           state["accesses"] / elapsed if elapsed else 0.0, nb, state["max_busy"],
                           float(np.mean(batch_sizes)) if batch_sizes else 0.0, state["peak"], state["load_s"],
                           state["fetch_s"], float(np.mean(state["gpu_ms"])) if state["gpu_ms"] else 0.0)
        return results, stats
