"""Benchmark: checked shared accesses per second on the plain single-program workload.

Workload: a shared-memory tree reduction over 2^24 int32 values uniform in [0, 100)
(SplitMix64 seed 1), 16384 blocks x 1024 threads, the barrier after level 3 missing
(so every block reports 32 races).  One step = one pass of the whole hot path: arena
reset, SIMT interpretation with access logging, race check of every barrier interval,
barrier checks, canonical report ordering.

  value  : checked shared accesses / s with programs resident on the device
  e2e    : the same metric through the C ABI from pinned host buffers, per step
           load_programs (H2D) + run_and_check + fetch_reports + fetch_memory (D2H)
  roofline / cpu_baseline / clocks as described in the design doc

--impl reference times the CPU oracle on a bounded block sample of the same workload.
Under torchrun each rank runs its own copy of the workload (seed 1 + rank): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "checked shared accesses/s (race-checked SIMT interpretation)"
UNIT = "accesses/s"
WORKLOAD = "plain single program: shared-memory tree reduction over 2^24 int32, 16384 blocks x 1024 threads, " \
           "missing barrier at level 3 (seed 1)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--mode", default="plain", choices=["plain", "batched"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-blocks", type=int, default=16384)
    ap.add_argument("--interp-variant", type=int, default=0, choices=[0, 1, 2],
                    help="plain interpreter kernel: 1 = one CTA/SM register budget, 2 = two CTAs/SM, 0 = auto")
    ap.add_argument("--blocks", type=int, default=16384,
                    help="blocks of the reduction (default: the full 2^24-element workload; smaller only "
                         "for profiling captures)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(rank: int, blocks: int = 16384):
    from paper_1211_6193_gb300.workloads import families
    return families.reduction_plain(n_blocks=blocks, bdim=1024, seed=1 + rank, omit_level=3)


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------- CPU oracle
def oracle_rate(prog, sample_blocks: int):
    import oracle
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    r = oracle.run([prog], max_blocks=sample_blocks, nthreads=cores)
    dt = time.perf_counter() - t0
    return r.shared_accesses / dt, r.thread_instrs / dt, cores, dt, r.shared_accesses


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    prog = workload(0, args.blocks)
    for _ in range(args.warmup):
        oracle_rate(prog, 64)
    per = []
    acc = ins = 0
    for _ in range(args.steps):
        rate, irate, cores, dt, n = oracle_rate(prog, args.cpu_sample_blocks)
        per.append(dt)
        acc += n
    total = sum(per)
    value = acc / total
    sample = f"blocks 0..{args.cpu_sample_blocks - 1} of the workload per step, oracle on {cores} host threads"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "parallelism": "cpu oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU
def run_native(args):
    import numpy as np
    import torch

    from paper_1211_6193_gb300 import binding
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    prog = workload(rank, args.blocks)
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    ctx = binding.Context(mode=args.mode, profile=True, interp_variant=args.interp_variant)
    batch = ctx.load_programs([prog])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)     # > 129 MB L2
    for _ in range(max(3, args.warmup)):
        batch.run_and_check()
    n_reports = len(batch.fetch_reports())
    st = batch.stats()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    stage = {"interp": [], "check": [], "compact": [], "reset": []}
    per_step = []
    with ClockSampler(local) as clocks:
        barrier()
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.run_and_check()
            e1.record(stream)
            e1.synchronize()
            per_step.append(e0.elapsed_time(e1))
            s = batch.stats()
            stage["interp"].append(s.ms_interp)
            stage["check"].append(s.ms_check)
            stage["compact"].append(s.ms_compact)
            stage["reset"].append(s.ms_reset)
        barrier()
        t_wall = time.perf_counter() - t_wall
    clk = clocks.summary()
    dev_ms = sum(per_step)
    if world > 1:
        t = torch.tensor([dev_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        dev_ms = float(t.item())
    acc_per_step = st.shared_accesses
    value = world * acc_per_step * args.steps / (dev_ms / 1e3)
    thread_instr_rate = world * st.thread_instrs * args.steps / (dev_ms / 1e3)

    # ---- roofline of the dominant kernel (algorithmic bytes / CUDA-event duration)
    interp_ms = statistics.mean(stage["interp"])
    check_ms = statistics.mean(stage["check"])
    compact_ms = statistics.mean(stage["compact"])
    dominant = max((interp_ms, "interpreter"), (check_ms, "race check"), (compact_ms, "compaction"))
    interp_bytes = 8 * st.shared_accesses + 4 * st.global_accesses
    check_bytes = 8 * st.shared_accesses + 16 * (n_reports)
    compact_bytes = 16 * n_reports + 32 * n_reports
    dom_bytes, dom_ms = {"interpreter": (interp_bytes, interp_ms), "race check": (check_bytes, check_ms),
                         "compaction": (compact_bytes, compact_ms)}[dominant[1]]
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": dominant[1], "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None, "peak_source": peak_src,
                "stage_ms": {"reset": statistics.mean(stage["reset"]), "interp": interp_ms, "check": check_ms,
                             "compact": compact_ms},
                "checker_hbm_frac": (check_bytes / (check_ms / 1e3) / 1e9) / hbm_peak if check_ms > 0 else None}

    # ---- end to end through the C ABI from pinned host buffers
    arena_pinned = torch.empty(prog.global_init.size, dtype=torch.int32, pin_memory=True)
    arena_pinned.numpy()[:] = prog.global_init
    prog_pinned = type(prog)(prog.code, prog.kernel_entry, prog.launches, arena_pinned.numpy(), prog.name)
    out_arena = torch.empty(prog.global_init.size, dtype=torch.int32, pin_memory=True).numpy()
    h2d = prog.global_init.nbytes + prog.code.nbytes
    d2h = out_arena.nbytes + n_reports * 32
    e2e_times = []
    ctx_e2e = binding.Context(mode=args.mode, report_cap=max(16, n_reports), interp_variant=args.interp_variant)
    for i in range(1 + min(args.steps, 5)):
        barrier()
        t0 = time.perf_counter()
        with ctx_e2e.load_programs([prog_pinned]) as b:
            b.run_and_check()
            reps = b.fetch_reports()
            b.fetch_memory(0, out_arena)
        torch.cuda.synchronize()
        if i:
            e2e_times.append(time.perf_counter() - t0)
    e2e_value = world * acc_per_step / statistics.mean(e2e_times)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, irate, cores, dt, n = oracle_rate(prog, args.cpu_sample_blocks)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"blocks 0..{args.cpu_sample_blocks - 1} of the workload ({n} accesses, {dt:.1f} s)",
               "thread_instrs_per_s": irate}
    kernels_per_step = 6 if args.mode == "plain" else 6
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.blocks == 16384 else f"reduction, {args.blocks} blocks x 1024",
                       "mode": args.mode, "blocks": args.blocks, "threads_per_block": 1024,
                       "parallelism": f"{world} independent replicas" if world > 1 else "single GPU",
                       "l2": "flushed between timed steps (256 MB write), log > L2"},
            "sim_thread_instrs_per_s": thread_instr_rate,
            "shared_accesses_per_step": acc_per_step, "reports_per_step": n_reports,
            "wall_s": t_wall,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clk,
            "gpu_launches": kernels_per_step * args.steps}
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.free()
    ctx.close()
    ctx_e2e.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
