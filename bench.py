"""Benchmark: checked accesses/s and simulated thread-instructions/s, batched vs plain, with
the HBM roofline of the whole hot path.

Default workload (batched): 4096 seed-generated programs (reduction / 1-D stencil radius 1-8
/ 32x32 tiled transpose / 256-bin shared-atomic histogram), grids log-uniform in [1, 4096],
blockDim 32-1024, shared arrays up to 48 KB, 20-400 instructions, 30% with one planted bug
(SplitMix64 seed 3): 1.97M blocks, 1.0e9 simulated threads, 6.1e9 checked shared accesses.
One step = one pass of the whole hot path over the resident batch: arena reset, SIMT
interpretation of every launch with access logging (one persistent launch), race check of
every barrier interval, barrier checks, canonical report ordering.

  value  : checked shared accesses / s, batched path, programs resident on the device
  plain_path : the same programs through one kernel launch per (program, launch)
  e2e    : the same metric through the C ABI from pinned host buffers, per step
           load_programs (H2D) + run_and_check + fetch_reports + fetch_memory of every
           program (D2H)
  roofline : the algorithmic HBM bytes of a step (16 B per checked shared access, 4 B per
             simulated global load or store, 32 B per report, the initial and final arenas)
             over the dominant kernel's (the interpreter's) CUDA-event time, against the
             measured copy bandwidth; beside it the interpreter's issue picture and the race
             check's own HBM roofline
  cpu_baseline : the CPU oracle on the host cores, on a bounded block sample
  clocks       : nvidia-smi samples of the SM clock and throttle reasons while timing

Other workloads (--workload): ``reduction`` = the plain 2^24-element tree reduction (16384 x
1024 threads, missing barrier at level 3), ``stencil2d`` = the 8192^2, 16-launch log-heavy
stencil, ``serving`` = continuous batching at 2000 jobs/s.
Kernel shapes (interpreter CTAs per SM or register budget, race-check variant) are picked
by the autotuner before the timed region unless a shape flag or --no-tune fixes them.
--impl reference times the CPU oracle on a bounded block sample of the same workload.
Under torchrun each rank runs its own copy of the workload (seed + rank): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "checked accesses/sec + sim thread-instr/sec (batched vs plain), HBM % roofline"
UNIT = "accesses/s"
WORKLOADS = {
    "reduction": "plain single program: shared-memory tree reduction over 2^24 int32, 16384 blocks x 1024 threads, "
                 "missing barrier at level 3 (seed 1)",
    "batched": "batched: 4096 seed-generated programs (reduction / 1-D stencil / 32x32 transpose / shared-atomic "
               "histogram), blocks log-uniform 1-4096, blockDim 32-1024, 30% planted bugs (seed 3)",
    "stencil2d": "log-heavy: 2-D 5-point stencil on 8192x8192 int32, 32x32 blocks, 16 launches, staging barrier "
                 "omitted in launch 8 (seed 4)",
    "serving": "serving: Poisson arrivals at 2000 jobs/s (seed 5) of programs from the batched generator "
               "(pool of 512, seed 5), admission by predicted log bytes under a 120 GB budget",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 200 for the native reduction, whose step takes ~4 ms, so "
                         "that the clock samples, taken every 200 ms, fall inside the timed region; else 10)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="batched", choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default="plain", choices=["plain", "batched"])
    ap.add_argument("--interp-variant", type=int, default=0, choices=[0, 1, 2],
                    help="plain interpreter kernel: 1 = one CTA/SM register budget, 2 = two CTAs/SM, 0 = auto")
    ap.add_argument("--ctas-per-sm", type=int, default=0, choices=[0, 1, 2],
                    help="batched mode: 1 = every launch in the persistent interpreter (one CTA per SM), 2 = "
                         "programs of one-group blocks one block per CTA, two CTAs per SM (0 = autotuner)")
    ap.add_argument("--check-variant", type=int, default=0, choices=[0, 1, 2, 3, 4, 5, 6, 7],
                    help="race-check kernel shape (0 = default); setting a shape flag skips the autotuner")
    ap.add_argument("--fused-check", action="store_true",
                    help="race check inside the interpreter on per-word summaries (no access log)")
    ap.add_argument("--no-tune", action="store_true", help="library default shapes instead of the autotuner")
    ap.add_argument("--tune-cache", default=None, help="JSON file caching tuned shapes per workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--global-check", action="store_true",
                    help="measure the workload with the global-memory race check on (sr_opts.check_global)")
    ap.add_argument("--no-global-leg", action="store_true",
                    help="skip the global-memory race check leg (measured on the plain reduction)")
    ap.add_argument("--cpu-sample-blocks", type=int, default=0, help="oracle sample (blocks per launch; 0 = auto)")
    ap.add_argument("--serve-seconds", type=float, default=20.0, help="serving trace length (s)")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="serving arrival rate (jobs/s)")
    ap.add_argument("--serve-runs", type=int, default=3, help="serving: runs of the trace (median reported)")
    ap.add_argument("--serve-inflight", type=int, default=4, help="serving: worker threads (streams)")
    ap.add_argument("--blocks", type=int, default=16384,
                    help="blocks of the reduction (default: the full workload; smaller only for profiling)")
    ap.add_argument("--shard", action="store_true",
                    help="under torchrun: split the one batch across the ranks (strong scaling; programs "
                         "assigned by reserved log bytes) instead of one copy per rank (weak scaling)")
    ap.add_argument("--programs", type=int, default=4096,
                    help="programs of the batched workload, the first N of the same seeded batch "
                         "(default: the full workload; smaller only for profiling)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 200 if args.impl == "native" and args.workload == "reduction" else 10
    return args


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def workload(name: str, rank: int, blocks: int = 16384, programs: int = 4096):
    from paper_1211_6193_gb300.workloads import families, stencil2d
    if name == "reduction":
        return [families.reduction_plain(n_blocks=blocks, bdim=1024, seed=1 + rank, omit_level=3)]
    if name == "batched":
        return families.batch(n_programs=programs, seed=3 + rank)
    if name == "serving":
        return families.batch(n_programs=512, seed=5 + rank)
    return [stencil2d.program(log2w=13, steps=16, buggy_launch=8, seed=4 + rank)]


def workload_label(args):
    if args.workload == "reduction" and args.blocks != 16384:
        return f"reduction, {args.blocks} blocks x 1024 threads (profiling size)"
    if args.workload == "batched" and args.programs != 4096:
        return f"batched, the first {args.programs} of the 4096 seed-generated programs (profiling size)"
    return WORKLOADS[args.workload]


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
        num = lambda x: x.replace(".", "").isdigit()
        sm = [float(r[1]) for r in rows if num(r[1])]
        mx = [float(r[2]) for r in rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------- CPU oracle
# the end-to-end leg splits a batch into this many parts, each on its own context and stream
E2E_PARTS = 4


def oracle_rate(progs, sample_blocks: int, nthreads: int = 0):
    """Oracle on `sample_blocks` blocks of every launch, on `nthreads` host threads (0 = all
    cores)."""
    import oracle
    cores = nthreads or os.cpu_count() or 1
    t0 = time.perf_counter()
    r = oracle.run(progs, max_blocks=sample_blocks, nthreads=cores)
    dt = time.perf_counter() - t0
    return r.shared_accesses / dt, r.thread_instrs / dt, cores, dt, r.shared_accesses


def default_sample(name: str) -> int:
    return {"reduction": 16384, "batched": 4, "stencil2d": 256, "serving": 8}[name]


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    progs = workload(args.workload, 0, args.blocks, args.programs)
    sample = args.cpu_sample_blocks or default_sample(args.workload)
    for _ in range(args.warmup):
        oracle_rate(progs, 1)
    per, acc = [], 0
    cores = os.cpu_count() or 1
    for _ in range(args.steps):
        _, _, cores, dt, n = oracle_rate(progs, sample)
        per.append(dt)
        acc += n
    value = acc / sum(per)
    desc = f"first {sample} blocks of every launch per step, oracle on {cores} host threads"
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(per) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": workload_label(args), "parallelism": "cpu oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


# ----------------------------------------------------------------- GPU
def src_sha(*names):
    h = hashlib.sha1()
    for n in names:
        with open(os.path.join(ROOT, "paper_1211_6193_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_per_launch(workload: str, kernel: str, src: str, units: dict):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu capture (taken
    on a smaller case of the same workload and scaled by its unit, blocks or logged records),
    if one was taken on this source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    for t in json.load(open(path)).get("captures", []):
        if t["workload"] == workload and t["kernel"] == kernel and t["src_sha1"] == src:
            return (t["dram_read"] + t["dram_write"]) / t["units"] * units[t["unit"]]
    return None


def check_kernel(variant: int) -> str:
    """Kernel name of a race-check shape (variants 1-2: TMA ring, 3-5: register-staged, 6-7: lean
    one-warp)."""
    return "k_check" if variant in (1, 2) else "k_check_lean" if variant in (6, 7) else "k_check_reg"


def measure(binding, torch, progs, opts, steps, warmup, flush, stream):
    """Time `steps` runs of run_and_check on resident programs (L2 flushed between steps).
    Every leg starts with PyTorch's cached device blocks released, so that the library's log
    budget (half the free memory by default) and its waves are the same whichever leg ran
    before."""
    torch.cuda.empty_cache()
    ctx = binding.Context(profile=True, use_graph=False, **opts)
    batch = ctx.load_programs(progs)
    for _ in range(max(3, warmup)):
        batch.run_and_check()
    n_reports = len(batch.fetch_reports())
    stats = batch.stats()
    stage = {"reset": [], "interp": [], "check": [], "global": [], "compact": []}
    per_step = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.run_and_check()
        e1.record(stream)
        e1.synchronize()
        per_step.append(e0.elapsed_time(e1))
        s = batch.stats()
        for k in stage:
            stage[k].append(getattr(s, "ms_" + k))
    batch.free()
    ctx.close()
    return stats, n_reports, per_step, {k: statistics.mean(v) for k, v in stage.items()}


def run_serving(args):
    import torch

    from paper_1211_6193_gb300 import serving
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pool = serving.job_pool(512, seed=5 + rank)
    # the jobs' inputs sit in page-locked host memory (as a server's receive buffers would), so
    # that their uploads are DMA copies rather than driver-staged pageable ones
    sizes = [p.global_init.size for p in pool]
    pin = torch.empty(max(1, sum(sizes)), dtype=torch.int32, pin_memory=True).numpy()
    pinned, off = [], 0
    for p, n in zip(pool, sizes):
        v = pin[off:off + n]
        v[:] = p.global_init
        pinned.append(type(p)(p.code, p.kernel_entry, p.launches, v, p.name))
        off += n
    pool = pinned
    arrivals = serving.poisson_trace(args.serve_rate, args.serve_seconds, seed=5 + rank)
    jobs = [serving.Job(k, pool[k % len(pool)], t) for k, t in enumerate(arrivals)]
    shapes = {"check_variant": args.check_variant} if args.check_variant else {}
    srv = serving.Server(log_budget_bytes=120 << 30, max_inflight=args.serve_inflight, **shapes)
    # warm-up: load the kernels, then two seconds of the trace (fills the page-locked host cache
    # and the contexts' device pools with the sizes the runs will ask for)
    srv.serve([serving.Job(k, pool[k], 0.0) for k in range(16)])
    srv.serve([serving.Job(j.jid, j.program, j.arrival) for j in jobs if j.arrival < 2.0])
    runs = []
    with ClockSampler(local) as clocks:
        for _ in range(args.serve_runs):
            torch.cuda.synchronize()
            _, st = srv.serve(jobs, on_result=lambda jid, r: None)  # latency recorded, result dropped
            torch.cuda.synchronize()
            runs.append(st)
    srv.close()
    med = sorted(runs, key=lambda r: r.accesses_per_s)[len(runs) // 2]
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": med.accesses_per_s * world, "unit": UNIT, "n_gpus": world,
            "steps": len(runs), "warmup": 1, "ms_per_step": med.seconds * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOADS["serving"].replace("2000 jobs/s", f"{args.serve_rate:g} jobs/s"),
                       "trace_seconds": args.serve_seconds, "jobs": med.jobs, "runs": len(runs),
                       "workers": args.serve_inflight, "shapes": shapes or "library default",
                       "inputs": "page-locked host memory", "value": "the run with the median throughput"},
            "serving": {"p50_latency_ms": med.p50_ms, "p99_latency_ms": med.p99_ms, "jobs_per_s": med.jobs_per_s,
                        "p50_latency_ms_runs": [r.p50_ms for r in runs],
                        "p99_latency_ms_runs": [r.p99_ms for r in runs],
                        "jobs_per_s_runs": [r.jobs_per_s for r in runs],
                        "batches": med.batches, "mean_batch_jobs": med.mean_batch_jobs,
                        "max_inflight_batches": med.max_inflight_seen, "peak_log_bytes": med.peak_log_bytes,
                        "worker_load_s": med.host_load_s, "worker_fetch_s": med.host_fetch_s,
                        "mean_batch_gpu_ms": med.mean_batch_gpu_ms},
            "clocks": clocks.summary()}), flush=True)


def run_native(args):
    import torch

    from paper_1211_6193_gb300 import autotune, binding
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    shard = args.shard and world > 1 and args.workload == "batched"
    if shard:
        from paper_1211_6193_gb300 import dist as sdist
        progs = workload(args.workload, 0, args.blocks, args.programs)
        progs = [progs[i] for i in sdist.shard(progs, world)[rank]]
    else:
        progs = workload(args.workload, rank, args.blocks, args.programs)
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(pk)) if os.path.exists(pk) else {}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)     # > 129 MB L2
    nblocks = sum(l.grid for p in progs for l in p.launches)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    mode = "batched" if args.workload == "batched" else args.mode

    def shapes(m):
        """Kernel shapes for mode m: fixed by the flags, else picked by the autotuner (untimed)."""
        if args.interp_variant or args.check_variant or args.ctas_per_sm or args.no_tune or args.fused_check:
            o = {"mode": m, "interp_variant": args.interp_variant, "check_variant": args.check_variant}
            if args.ctas_per_sm:
                o["ctas_per_sm"] = args.ctas_per_sm
            if args.fused_check:
                o["fused_check"] = 1
            return o, "flags"
        sample = progs[::8] if len(progs) >= 64 else progs     # a strided eighth keeps the mix
        t = autotune.tune(sample, m, cache_path=args.tune_cache)
        return dict(t.options), ("cache" if t.cached else {"interp_ms": t.interp_ms, "check_ms": t.check_ms,
                                                           "fused_ms": t.fused_ms})

    opts, tuning = shapes(mode)
    if args.global_check:
        opts["check_global"] = 1
    with ClockSampler(local) as clocks:
        barrier()
        t_wall = time.perf_counter()
        st, n_reports, per_step, stage = measure(binding, torch, progs, opts, args.steps, args.warmup, flush, stream)
        barrier()
        t_wall = time.perf_counter() - t_wall
    clk = clocks.summary()
    dev_ms = sum(per_step)
    all_acc, all_instr = st.shared_accesses, st.thread_instrs
    if world > 1:
        t = torch.tensor([dev_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        dev_ms = float(t.item())
        n = torch.tensor([float(all_acc), float(all_instr)], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(n, op=torch.distributed.ReduceOp.SUM)
        all_acc, all_instr = int(n[0].item()), int(n[1].item())
    value = all_acc * args.steps / (dev_ms / 1e3)              # whole job: every rank's accesses
    thread_instr_rate = all_instr * args.steps / (dev_ms / 1e3)

    plain = None
    if args.workload == "batched":     # the same programs through one kernel launch per (program, launch)
        popts, _ = shapes("plain")
        pst, _, pper, pstage = measure(binding, torch, progs, popts, max(2, args.steps // 2), 1, flush, stream)
        pms = sum(pper) / len(pper)
        plain = {"value": pst.shared_accesses / (pms / 1e3), "ms_per_step": pms, "stage_ms": pstage,
                 "batched_speedup": pms / (dev_ms / args.steps), "shapes": popts, "waves": pst.waves}

    # ---- roofline of the whole hot path (HBM): the algorithmic bytes of one step, over the
    # dominant kernel's (the interpreter's) CUDA-event time, against the measured copy bandwidth
    arena_words = sum((p.global_init.size + 3) & ~3 for p in progs)
    alg = {"checked_shared_access": 16, "simulated_global_access": 4, "report": 32, "arena_word": 8}
    step_bytes = (alg["checked_shared_access"] * st.shared_accesses + alg["simulated_global_access"] *
                  st.global_accesses + alg["report"] * n_reports + alg["arena_word"] * arena_words)
    # (batched mode with two CTAs per SM: the interpreter stage is two kernels, the one-block-per-CTA
    # grid of the programs of one-group blocks, then the persistent kernel for the rest)
    interp_kernel = ("k_interp_plain" if mode == "plain" else
                     "k_interp_blocks + k_interp_batched" if opts.get("ctas_per_sm") == 2 else "k_interp_batched")
    achieved = step_bytes / (stage["interp"] / 1e3) / 1e9
    isha, csha = src_sha("interp.cu", "sr_internal.h"), src_sha("check.cu", "sr_internal.h")
    fused = bool(opts.get("fused_check"))
    units = {"block": nblocks, "record": st.shared_accesses}
    int_peak = 152 * 128 * sm_max * 1e6            # int32 lane-ops/s: 152 SMs x 128 lanes x max clock
    roofline = {
        "bound": "hbm", "kernel": interp_kernel, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
        "frac": achieved / hbm_peak, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs, copy)",
        "traffic": None if fused else traffic_per_launch(args.workload, interp_kernel, isha, units),
        "algorithmic_bytes_per_step": step_bytes,
        "algorithmic_bytes": "16 B per checked shared access (8 B record written + read), 4 B per simulated "
                             "global load/store, 32 B per report, 8 B per arena word (initial read + final write)",
        "step_frac": step_bytes / (dev_ms / args.steps / 1e3) / 1e9 / hbm_peak,
        "stage_ms": stage,
        "interpreter_issue": {
            "sim_thread_instrs_per_s": st.thread_instrs / (stage["interp"] / 1e3),
            "int32_lane_peak": int_peak, "frac_of_lane_peak": st.thread_instrs / (stage["interp"] / 1e3) / int_peak,
            "note": "issue-bound: real warp-instructions per simulated warp-instruction and issue-active % are "
                    "in profiles/ (ncu, small case)"},
    }
    if fused:      # races decided inside the interpreter: no log is written, the check stage only skips
        roofline["checker"] = {"bound": None, "kernel": None, "stage_ms": stage["check"],
                               "note": "fused race check: no access log written or read"}
    else:
        check_bytes = 8 * st.shared_accesses + 16 * n_reports
        check_gbs = check_bytes / (stage["check"] / 1e3) / 1e9 if stage["check"] > 0 else 0.0
        roofline["checker"] = {
            "bound": "hbm", "kernel": check_kernel(opts.get("check_variant", 0)), "achieved": check_gbs,
            "peak": hbm_peak, "unit": "GB/s", "frac": check_gbs / hbm_peak, "peak_source": peak_src,
            "algorithmic_bytes": "8 B read per logged access + 16 B per race entry",
            "traffic": traffic_per_launch(args.workload, check_kernel(opts.get("check_variant", 0)), csha, units)}

    # ---- the global-memory race check (sr_opts.check_global) as a leg of its own, on the plain
    # reduction (2^24 global loads + 16384 stores per step): its stage time and HBM roofline,
    # 32 algorithmic bytes per logged global access (16 B record written once and read once)
    global_leg = None
    if args.workload == "batched" and not args.no_global_leg:
        gprogs = workload("reduction", rank)
        gopts = {"mode": "plain", "interp_variant": 2, "check_variant": 6, "check_global": 1}
        gst, gn, gper, gstage = measure(binding, torch, gprogs, gopts, 3, 1, flush, stream)
        ms_g = gstage["global"]
        gbs = 32 * gst.global_records / (ms_g / 1e3) / 1e9 if ms_g > 0 else 0.0
        global_leg = {"workload": WORKLOADS["reduction"], "records_per_step": gst.global_records,
                      "stage_ms": gstage, "ms_per_step": statistics.mean(gper), "reports_per_step": gn,
                      "roofline": {"bound": "hbm", "kernels": "k_ggather, k_rs_upsweep, k_rs_pass, k_grun",
                                   "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                                   "algorithmic_bytes": "32 B per logged global access (16 B record written, "
                                                        "read once); radix passes beyond that are "
                                                        "implementation cost"}}

    # ---- end to end through the C ABI from page-locked host buffers, per step: load_programs
    # (code and initial arenas host -> device), run_and_check, fetch_reports and one fetch of
    # every final arena (device -> host).  Timed two ways: the whole batch as one call sequence,
    # and split in E2E_PARTS parts (balanced by reserved log bytes) on as many contexts and
    # streams, each part's uploads, downloads and host work overlapping the others' kernels -
    # the `e2e` figure.  Device memory from the contexts' stream-ordered pools (the C ABI default).
    sizes = [p.global_init.size for p in progs]
    pin = torch.empty(max(1, sum(sizes)), dtype=torch.int32, pin_memory=True).numpy()
    progs_pinned, off = [], 0
    for p, n in zip(progs, sizes):
        v = pin[off:off + n]
        v[:] = p.global_init
        progs_pinned.append(type(p)(p.code, p.kernel_entry, p.launches, v, p.name))
        off += n
    h2d = sum(p.global_init.nbytes + p.code.nbytes for p in progs)
    d2h = 4 * sum((n + 3) & ~3 for n in sizes) + 32 * n_reports

    def e2e_time(groups):
        ctxs = [binding.Context(report_cap=max(16, n_reports), torch_allocator=False, **opts) for _ in groups]
        streams = [torch.cuda.current_stream()] if len(groups) == 1 else [torch.cuda.Stream() for _ in groups]
        times = []
        for i in range(1 + min(args.steps, 5)):
            barrier()
            t0 = time.perf_counter()
            batches = []
            for g, c, s in zip(groups, ctxs, streams):
                b = c.load_programs(g, stream=s)
                b.run_and_check(stream=s)
                batches.append(b)
            for b in batches:
                b.fetch_reports(pinned=True)
                b.fetch_all_memory(pinned=True)
                b.free()
            torch.cuda.synchronize()
            if i:
                times.append(time.perf_counter() - t0)
        for c in ctxs:
            c.close()
        t = statistics.mean(times)
        if world > 1:
            tt = torch.tensor([t], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
            t = float(tt.item())
        return t

    torch.cuda.empty_cache()
    t_single = e2e_time([progs_pinned])
    e2e = {"value": all_acc / t_single, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "form": "one batch"}
    if len(progs_pinned) >= E2E_PARTS:
        from paper_1211_6193_gb300 import dist as sdist
        parts = [[progs_pinned[i] for i in idx] for idx in sdist.shard(progs, E2E_PARTS)]
        torch.cuda.empty_cache()
        t_pipe = e2e_time(parts)
        e2e = {"value": all_acc / t_pipe, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h),
               "form": f"{E2E_PARTS} part-batches on {E2E_PARTS} streams (the copies and host work of each "
                       "overlap the others' kernels)", "one_batch_value": all_acc / t_single}
    del pin, progs_pinned

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = args.cpu_sample_blocks or default_sample(args.workload)
        rate, irate, cores, dt, n = oracle_rate(progs, sample)
        # and on one thread, on a quarter of that sample (the oracle as written, no threads)
        s1 = max(1, sample // 4)
        rate1, _, _, dt1, n1 = oracle_rate(progs, s1, nthreads=1)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {sample} blocks of every launch ({n} accesses, {dt:.1f} s)",
               "thread_instrs_per_s": irate,
               "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                 "sample": f"first {s1} blocks of every launch ({n1} accesses, {dt1:.1f} s)"}}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if shard else "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": workload_label(args), "mode": mode, "shapes": opts, "tuning": tuning,
                       "blocks": nblocks,
                       "programs": len(progs),
                       "parallelism": (f"{world} ranks, one batch sharded by reserved log bytes" if shard else
                                       f"{world} independent replicas") if world > 1 else "single GPU",
                       "l2": "flushed between timed steps (256 MB write); logs exceed L2"},
            "sim_thread_instrs_per_s": thread_instr_rate, "shared_accesses_per_step": st.shared_accesses,
            "reports_per_step": n_reports, "wall_s": t_wall, "e2e": e2e, "roofline": roofline,
            "cpu_baseline": cpu, "clocks": clk,
            "gpu_launches": args.steps * st.kernels, "waves": st.waves}
    if plain is not None:
        line["plain_path"] = plain
    if global_leg is not None:
        line["global_check"] = global_leg
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
