"""Autotuner: kernel shapes of a workload picked by measurement.

Four knobs of the library decide how the hot path maps onto the GPU, and the best
setting depends on the workload's block sizes, barrier-interval lengths and shared-array
sizes:

  * interpreter CTAs per SM (``ctas_per_sm``, batched mode) or the register budget of the
    plain interpreter (``interp_variant``): how many simulated blocks share an SM;
  * the race-check kernel shape (``check_variant``): consumer threads per CTA, records per
    stage, staging (TMA ring or registers) and CTAs per SM -- the log-tile width;
  * where the race check runs (``fused_check``): over the access log after the interpreter,
    or inside the interpreter on per-word summaries with no log.

(The race check groups records by their whole 14-bit address in one direct-indexed
table, a one-digit counting sort, so there is no digit width left to choose.)

The stages are separable, so each is tuned on its own time from the library's per-stage
CUDA events: interpreter candidates with the default checker, then every checker
variant behind the fastest interpreter, then the fused check behind that interpreter
shape, kept only if its whole run beats interpreter plus checker.  Every candidate must
produce the same reports
(any difference is a bug, not a tuning outcome).  Choices are cached per workload
signature (device, mode, program shapes) in a JSON file.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

from .workloads.ir import Program

CHECK_VARIANTS = (1, 2, 3, 4, 5, 6, 7)
INTERP_CANDIDATES = {
    "plain": ({"interp_variant": 1}, {"interp_variant": 2}),
    "batched": ({"ctas_per_sm": 1}, {"ctas_per_sm": 2}),
}

# measure(programs, options) -> (ms_interp, ms_check, digest of the reports); raises
# NotApplicable when the library rejects the shape for this workload
Measure = Callable[[Sequence[Program], Dict[str, int]], Tuple[float, float, str]]


class NotApplicable(Exception):
    """The candidate shape cannot run this workload (e.g. a block's shared memory does not fit)."""


@dataclass
class Tuned:
    options: Dict[str, int]                       # keyword options for binding.Context
    interp_ms: Dict[str, float] = field(default_factory=dict)
    check_ms: Dict[str, float] = field(default_factory=dict)
    fused_ms: Optional[float] = None              # interpreter with the fused check, if tried
    cached: bool = False


def signature(programs: Sequence[Program], mode: str, device: str, fused: bool = True) -> str:
    """Digest of what the choice depends on: device, mode and every launch's shape."""
    h = hashlib.sha256(f"{device}|{mode}|{fused}".encode())
    for p in programs:
        h.update(np.int64(p.ncode).tobytes())
        for l in p.launches:
            h.update(np.array([l.kernel, l.grid, l.block_dim, l.shmem_words], np.int64).tobytes())
    return h.hexdigest()[:32]


def gpu_measure(repeats: int = 3) -> Measure:
    """Times one candidate through the C ABI: a warm-up run, then the best of `repeats`."""
    from . import binding

    def measure(programs, options):
        try:
            return _run(programs, options)
        except binding.SimtCheckError as e:
            if e.code == binding.SR_E_INVAL:
                raise NotApplicable(str(e)) from e
            raise

    def _run(programs, options):
        with binding.Context(profile=True, **options) as ctx, ctx.load_programs(programs) as b:
            b.run_and_check()
            reps = b.fetch_reports()
            ti, tc = [], []
            for _ in range(repeats):
                b.run_and_check()
                b.fetch_reports()
                st = b.stats()
                ti.append(st.ms_interp)
                tc.append(st.ms_check)
        return min(ti), min(tc), hashlib.sha256(reps.tobytes()).hexdigest()

    return measure


def _key(opts: Dict[str, int]) -> str:
    return ",".join(f"{k}={v}" for k, v in sorted(opts.items()))


def tune(programs: Sequence[Program], mode: str = "plain", measure: Optional[Measure] = None,
         cache_path: Optional[str] = None, device: Optional[str] = None, fused: bool = True) -> Tuned:
    """Pick interpreter and checker shapes for `programs` in `mode` ('plain' or 'batched');
    `fused` also tries the fused race check."""
    if mode not in INTERP_CANDIDATES:
        raise ValueError(f"unknown mode {mode!r}")
    if device is None:
        import torch
        device = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    sig = signature(programs, mode, device, fused)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if sig in cache:
            return Tuned(dict(cache[sig]), cached=True)
    measure = measure or gpu_measure()

    digests = set()
    out = Tuned({"mode": mode})
    best_i, best_t = None, float("inf")
    for cand in INTERP_CANDIDATES[mode]:
        opts = dict(cand, mode=mode)
        try:
            ti, _, dg = measure(programs, opts)
        except NotApplicable:
            continue
        digests.add(dg)
        out.interp_ms[_key(cand)] = ti
        if ti < best_t:
            best_i, best_t = cand, ti
    if best_i is None:
        raise NotApplicable(f"no interpreter shape of mode {mode!r} can run this workload")
    best_v, best_c = None, float("inf")
    for v in CHECK_VARIANTS:
        opts = dict(best_i, mode=mode, check_variant=v)
        _, tc, dg = measure(programs, opts)
        digests.add(dg)
        out.check_ms[str(v)] = tc
        if tc < best_c:
            best_v, best_c = v, tc
    if len(digests) != 1:
        raise RuntimeError("kernel variants disagree on the reports: a parity bug, not a tuning outcome")
    out.options = dict(best_i, mode=mode, check_variant=best_v)
    if fused:
        try:
            ti, tc, dg = measure(programs, dict(best_i, mode=mode, fused_check=1))
        except NotApplicable:
            ti = None
        if ti is not None:
            digests.add(dg)
            out.fused_ms = ti + tc
            if out.fused_ms < best_t + best_c:
                out.options = dict(best_i, mode=mode, fused_check=1)
    if cache_path:
        cache[sig] = out.options
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return out
