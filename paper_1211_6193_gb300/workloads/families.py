"""Seeded generators of simulated CUDA programs: the four kernel families of the batched
workload, the plain 2^24-element reduction, and planted-bug variants.

These build *inputs* only (IR code, launch configuration, initial arena); they hold
none of the checker's logic.  Register conventions: r0/r1 = kernel params (input and
output word offsets), r2 = tid, r3 = bid, r13..r15 scratch; block-size-dependent
constants are folded into immediates by the generator.

Planted bugs (Sec. 3.2 shows the first and last kind on Fig. 1):
* ``missing_barrier`` - one ``__syncthreads()`` removed;
* ``off_by_one``      - a bound or index one past its correct value;
* ``divergent_barrier`` - a ``__syncthreads()`` reached by only part of the block.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional, Tuple

import numpy as np

from . import rng
from .ir import (BDIM, BID, TID, MAX_SHMEM_WORDS, Asm, Launch, Program, RZ, r0, r1, r2, r3, r4, r5, r6,
                 r7, r8, r9, r10, r11, r12, r13, r14, r15)

FAMILIES = ("reduction", "stencil1d", "transpose", "histogram")
BUGS = ("missing_barrier", "off_by_one", "divergent_barrier")


def _filler(a: Asm, n: int) -> None:
    """n straight-line ALU instructions on scratch registers (LCG steps on r15)."""
    for i in range(n):
        if i % 2 == 0:
            a.mul(r15, r15, 1103515245)
        else:
            a.add(r15, r15, 12345)


def _divergent_guard(a: Asm, bdim: int, tag: str) -> None:
    """A barrier executed only by threads tid < bdim/2 (bdim >= 32 so both halves exist)."""
    a.slt(r14, r2, max(1, bdim // 2)).brz(r14, f"div_{tag}").bar().label(f"div_{tag}")


# ------------------------------------------------------------------ reduction
def reduction_kernel(bdim: int, omit_barrier_level: Optional[int] = None,
                     off_by_one_level: Optional[int] = None, divergent_level: Optional[int] = None,
                     filler: int = 0, use_bdim_sreg: bool = False) -> Asm:
    """Shared-memory tree reduction of ``in[bid*bdim .. +bdim)`` into ``out[bid]``.

    Level l (0-based) uses stride s = P/2^(l+1), P = next power of two >= bdim; threads
    with tid < min(s, bdim - s) add sh[tid + s] into sh[tid]; a barrier closes each level.
    """
    a = Asm()
    a.s2r(r2, TID).s2r(r3, BID)
    _filler(a, filler)
    if use_bdim_sreg:
        a.s2r(r4, BDIM).mul(r5, r3, r4)
    else:
        a.mul(r5, r3, bdim)
    a.add(r5, r5, r2).add(r5, r5, r0).ldg(r6, r5).sts(r2, r6).bar()
    P = 1 << max(0, (bdim - 1).bit_length())
    s, level = P // 2, 0
    while s >= 1:
        lim = min(s, bdim - s)
        if level == off_by_one_level:
            a.sle(r8, r2, lim)
        else:
            a.slt(r8, r2, lim)
        a.brz(r8, f"skip{level}")
        if level == divergent_level:
            a.bar()
        a.lds(r10, r2).lds(r11, r2, s).add(r10, r10, r11).sts(r2, r10)
        a.label(f"skip{level}")
        if level != omit_barrier_level:
            a.bar()
        s //= 2
        level += 1
    a.brnz(r2, "done").lds(r10, RZ).add(r5, r1, r3).stg(r5, r10).label("done").exit()
    return a


def reduction_levels(bdim: int) -> int:
    return max(0, (bdim - 1).bit_length())


def reduction_plain(n_blocks: int = 16384, bdim: int = 1024, seed: int = 1, omit_level: Optional[int] = 3,
                    values: Optional[np.ndarray] = None) -> Program:
    """The plain single-program workload: tree reduction over n_blocks*bdim int32 values
    uniform in [0, 100) from SplitMix64(seed) (``(x >> 32) % 100``), one missing barrier
    (after level ``omit_level``, stride 64 for bdim 1024)."""
    n = n_blocks * bdim
    if values is None:
        values = rng.uniform_mod(seed, n, 100)
    arena = np.zeros(n + n_blocks, dtype=np.int32)
    arena[:n] = values
    code = reduction_kernel(bdim, omit_barrier_level=omit_level).assemble()
    return Program(code, [0], [Launch(0, n_blocks, bdim, bdim, (0, n))], arena,
                   name=f"reduction_{n_blocks}x{bdim}", meta={"family": "reduction", "n": n})


# ------------------------------------------------------------------ 1-D stencil
def stencil1d_kernel(bdim: int, radius: int, n_total: int, bug: Optional[str] = None, filler: int = 0) -> Asm:
    """out[g] = sum_{j=-r..r} in[g+j] (zero outside [0, n_total)), via a shared tile with halo."""
    r = radius
    a = Asm()
    a.s2r(r2, TID).s2r(r3, BID)
    _filler(a, filler)
    a.mul(r5, r3, bdim).add(r5, r5, r2)                  # gid
    a.add(r6, r5, r0).ldg(r7, r6).sts(r2, r7, r)         # sh[tid + r] = in[gid]
    a.slt(r8, r2, r).brz(r8, "no_left")                  # left halo: tid < r
    if bug == "divergent_barrier":
        a.bar()
    a.mov(r9, 0).slt(r10, r5, r).brnz(r10, "left_zero").ldg(r9, r6, -r).label("left_zero")
    a.sts(r2, r9).label("no_left")
    a.slt(r8, r2, bdim - r).brnz(r8, "no_right")        # right halo: tid >= bdim - r
    a.mov(r9, 0).slt(r10, r5, n_total - r).brz(r10, "right_zero").ldg(r9, r6, r).label("right_zero")
    a.sts(r2, r9, 2 * r).label("no_right")
    if bug != "missing_barrier":
        a.bar()
    taps = 2 * r + 1 + (1 if bug == "off_by_one" else 0)
    a.lds(r11, r2, 0)
    for j in range(1, taps):
        a.lds(r12, r2, j).add(r11, r11, r12)
    a.add(r6, r5, r1).stg(r6, r11).exit()
    return a


# ------------------------------------------------------------------ tiled transpose
def transpose_kernel(bdim: int, bug: Optional[str] = None, filler: int = 0) -> Asm:
    """Block b transposes its 32x32 tile: out[b][y][x] = in[b][x][y], through a 32x33 tile."""
    assert bdim % 32 == 0
    tyn = bdim // 32
    iters = -(-32 // tyn)
    a = Asm()
    a.s2r(r2, TID).s2r(r3, BID)
    _filler(a, filler)
    a.and_(r4, r2, 31).shr(r5, r2, 5)                     # tx, ty
    a.shl(r6, r3, 10).add(r6, r6, r0)                     # in tile base
    a.shl(r7, r3, 10).add(r7, r7, r1)                     # out tile base
    for c in range(iters):
        y0 = c * tyn
        if y0 + tyn > 32:
            a.slt(r8, r5, 32 - y0).brz(r8, f"ld_skip{c}")
        a.add(r9, r5, y0).shl(r10, r9, 5).add(r10, r10, r4).add(r10, r10, r6).ldg(r11, r10)
        a.mul(r12, r9, 33).add(r12, r12, r4).sts(r12, r11)    # tile[y][x]
        if y0 + tyn > 32:
            a.label(f"ld_skip{c}")
    if bug == "divergent_barrier":
        _divergent_guard(a, bdim, "t")
    if bug != "missing_barrier":
        a.bar()
    for c in range(iters):
        y0 = c * tyn
        if y0 + tyn > 32:
            a.slt(r8, r5, 32 - y0).brz(r8, f"st_skip{c}")
        a.add(r9, r5, y0).mul(r12, r4, 33).add(r12, r12, r9)
        if bug == "off_by_one":
            a.lds(r11, r12, 1)                                # tile[x][y + 1]
        else:
            a.lds(r11, r12)                                   # tile[x][y]
        a.shl(r10, r9, 5).add(r10, r10, r4).add(r10, r10, r7).stg(r10, r11)
        if y0 + tyn > 32:
            a.label(f"st_skip{c}")
    a.exit()
    return a


# ------------------------------------------------------------------ shared-atomic histogram
def histogram_kernel(bdim: int, elems: int, bug: Optional[str] = None, bug_at: int = 0, filler: int = 0) -> Asm:
    """256-bin histogram of ``in[(bid*bdim + tid)*elems + e] & 255`` with shared atomics;
    out[bid*256 + i] = bin i.  ``bug_at`` picks which of the two barriers a bug touches."""
    a = Asm()
    a.s2r(r2, TID).s2r(r3, BID)
    _filler(a, filler)
    a.mov(r13, 1)
    zero_iters = -(-256 // bdim)
    for c in range(zero_iters):
        if (c + 1) * bdim > 256:
            a.slt(r8, r2, 256 - c * bdim).brz(r8, f"z_skip{c}")
        a.sts(r2, RZ, c * bdim)
        if (c + 1) * bdim > 256:
            a.label(f"z_skip{c}")
    if bug == "divergent_barrier" and bug_at == 0:
        _divergent_guard(a, bdim, "h0")
    if not (bug == "missing_barrier" and bug_at == 0):
        a.bar()
    a.mul(r5, r3, bdim).add(r5, r5, r2).mul(r5, r5, elems).add(r5, r5, r0)
    for e in range(elems):
        a.ldg(r6, r5, e).and_(r6, r6, 255)
        if bug == "off_by_one":
            a.add(r6, r6, 1)
        a.atoms(r6, r13)
    if bug == "divergent_barrier" and bug_at == 1:
        _divergent_guard(a, bdim, "h1")
    if not (bug == "missing_barrier" and bug_at == 1):
        a.bar()
    a.shl(r7, r3, 8).add(r7, r7, r1).add(r7, r7, r2)
    for c in range(zero_iters):
        if (c + 1) * bdim > 256:
            a.slt(r8, r2, 256 - c * bdim).brz(r8, f"o_skip{c}")
        a.lds(r9, r2, c * bdim).stg(r7, r9, c * bdim)
        if (c + 1) * bdim > 256:
            a.label(f"o_skip{c}")
    a.exit()
    return a


# ------------------------------------------------------------------ family programs
@dataclass
class FamilySpec:
    family: str
    grid: int
    bdim: int
    shmem_words: int
    target_len: int
    bug: Optional[str]
    bug_arg: int
    radius: int = 0
    elems: int = 1


def _need_words(spec: FamilySpec) -> int:
    if spec.family == "reduction":
        return spec.bdim
    if spec.family == "stencil1d":
        return spec.bdim + 2 * spec.radius
    if spec.family == "transpose":
        return 32 * 33
    return 256


def build_family(spec: FamilySpec, seed: int) -> Program:
    """Assemble one family program and its seeded input arena."""
    g, b = spec.grid, spec.bdim

    def assemble(filler: int) -> Asm:
        if spec.family == "reduction":
            nl = reduction_levels(b)
            lvl = spec.bug_arg % max(1, nl)
            return reduction_kernel(
                b, omit_barrier_level=lvl if spec.bug == "missing_barrier" else None,
                off_by_one_level=lvl if spec.bug == "off_by_one" else None,
                divergent_level=lvl if spec.bug == "divergent_barrier" else None, filler=filler)
        if spec.family == "stencil1d":
            return stencil1d_kernel(b, spec.radius, g * b, spec.bug, filler)
        if spec.family == "transpose":
            return transpose_kernel(b, spec.bug, filler)
        return histogram_kernel(b, spec.elems, spec.bug, spec.bug_arg % 2, filler)

    base_len = len(assemble(0).code)
    code = assemble(max(0, spec.target_len - base_len)).assemble()
    if spec.family == "reduction":
        n_in, n_out = g * b, g
        vals = rng.uniform_mod(seed, n_in, 100)
    elif spec.family == "stencil1d":
        n_in, n_out = g * b, g * b
        vals = rng.uniform_range(seed, n_in, -1000, 1000)
    elif spec.family == "transpose":
        n_in, n_out = g * 1024, g * 1024
        vals = rng.uniform_i32(seed, n_in)
    else:
        n_in, n_out = g * b * spec.elems, g * 256
        vals = rng.uniform_i32(seed, n_in)
    arena = np.zeros(n_in + n_out, dtype=np.int32)
    arena[:n_in] = vals
    meta = {"family": spec.family, "bug": spec.bug, "bug_arg": spec.bug_arg, "radius": spec.radius,
            "elems": spec.elems, "n_in": n_in, "n_out": n_out}
    return Program(code, [0], [Launch(0, g, b, spec.shmem_words, (0, n_in))], arena,
                   name=f"{spec.family}_g{g}_b{b}" + (f"_{spec.bug}" if spec.bug else ""), meta=meta)


def draw_spec(seed: int, max_grid: int = 4096, bug_rate: float = 0.3,
              families: Tuple[str, ...] = FAMILIES) -> FamilySpec:
    """Draw one program's shape: family uniform; grid = floor(2^(12u)) clamped to
    [1, max_grid]; blockDim = 32*U{1..32}; shared words uniform in [need, 48 KB];
    static length uniform in [20, 400]; with probability ``bug_rate`` one planted bug."""
    R = rng.SplitMix64(seed)
    fam = families[R.randint(0, len(families) - 1)]
    grid = int(math.floor(2.0 ** (12.0 * R.uniform())))
    grid = max(1, min(max_grid, grid))
    bdim = 32 * R.randint(1, 32)
    radius = R.randint(1, 8)
    elems = R.randint(1, 8)
    target = R.randint(20, 400)
    bug = BUGS[R.randint(0, 2)] if R.uniform() < bug_rate else None
    bug_arg = R.randint(0, 1 << 20)
    spec = FamilySpec(fam, grid, bdim, 0, target, bug, bug_arg, radius, elems)
    need = _need_words(spec)
    spec.shmem_words = R.randint(need, MAX_SHMEM_WORDS)
    return spec


def batch(n_programs: int = 4096, seed: int = 3, max_grid: int = 4096, bug_rate: float = 0.3,
          families: Tuple[str, ...] = FAMILIES, indices=None) -> List[Program]:
    """The batched workload: program i drawn from SplitMix64 sub-stream (seed, i).  With
    ``indices``, only those programs of the n_programs (the same ones, in that order)."""
    out = []
    for i in (range(n_programs) if indices is None else indices):
        s = rng.derive(seed, i)
        out.append(build_family(draw_spec(s, max_grid, bug_rate, families), s))
    return out
