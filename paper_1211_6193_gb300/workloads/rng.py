"""SplitMix64: the seeded generator behind every synthetic input.

Published definition (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; the 64-bit finaliser constants as in Vigna's public
reference code): state += 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds
and a final xor-shift.  Written here from that definition; it carries none of the
checker's arithmetic.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB


def _mix(z: int) -> int:
    z = ((z ^ (z >> 30)) * M1) & MASK64
    z = ((z ^ (z >> 27)) * M2) & MASK64
    return z ^ (z >> 31)


class SplitMix64:
    """Scalar stream: output i (0-based) is mix(seed + (i + 1) * GAMMA)."""

    def __init__(self, seed: int) -> None:
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + GAMMA) & MASK64
        return _mix(self.state)

    def randint(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi] (inclusive) from the high 32 bits."""
        return lo + (self.next_u64() >> 32) % (hi - lo + 1)

    def uniform(self) -> float:
        """Float in [0, 1) from the high 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def choice(self, seq):
        return seq[self.randint(0, len(seq) - 1)]


_CHUNK = 1 << 16


def _outputs(seed: int, n: int, offset: int, finish, dtype) -> np.ndarray:
    """Outputs offset..offset+n-1, chunk by chunk (in place, cache-sized), each chunk passed
    through ``finish(z_uint64, out_chunk)``."""
    out = np.empty(n, dtype=dtype)
    z = np.empty(min(max(n, 1), _CHUNK), dtype=np.uint64)
    t = np.empty_like(z)
    g, m1, m2 = np.uint64(GAMMA), np.uint64(M1), np.uint64(M2)
    base = np.uint64(seed & MASK64)
    with np.errstate(over="ignore"):
        for c0 in range(0, n, _CHUNK):
            c1 = min(n, c0 + _CHUNK)
            zc, tc = z[: c1 - c0], t[: c1 - c0]
            zc[:] = np.arange(offset + c0 + 1, offset + c1 + 1, dtype=np.uint64)
            np.multiply(zc, g, out=zc)
            np.add(zc, base, out=zc)                           # seed + (i + 1) * GAMMA
            np.right_shift(zc, np.uint64(30), out=tc)
            np.bitwise_xor(zc, tc, out=zc)
            np.multiply(zc, m1, out=zc)
            np.right_shift(zc, np.uint64(27), out=tc)
            np.bitwise_xor(zc, tc, out=zc)
            np.multiply(zc, m2, out=zc)
            np.right_shift(zc, np.uint64(31), out=tc)
            np.bitwise_xor(zc, tc, out=zc)
            finish(zc, out[c0:c1])
    return out


def stream(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+n-1 of the stream seeded with ``seed`` (uint64 array)."""
    def keep(z, o):
        o[:] = z
    return _outputs(seed, n, offset, keep, np.uint64)


def uniform_mod(seed: int, n: int, modulus: int, offset: int = 0) -> np.ndarray:
    """int32 values ``(x >> 32) % modulus`` for the first n outputs."""
    m = np.uint64(modulus)

    def finish(z, o):
        np.right_shift(z, np.uint64(32), out=z)
        np.remainder(z, m, out=z)
        o[:] = z
    return _outputs(seed, n, offset, finish, np.int32)


def uniform_range(seed: int, n: int, lo: int, hi: int, offset: int = 0) -> np.ndarray:
    """int32 values uniform in [lo, hi] (inclusive)."""
    return (uniform_mod(seed, n, hi - lo + 1, offset).astype(np.int64) + lo).astype(np.int32)


def uniform_i32(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Full-range int32 values (high 32 bits reinterpreted)."""
    def finish(z, o):
        np.right_shift(z, np.uint64(32), out=z)
        o.view(np.uint32)[:] = z
    return _outputs(seed, n, offset, finish, np.int32)


def derive(seed: int, index: int) -> int:
    """Seed of the index-th independent sub-stream of ``seed`` (one program of a batch)."""
    return _mix(((seed & 0xFFFFFFFF) << 32 | (index & 0xFFFFFFFF)) & MASK64)
