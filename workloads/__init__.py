"""Seeded synthetic workloads shaped like the paper's PRNG runs.

Shared by the tests, the benchmark and (for sizes only) the oracle side.  It
draws *parameters* -- stream counts, iteration counts, run seeds, arrival
times -- and holds none of the generator's own arithmetic (no hash, no
xorshift, no seed key).  Its splitmix64 is the draw rule the workload
definitions name for their parameter sequences; the library and the oracle
each carry their own code for the generator.

Draw rules:
* ``SplitMix64(start)``: state starts at ``start``; each draw adds the golden
  gamma 0x9e3779b97f4a7c15 and returns the finalised state (Steele, Lea and
  Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014).
* uniform double ``u = (draw >> 11) * 2^-53`` in [0, 1).
* log-uniform integer in [lo, hi]: ``floor(2^(log2 lo + u (log2 hi - log2 lo)))``
  clamped to [lo, hi].
* exponential gap with rate lam: ``-ln(1 - u) / lam``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List

_M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
GIB = 1 << 30


class SplitMix64:
    def __init__(self, start: int):
        self.state = start & _M64

    def next(self) -> int:
        self.state = (self.state + GAMMA) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next() >> 11) * (1.0 / (1 << 53))

    def log_uniform_int(self, lo: int, hi: int) -> int:
        u = self.uniform()
        v = math.floor(2.0 ** (math.log2(lo) + u * (math.log2(hi) - math.log2(lo))))
        return min(max(v, lo), hi)

    def exponential(self, rate: float) -> float:
        return -math.log1p(-self.uniform()) / rate


# --------------------------------------------------------------------------
# The plain method: 2^16 streams x 100 iterations, seed 0, device-resident.
# --------------------------------------------------------------------------
PLAIN = dict(streams=1 << 16, iterations=100, seed=0)

# Paper-shaped streaming run: 2^22 streams x 1024 iterations, seed 12345,
# through two 32 MiB device buffers into host memory (32 GiB in total).
STREAMING = dict(streams=1 << 22, iterations=1024, seed=12345, device_buffer_bytes=32 << 20)


@dataclass(frozen=True)
class Instance:
    streams: int
    iterations: int
    seed: int

    @property
    def nbytes(self) -> int:
        return 8 * self.streams * self.iterations


def batched_instances(count: int = 512, seed_start: int = 7, size_start: int = 1007,
                      streams_lo: int = 1 << 8, streams_hi: int = 1 << 20,
                      iters_lo: int = 1, iters_hi: int = 4096,
                      cap_bytes: int = 8 * GIB) -> List[Instance]:
    """Independent generator instances of uneven sizes.

    Seeds come from ``SplitMix64(seed_start)``; stream and iteration counts
    (log-uniform, streams drawn before iterations for each instance) from
    ``SplitMix64(size_start)``.  If the total output exceeds ``cap_bytes``,
    every iteration count is scaled by cap/total (floor, at least 1), then
    the largest instance (lowest index on ties) loses one iteration at a time
    until the cap holds.
    """
    seeds = SplitMix64(seed_start)
    sizes = SplitMix64(size_start)
    raw = []
    for _ in range(count):
        s = seeds.next()
        n = sizes.log_uniform_int(streams_lo, streams_hi)
        t = sizes.log_uniform_int(iters_lo, iters_hi)
        raw.append([n, t, s])
    total = sum(8 * n * t for n, t, _ in raw)
    if total > cap_bytes:
        scale = cap_bytes / total
        for r in raw:
            r[1] = max(1, math.floor(r[1] * scale))
        total = sum(8 * n * t for n, t, _ in raw)
        while total > cap_bytes:
            k = max(range(len(raw)), key=lambda j: (8 * raw[j][0] * raw[j][1], -j))
            if raw[k][1] <= 1:
                break
            raw[k][1] -= 1
            total -= 8 * raw[k][0]
    return [Instance(n, t, s) for n, t, s in raw]


@dataclass(frozen=True)
class Request:
    arrival_s: float
    streams: int
    iterations: int
    seed: int

    @property
    def nbytes(self) -> int:
        return 8 * self.streams * self.iterations


def served_requests(rate_per_s: float = 2000.0, duration_s: float = 60.0,
                    seed_start: int = 99, arrival_start: int = 1099, size_start: int = 2099,
                    streams_lo: int = 1 << 10, streams_hi: int = 1 << 22,
                    iters_lo: int = 1, iters_hi: int = 512) -> List[Request]:
    """Poisson arrivals at ``rate_per_s`` over ``duration_s`` seconds.

    Gaps come from ``SplitMix64(arrival_start)``, run seeds from
    ``SplitMix64(seed_start)``, sizes (streams then iterations, log-uniform)
    from ``SplitMix64(size_start)``.
    """
    arr = SplitMix64(arrival_start)
    seeds = SplitMix64(seed_start)
    sizes = SplitMix64(size_start)
    out: List[Request] = []
    t = 0.0
    while True:
        t += arr.exponential(rate_per_s)
        if t >= duration_s:
            break
        n = sizes.log_uniform_int(streams_lo, streams_hi)
        it = sizes.log_uniform_int(iters_lo, iters_hi)
        out.append(Request(t, n, it, seeds.next()))
    return out


def sweep_points(streams_exps=(16, 18, 20, 22, 24, 26, 28), vpts=(1, 2, 4, 8, 16, 32, 64),
                 min_bytes: int = 16 * GIB):
    """Roofline sweep: (streams, values per thread, iterations) with enough
    iterations that each point writes at least ``min_bytes``."""
    pts = []
    for e in streams_exps:
        n = 1 << e
        t = max(1, -(-min_bytes // (8 * n)))
        for v in vpts:
            pts.append((n, v, t))
    return pts
