"""Plain profiler arithmetic of the cf4ocl profiler module (Section 3.3) and
the profiling summary it prints for the PRNG example (Section 4.1, figure
"Possible profiling summary").

TEST INFRASTRUCTURE ONLY (see the package docstring).

An event is ``(queue, name, start, end)`` in seconds.  From a list of events:

* aggregate time of a name = sum of the durations of its events; its
  relative time = aggregate / total, total = sum of all durations;
* overlap of two events on *different* queues = length of the intersection
  of their intervals (events on one in-order queue never overlap, Section
  3.3); overlaps are summed per ordered name pair (name of the event that
  starts later, name of the event already running) -- the paper does not fix
  the order of the pair, this is the reading used throughout;
* effective event time = total - sum of all overlaps;
* device share = effective / elapsed wall time, host share = 1 - device.

Every pair of events is compared directly (quadratic), which is slow but
leaves nothing to check beyond the definitions above.
"""
from __future__ import annotations

from collections import defaultdict
from dataclasses import dataclass
from typing import Dict, Iterable, List, Tuple


@dataclass(frozen=True)
class Event:
    queue: str
    name: str
    start: float
    end: float

    @property
    def duration(self) -> float:
        return self.end - self.start


@dataclass
class Analysis:
    aggregate: Dict[str, float]          # name -> absolute time
    relative: Dict[str, float]           # name -> percent of total
    total: float
    overlaps: Dict[Tuple[str, str], float]
    overlap_total: float
    effective: float
    elapsed: float
    device_pct: float
    host_pct: float


def analyse(events: Iterable[Event], elapsed: float) -> Analysis:
    evs: List[Event] = list(events)
    agg: Dict[str, float] = defaultdict(float)
    for e in evs:
        agg[e.name] += e.duration
    total = sum(agg.values())
    rel = {k: (100.0 * v / total if total > 0 else 0.0) for k, v in agg.items()}
    ovl: Dict[Tuple[str, str], float] = defaultdict(float)
    for a in range(len(evs)):
        for b in range(a + 1, len(evs)):
            ea, eb = evs[a], evs[b]
            if ea.queue == eb.queue:
                continue
            length = min(ea.end, eb.end) - max(ea.start, eb.start)
            if length <= 0:
                continue
            later, earlier = (ea, eb) if (ea.start, a) > (eb.start, b) else (eb, ea)
            ovl[(later.name, earlier.name)] += length
    ovl_total = sum(ovl.values())
    eff = total - ovl_total
    dev = 100.0 * eff / elapsed if elapsed > 0 else 0.0
    return Analysis(dict(agg), rel, total, dict(ovl), ovl_total, eff, elapsed, dev, 100.0 - dev)
