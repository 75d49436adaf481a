"""Served form: continuous batching of generation requests.

``Server`` wraps the native scheduler of ``include/rng.h`` (admission against
a device-memory budget, steps over all admitted requests, states resident on
the device between steps).  ``run_load`` drives it with timed arrivals and
reports latency percentiles and throughput.
"""
from __future__ import annotations

import ctypes
import gc
import threading
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np
import torch

from . import _capi as C


class Server:
    def __init__(self, *, hbm_budget_bytes: int = 64 << 30, max_active: int = 1024,
                 step_bytes: int = 2 << 30, max_steps_in_flight: int = 2, values_per_thread: int = 4,
                 max_units_per_step: int = 1 << 20, mode: int = 1, stream=None,
                 device: Optional[int] = None):
        lib = C.load()
        o = C.RngServerOpts()
        lib.rng_server_opts_default(ctypes.byref(o))
        o.hbm_budget_bytes = hbm_budget_bytes
        o.max_active = max_active
        o.step_bytes = step_bytes
        o.max_steps_in_flight = max_steps_in_flight
        o.values_per_thread = values_per_thread
        o.max_units_per_step = max_units_per_step
        o.mode = mode
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        if stream is None:
            stream = torch.cuda.Stream(device=self.device)
        self._torch_stream = stream
        o.stream = stream.cuda_stream if isinstance(stream, torch.cuda.Stream) else int(stream)
        o.device = -1 if device is None else device
        self._lib = lib
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            C.check(lib.rng_server_create, ctypes.byref(o), ctypes.byref(self._h))

    def submit(self, seed: int, streams: int, iterations: int) -> int:
        t = ctypes.c_uint64()
        C.check(self._lib.rng_server_submit, self._h, seed & ((1 << 64) - 1), streams, iterations,
                ctypes.byref(t))
        return t.value

    def submit_ex(self, seed: int, streams: int, iterations: int, *, keep_state: bool = False,
                  continue_ticket: int = 0) -> int:
        """Submit with state retention and/or as the continuation of a kept request."""
        t = ctypes.c_uint64()
        C.check(self._lib.rng_server_submit_ex, self._h, seed & ((1 << 64) - 1), streams, iterations,
                1 if keep_state else 0, continue_ticket, ctypes.byref(t))
        return t.value

    def poll(self, max_items: int = 256, timeout_ms: int = 50):
        """Completed requests: list of (ticket, device address, latency seconds)."""
        tk = (ctypes.c_uint64 * max_items)()
        outs = (ctypes.c_void_p * max_items)()
        lat = (ctypes.c_double * max_items)()
        n = ctypes.c_uint32()
        C.check(self._lib.rng_server_poll, self._h, max_items, tk, outs, lat, ctypes.byref(n), timeout_ms)
        return [(tk[i], outs[i], lat[i]) for i in range(n.value)]

    def read(self, ticket: int, first: int, count: int) -> np.ndarray:
        buf = np.empty(count, dtype=np.uint64)
        C.check(self._lib.rng_server_read, self._h, ticket, first, count, ctypes.c_void_p(buf.ctypes.data))
        return buf

    def release(self, ticket: int):
        C.check(self._lib.rng_server_release, self._h, ticket)

    def stats(self) -> Dict[str, int]:
        st = C.RngServerStats()
        self._lib.rng_server_get_stats(self._h, ctypes.byref(st))
        return {name: getattr(st, name) for name, _ in C.RngServerStats._fields_}

    def close(self):
        if self._h:
            self._lib.rng_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


@dataclass
class LoadResult:
    latencies_s: Dict[int, float] = field(default_factory=dict)   # request index -> latency
    wall_s: float = 0.0
    bytes: int = 0
    submit_lag_s: float = 0.0  # worst lateness of a submission behind its arrival time

    def percentile(self, q: float) -> float:
        return float(np.percentile(np.array(list(self.latencies_s.values())), q))


def run_load(server: Server, requests: Sequence, *, time_scale: float = 1.0,
             on_complete: Optional[Callable[[int, int, int], None]] = None,
             timeout_s: float = 600.0) -> LoadResult:
    """Submits ``requests`` (objects with arrival_s, streams, iterations, seed)
    at their arrival times and waits for all of them.  ``on_complete(index,
    ticket, device_address)`` runs before each output is released."""
    res = LoadResult()
    ticket_to_idx: Dict[int, int] = {}
    lock = threading.Lock()
    remaining = [len(requests)]
    errors: List[BaseException] = []

    def collector():
        try:
            while True:
                with lock:
                    if remaining[0] == 0:
                        return
                for t, addr, lat in server.poll(512, 20):
                    with lock:
                        idx = ticket_to_idx.get(t)
                    while idx is None:  # submitted but not yet recorded by the submitter
                        time.sleep(0)
                        with lock:
                            idx = ticket_to_idx.get(t)
                    if on_complete is not None:
                        on_complete(idx, t, addr)
                    server.release(t)
                    with lock:
                        res.latencies_s[idx] = lat
                        remaining[0] -= 1
        except BaseException as e:  # surface in the caller
            errors.append(e)

    th = threading.Thread(target=collector, daemon=True)
    gc_was_enabled = gc.isenabled()
    gc.disable()  # a collection pause would delay submissions behind their arrival times
    t0 = time.perf_counter()
    th.start()
    for i, r in enumerate(requests):
        target = t0 + r.arrival_s * time_scale
        while True:
            now = time.perf_counter()
            if now >= target:
                break
            if target - now > 0.0005:
                time.sleep(target - now - 0.0003)
        res.submit_lag_s = max(res.submit_lag_s, time.perf_counter() - target)
        t = server.submit(r.seed, r.streams, r.iterations)
        with lock:
            ticket_to_idx[t] = i
        res.bytes += 8 * r.streams * r.iterations
        if errors:
            break
    th.join(timeout_s)
    res.wall_s = time.perf_counter() - t0
    if gc_was_enabled:
        gc.enable()
    if errors:
        raise errors[0]
    if th.is_alive():
        raise TimeoutError(f"{remaining[0]} requests still outstanding after {timeout_s} s")
    return res
