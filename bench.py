"""Benchmark of the massive PRNG hot path on GB300.

Workload (default): the paper-shaped streaming run -- 2^22 streams x 1024
iterations, seed 12345, uint64 output in the iteration-major layout (32 GiB
per step).  One step = rng_init + rng_generate over the whole workload.

* ``value``: device-resident generation, GB/s of uint64 output (8 bytes per
  value), the output written into a 32 GiB device buffer (larger than L2, so
  no flush is needed between steps), timed with CUDA events on the
  generator's compute stream.
* ``e2e``: the same step through the C ABI with a host output buffer (32 GiB
  of page-locked memory from rng_host_alloc, backed by transparent huge
  pages): by default the kernel stores straight into it over the host link;
  ``e2e.double_buffer`` times the paper's double buffer (two 32 MiB device
  buffers, copy-engine reads on a copy stream while the next buffer is
  generated).  Every timed region includes every device-to-host byte.
* ``roofline``: the row kernel's average launch time from the library's own
  CUDA events (recorded on the stream it launches on) over the timed region.
* ``cpu_baseline``: the CPU oracle timed on a bounded sample on rank 0.
* ``plain``, ``batched``, ``checksum``, ``sweep``, ``served`` (one GPU): the
  other workloads -- the plain method (2^16 x 100), the batched form (512
  instances, 8 GiB, one CUDA-graph launch) against the plain form, the
  generate-and-checksum mode against its integer-ALU roofline, a compact
  roofline sweep over stream counts, and the served form (Poisson 2000
  req/s for ``--duration`` seconds, p50/p99 latency) -- each with its own
  config and the clocks sampled during its own timed region.

``--impl reference`` times the CPU oracle instead (the method's plain
definition, single-threaded) on a bounded sample of the same workload.
Under torchrun every rank generates its own block of 2^22 stream ids (weak
scaling, no data exchange); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
GIB = 1 << 30

WORKLOADS = {
    "streaming": dict(streams=1 << 22, iterations=1024, seed=12345, device_buffer_bytes=32 << 20,
                      name="paper-shaped streaming run: 2^22 streams x 1024 iterations, seed 12345"),
    "plain": dict(streams=1 << 16, iterations=100, seed=0, device_buffer_bytes=32 << 20,
                  name="plain method: 2^16 streams x 100 iterations, seed 0"),
}

# ALU-pipe lane operations per value of checksum_kernel<16> in output modes
# 0 and 1, from their ncu captures: ALU-pipe utilisation (85.5 %, 74.9 %) x 64
# lanes x 152 SMs x 1.85 GHz x duration (184.2 us, 209.7 us) over 2^22 x 64
# values.
CHECKSUM_ALU_OPS_PER_VALUE = {0: 10.6, 1: 10.5}
NOMINAL_HBM_GBPS = 7900.0  # GB300 HBM3e, nominal
METRIC = "GB/s of uint64 PRNG output (device and host-streamed) vs roofline; p50/p99 req latency"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return rank, ws


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in ("kernels.cu", "prng_math.cuh", "internal.h"):
        with open(os.path.join(ROOT, "paper_1609_01257_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


PROFILES_DIR = os.path.join(ROOT, "profiles")

# What the row-kernel launch ran (Generator.last_launch()["kernel"]).
KERNEL_LABEL = {"register": "register stores (each thread stores its values)",
                "staged": "rows staged in shared memory, stored as line-aligned 16-byte pieces",
                "bulk": "rows staged in shared memory ({nb} buffers), written by TMA bulk copies (cp.async.bulk)"}
KERNEL_FN = {"register": "rows_kernel", "staged": "rows_staged_kernel", "bulk": "rows_bulk_kernel"}
STORE_POLICY_LABEL = {0: "default stores", 1: "streaming stores (st.global.cs); bulk copies where measured faster",
                      2: "bulk copies for every device row"}


def _traffic_per_launch(workload: str, kernel: str = "rows_kernel"):
    """DRAM bytes per launch of `kernel` from its committed ncu summary
    (profiles/<kernel>_traffic.md), when it was taken on the current kernel
    source; else None."""
    try:
        txt = open(os.path.join(PROFILES_DIR, f"{kernel}_traffic.md")).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    m = re.search(rf"traffic_bytes_per_launch\[{workload}\]:\s*([0-9.eE+]+)", txt)
    if not m or not m_hash or m_hash.group(1) != _kernel_source_hash():
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every `interval_ms` from
    before the warm-up until after the timed region; each line is stamped
    with the host time it arrived, so the samples that fall inside the timed
    region can be told apart."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 20):
        self.gpu = gpu_index
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []
        self.reader = None

    def start(self, wait_s: float = 3.0):
        """Starts sampling and waits (up to wait_s) for the first sample."""
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.interval_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                bufsize=1)
        except OSError:
            self.proc = None
            return

        def read():
            for line in self.proc.stdout:
                self.lines.append((time.time(), line))

        self.reader = threading.Thread(target=read, daemon=True)
        self.reader.start()
        end = time.time() + wait_s
        while not self.lines and time.time() < end:
            time.sleep(0.01)

    def window(self, t0: float, t1: float):
        """Median clock etc. of the samples stamped within [t0, t1], while
        sampling goes on (the samples nearest to a region shorter than the
        sampling interval)."""
        if not self.proc:
            return None
        time.sleep(2 * self.interval_ms / 1e3)  # let the sample after t1 arrive
        res = clocks_in_window(list(self.lines), t0, t1, margin_s=2 * self.interval_ms / 1e3)
        if res is not None:
            res["interval_ms"] = self.interval_ms
        return res

    def stop(self, t0: float | None = None, t1: float | None = None):
        """Median clock etc. of the samples stamped within [t0, t1] (host
        time around the timed region); if the region was shorter than the
        sampling interval, of every sample taken since start()."""
        if not self.proc:
            return None
        time.sleep(2 * self.interval_ms / 1e3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        if self.reader:
            self.reader.join(timeout=5)
        res = clocks_in_window(list(self.lines), t0, t1)
        if res is not None:
            res["interval_ms"] = self.interval_ms
        return res


def clocks_in_window(lines, t0, t1, margin_s: float | None = None):
    """parse_clock_samples over the (host time, line) samples stamped within
    [t0, t1].  When none is (a timed region shorter than the sampling
    interval): over those within `margin_s` of it if given, else over all."""
    res, window = None, "timed region"
    if t0 is not None and t1 is not None:
        res = parse_clock_samples("".join(l for ts, l in lines if t0 <= ts <= t1))
        if res is None and margin_s is not None:
            res = parse_clock_samples("".join(l for ts, l in lines if t0 - margin_s <= ts <= t1 + margin_s))
            window = (f"samples within {1e3 * margin_s:.0f} ms of the timed region "
                      "(shorter than the sampling interval)")
    if res is None:
        res = parse_clock_samples("".join(l for _, l in lines))
        window = "warm-up and timed region (the timed region is shorter than the sampling interval)"
    if res is not None:
        res["window"] = window
    return res


def parse_clock_samples(text: str):
    """Median SM clock, max clock and the throttle reasons seen, from
    `nvidia-smi --query-gpu=<ClockSampler.FIELDS> --format=csv,noheader,nounits`
    lines; None when no sample parses."""
    sms, maxes, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in text.strip().splitlines():
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sms.append(float(parts[1]))
            maxes.append(float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sms:
        return None
    return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxes), "reasons": sorted(reasons),
            "samples": len(sms)}


def cpu_oracle_sample(streams: int, seed: int, iterations: int, output_mode: int = 0):
    """Times the CPU oracle (single thread) on `iterations` rows of the workload."""
    sys.path.insert(0, ROOT)
    import oracle  # test infrastructure: the CPU baseline leg only
    oracle.build()
    t0 = time.perf_counter()
    out = oracle.generate(streams, seed, iterations, output_mode=output_mode)
    dt = time.perf_counter() - t0
    return out.nbytes, dt


def _oracle_worker_init():
    sys.path.insert(0, ROOT)
    import oracle  # test infrastructure: the CPU baseline leg only
    oracle.lib()


def _oracle_worker(job):
    import oracle
    n_sub, g0, seed, rows, mode = job
    return oracle.generate(n_sub, seed, rows, g0=g0, output_mode=mode).nbytes


def cpu_oracle_all_cores(streams: int, seed: int, iterations: int, reps: int = 3, output_mode: int = 0):
    """The same oracle, unchanged, run as one process per host core, each on a
    contiguous block of stream ids (the values of the whole workload, in
    column blocks).  Returns (bytes, median seconds of `reps` runs, processes)."""
    import multiprocessing as mp
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    per = (streams + cores - 1) // cores
    jobs = [(min(per, streams - g0), g0, seed, iterations, output_mode) for g0 in range(0, streams, per)]
    # spawn: this process already holds a CUDA context
    times = []
    with mp.get_context("spawn").Pool(len(jobs), initializer=_oracle_worker_init) as pool:
        pool.map(_oracle_worker, [(1, 0, seed, 1, output_mode)] * len(jobs), chunksize=1)
        for _ in range(reps):
            t0 = time.perf_counter()
            nbytes = sum(pool.map(_oracle_worker, jobs, chunksize=1))
            times.append(time.perf_counter() - t0)
    return nbytes, statistics.median(times), len(jobs)


def run_reference(args, wl):
    rank, ws = _dist()
    if rank != 0:
        return 0
    # Bounded sample per step: all streams, first `rows` iterations.
    rows = args.reference_rows
    times, nbytes = [], 0
    for _ in range(args.warmup):
        cpu_oracle_sample(wl["streams"], wl["seed"], rows, args.output_mode)
    for _ in range(args.steps):
        nbytes, dt = cpu_oracle_sample(wl["streams"], wl["seed"], rows, args.output_mode)
        times.append(dt)
    total = sum(times)
    gbs = nbytes * len(times) / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": wl["name"] + _mode_label(args), "streams": wl["streams"],
                   "iterations": wl["iterations"], "seed": wl["seed"], "output_mode": args.output_mode,
                   "parallelism": "none (host cores)"},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"{wl['streams']} streams x first {rows} iterations per step"},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_gpu(args, wl):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import paper_1609_01257_gb300 as rng

    rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x: float) -> float:
        if ws == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    n, T, seed = wl["streams"], wl["iterations"], wl["seed"]
    nbytes = 8 * n * T
    gen = rng.Generator(n, seed, output_mode=args.output_mode, stream_offset=rank * n, device_buffer_bytes=wl["device_buffer_bytes"],
                        values_per_thread=args.values_per_thread, block_threads=args.block_threads,
                        store_width=args.store_width, grid_blocks=args.grid_blocks, store_policy=args.store_policy,
                        init=False)
    stream = gen.stream
    out = torch.empty((T, n), dtype=torch.uint64, device="cuda")
    torch.cuda.synchronize()

    def step_device():
        gen.init()
        gen.generate_to(T, out.data_ptr())

    # ---- device-resident leg ------------------------------------------------
    if L2Flush.needed(torch, nbytes):
        flush = L2Flush(torch)
        l2_note = flush.label()
    else:
        flush = None
        l2_note = (f"output {nbytes / GIB:g} GiB per step > 4 x {L2Flush.l2_size(torch) / 1e6:.0f} MB L2: "
                   "no flush needed")
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        if flush:
            flush(stream)
        step_device()
    gen.sync()
    barrier()
    gen.profile_reset()
    launches0 = rng.launch_count()
    t_start = time.time()
    dev_s = timed_steps(torch, stream, step_device, args.steps, flush)
    t_end = time.time()
    barrier()
    clk = clocks.window(t_start, t_end)
    launches = rng.launch_count() - launches0
    del flush
    dev_s = max_over_ranks(dev_s)
    k_count, k_total = gen.profile_stat("RNG_KERNEL")
    k_avg = max_over_ranks(k_total / max(k_count, 1))
    value = nbytes * ws * args.steps / dev_s / 1e9
    ran = gen.last_launch()
    vpt, block, grid = ran["values_per_thread"], ran["block"], ran["grid"]
    del out
    torch.cuda.empty_cache()
    # Denominators measured on this GPU, outside the timed regions.
    write_ceiling = measure_write_ceiling(torch)
    link = measure_host_link(torch) if not args.skip_e2e else None

    # ---- end-to-end leg: host output through the C ABI ------------------------
    e2e = None
    if not args.skip_e2e:
        # One rank holds the whole step's output in page-locked memory; with
        # several ranks on one node each streams its step through a smaller
        # page-locked buffer (calls of `rows` iterations), so the ranks'
        # buffers together stay well inside host memory.  Same bytes over
        # the link either way.
        rows = T if ws == 1 else max(1, min(T, (2 * GIB) // (8 * n)))
        # Page-locked destination from the library's allocator (transparent
        # huge pages): into 64 KiB pages the copies over the host link stall
        # intermittently (`--workload host-dest`).
        host = rng.host_empty((rows, n))
        dest = {"allocator": "rng_host_alloc (anonymous memory, transparent huge pages, cudaHostRegister)",
                "bytes": host.nbytes, "huge_page_share": huge_page_share(host)}

        def host_leg(g, steps):
            def step_host():
                g.init()
                for _ in range(T // rows):
                    g.generate_to_host(rows, host)
                if T % rows:
                    g.generate_to_host(T % rows, host)

            for _ in range(max(1, min(args.warmup, 2))):
                step_host()
            barrier()
            g.profile_reset()
            t0 = time.perf_counter()
            marks = [t0]
            for _ in range(steps):
                step_host()
                marks.append(time.perf_counter())
            barrier()
            step_ms.append([round(1e3 * (b - a), 1) for a, b in zip(marks, marks[1:])])
            return max_over_ranks(time.perf_counter() - t0), g.profile()

        step_ms = []  # per-step host times of each leg, in the order the legs run

        # Default host path: the kernel stores straight into the page-locked
        # buffer over the host link.
        host_s, _ = host_leg(gen, args.e2e_steps)
        e2e = {"value": nbytes * ws * args.e2e_steps / host_s / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": 0, "d2h_bytes_per_step": nbytes,
               "steps": args.e2e_steps, "ms_per_step": 1e3 * host_s / args.e2e_steps,
               "path": "direct stores into page-locked host memory",
               "iterations_per_call": rows, "destination": dest, "step_ms": step_ms[0]}
        # The paper's double buffer: two device buffers, copy engine reads.
        # Timed without the event profiler; one more profiled step gives the
        # kernel/read/overlap split.
        gdb = rng.Generator(n, seed, output_mode=args.output_mode, stream_offset=rank * n, device_buffer_bytes=wl["device_buffer_bytes"],
                            host_path=1, profiling=False, init=False)
        db_s, _ = host_leg(gdb, args.e2e_steps)
        gdb.close()
        gdb = rng.Generator(n, seed, output_mode=args.output_mode, stream_offset=rank * n, device_buffer_bytes=wl["device_buffer_bytes"],
                            host_path=1, init=False)
        _, prof = host_leg(gdb, 1)
        gdb.close()
        e2e["double_buffer"] = {
            "value": nbytes * ws * args.e2e_steps / db_s / 1e9, "unit": "GB/s",
            "ms_per_step": 1e3 * db_s / args.e2e_steps, "step_ms": step_ms[1],
            "profiled_step": {"read_buffer_s": prof["aggregate"].get("READ_BUFFER", (0, 0))[0],
                              "rng_kernel_s": prof["aggregate"].get("RNG_KERNEL", (0, 0))[0],
                              "overlap_s": sum(prof["overlaps"].values())}}
        # The same double buffer with its reads done by a copy kernel.
        gsm = rng.Generator(n, seed, output_mode=args.output_mode, stream_offset=rank * n, device_buffer_bytes=wl["device_buffer_bytes"],
                            host_path=3, profiling=False, init=False)
        sm_s, _ = host_leg(gsm, args.e2e_steps)
        gsm.close()
        e2e["double_buffer_copy_kernel"] = {"value": nbytes * ws * args.e2e_steps / sm_s / 1e9, "unit": "GB/s",
                                            "ms_per_step": 1e3 * sm_s / args.e2e_steps, "step_ms": step_ms[-1]}
        e2e["host_link_GBps"] = link
        e2e["frac_link"] = e2e["value"] / link
        del host

        # Host consumer (Section 5, "out" block): consumer threads fold every
        # row into its XOR and sum as it arrives through the staging slots.
        gh = rng.Generator(n, seed, output_mode=args.output_mode, stream_offset=rank * n, device_buffer_bytes=wl["device_buffer_bytes"],
                           profiling=False, init=False)

        def step_host_checksum():
            gh.init()
            gh.generate_host_checksum(T)

        for _ in range(max(1, min(args.warmup, 2))):
            step_host_checksum()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            step_host_checksum()
        barrier()
        hc_s = max_over_ranks(time.perf_counter() - t0)
        hc_stats = gh.host_stats()
        gh.close()
        e2e["host_checksum"] = {"value": nbytes * ws * args.e2e_steps / hc_s / 1e9, "unit": "GB/s",
                                "ms_per_step": 1e3 * hc_s / args.e2e_steps,
                                "consumers": "default (host cores but one, 1-16)",
                                "host_cores": os.cpu_count(), "last_step": hc_stats}

        # The paper's program as measured there: every value to stdout, here
        # /dev/null, through the staging slots and one writer thread.
        gf = rng.Generator(n, seed, output_mode=args.output_mode, stream_offset=rank * n, device_buffer_bytes=wl["device_buffer_bytes"],
                           profiling=False, init=False)
        fd = os.open(os.devnull, os.O_WRONLY)

        def step_fd():
            gf.init()
            gf.generate_fd(T, fd)

        for _ in range(max(1, min(args.warmup, 2))):
            step_fd()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            step_fd()
        barrier()
        fd_s = max_over_ranks(time.perf_counter() - t0)
        fd_stats = gf.host_stats()
        os.close(fd)
        gf.close()
        e2e["stdout_devnull"] = {"value": nbytes * ws * args.e2e_steps / fd_s / 1e9, "unit": "GB/s",
                                 "ms_per_step": 1e3 * fd_s / args.e2e_steps, "last_step": fd_stats}

    gen.close()
    peaks, src = _peaks()
    # The other workloads (the plain method, batched and served forms,
    # generate-and-checksum mode, the roofline sweep), each timed in its own
    # window with its own clock summary; one GPU only.
    extra = {}
    if ws == 1 and not args.skip_configs:
        extra["plain"] = plain_leg(args, clocks, write_ceiling, peaks["hbm_gbs"])
        extra["batched"] = batched_leg(args, clocks, write_ceiling)
        extra["checksum"] = checksum_leg(args, WORKLOADS["streaming"], clocks)
        extra["sweep"] = sweep_leg(args, clocks)
        extra["served"] = served_leg(args, clocks)
    clocks.stop()
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0

    achieved = nbytes / k_avg / 1e9
    traffic = _traffic_per_launch(args.workload, KERNEL_FN[ran["kernel"]])
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "values_per_s": value * 1e9 / 8, "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": wl["name"] + _mode_label(args), "streams_per_gpu": n, "iterations": T,
                   "seed": seed, "output_mode": args.output_mode,
                   "bytes_per_step_per_gpu": nbytes, "values_per_thread": vpt, "block": block, "grid": grid,
                   "stores": {"kernel": KERNEL_LABEL[ran["kernel"]].format(nb=ran["row_buffers"]),
                              "widest_values": args.store_width or "per shape",
                              "policy": STORE_POLICY_LABEL.get(args.store_policy, str(args.store_policy))},
                   "l2": l2_note,
                   "parallelism": f"dp{ws} (disjoint stream-id blocks)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "peak_source": f"{src}: hbm_gbs (copy, read+write) from MEASURED_PEAKS.json",
                     "kernel": KERNEL_FN[ran["kernel"]], "kernel_avg_ms": k_avg * 1e3, "launches": k_count,
                     "write_ceiling_GBps": write_ceiling, "frac_write_ceiling": achieved / write_ceiling,
                     "write_ceiling_source": "measured here: torch fill_ over 2 GiB, best of 10",
                     "nominal_GBps": NOMINAL_HBM_GBPS, "frac_nominal": achieved / NOMINAL_HBM_GBPS},
        "gpu_launches": launches,
        "e2e": e2e,
        "clocks": clk,
    }
    line.update(extra)
    if not args.skip_cpu_baseline and ws == 1:
        rows = args.cpu_rows or T
        nb, dt = cpu_oracle_sample(n, seed, rows, args.output_mode)
        line["cpu_baseline"] = {"value": nb / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
                                "sample": f"{n} streams x first {rows} iterations ({nb / GIB:.1f} GiB), "
                                          f"single-threaded C oracle, {dt:.1f} s"}
        nb_all, dt_all, procs = cpu_oracle_all_cores(n, seed, rows, output_mode=args.output_mode)
        line["cpu_baseline"]["all_cores"] = {
            "value": nb_all / dt_all / 1e9, "unit": "GB/s", "cores": procs,
            "sample": f"the same {nb_all / GIB:.1f} GiB as {procs} processes of the oracle on contiguous "
                      f"stream-id blocks, median of 3 runs, {dt_all:.2f} s"}
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


def huge_page_share(arr) -> float | None:
    """Share of the memory mapping holding `arr` that transparent huge pages
    back (AnonHugePages / Size in /proc/self/smaps); None when unreadable."""
    addr = arr.ctypes.data
    try:
        with open("/proc/self/smaps") as f:
            inside, size = False, None
            for line in f:
                head = line.split(None, 1)[0]
                if "-" in head and not head.endswith(":"):
                    a, b = (int(x, 16) for x in head.split("-"))
                    inside, size = a <= addr < b, b - a
                elif inside and head == "AnonHugePages:":
                    return int(line.split()[1]) * 1024 / size
    except (OSError, ValueError):
        pass
    return None


def measure_write_ceiling(torch, nbytes=2 * GIB, reps=10):
    """Write-only HBM ceiling on this GPU: best of `reps` `fill_` launches over
    `nbytes` (a plain store stream, no reads), timed with CUDA events."""
    buf = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    best = float("inf")
    for r in range(reps + 2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        buf.fill_(float(r))
        e1.record(s)
        e1.synchronize()
        if r >= 2:
            best = min(best, e0.elapsed_time(e1) * 1e-3)
    del buf
    return nbytes / best / 1e9


def measure_host_link(torch, nbytes=GIB, reps=10):
    """Device-to-host link rate: best of `reps` copy-engine copies of `nbytes`
    into page-locked memory (cudaMemcpyAsync), timed with CUDA events."""
    dev = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    host = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    s = torch.cuda.current_stream()
    best = float("inf")
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        host.copy_(dev, non_blocking=True)
        e1.record(s)
        e1.synchronize()
        if r >= 1:
            best = min(best, e0.elapsed_time(e1) * 1e-3)
    del dev, host
    return nbytes / best / 1e9


class L2Flush:
    """Evicts the output of the previous step from L2: writes a buffer of
    four times the L2 size on the given stream.  Used, outside the timed
    events, when one step writes less than that (the plain 52 MB workload;
    small jump-ahead states), so that each timed step starts from a cold L2."""

    def __init__(self, torch):
        self.l2_bytes = self.l2_size(torch)
        self.buf = torch.empty(4 * self.l2_bytes // 4, dtype=torch.int32, device="cuda")
        self.torch = torch
        self.n = 0

    @staticmethod
    def l2_size(torch) -> int:
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        return int(getattr(props, "L2_cache_size", 0)) or 129 * 10**6

    @staticmethod
    def needed(torch, step_bytes: int) -> bool:
        return step_bytes < 4 * L2Flush.l2_size(torch)

    def __call__(self, stream):
        self.n += 1
        with self.torch.cuda.stream(stream):
            self.buf.fill_(self.n)

    def label(self) -> str:
        return (f"L2 ({self.l2_bytes / 1e6:.0f} MB) flushed before every timed step by writing "
                f"{4 * self.l2_bytes / 1e6:.0f} MB outside the step's events; time = sum of the steps' events")


def timed_steps(torch, stream, step, steps: int, flush=None) -> float:
    """Seconds for `steps` calls of `step`, from CUDA events on `stream`.
    Without `flush`: one event pair around all steps.  With it: the flush
    runs before each step, outside that step's own event pair, and the
    result is the sum of the per-step times."""
    if flush is None:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3
    pairs = []
    for _ in range(steps):
        flush(stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        pairs.append((a, b))
    pairs[-1][1].synchronize()
    return sum(a.elapsed_time(b) for a, b in pairs) * 1e-3


def _mode_label(args) -> str:
    return ", xorshift64* output (mode 1)" if args.output_mode == 1 else ""


def _json_line(d):
    print(json.dumps(d), flush=True)


BATCHED_NAME = ("batched: 512 instances, streams log-uniform [2^8, 2^20], iterations log-uniform [1, 4096] "
                "capped at {cap:g} GiB, seeds splitmix64 from 7, one CUDA-graph launch")
SERVED_NAME = ("served: Poisson 2000 req/s for {dur:g} s, streams log-uniform [2^10, 2^22], iterations "
               "log-uniform [1, 512], seeds splitmix64 from 99, 64 GiB HBM budget, device outputs")


def batched_leg(args, clocks=None, write_ceiling=None):
    """Batched form: 512 independent instances (log-uniform sizes, 8 GiB total)
    in one CUDA-graph launch, against the plain form (one generator and one
    launch per instance) on the same GPU.  Output 8 GiB per step (> L2)."""
    import torch
    sys.path.insert(0, ROOT)
    import paper_1609_01257_gb300 as rng
    import workloads

    if args.batch_uniform:
        # A uniform batch instead of the drawn mix: `count` instances of
        # `streams` x `iterations`, seeds 0 .. count-1.
        n_u, t_u, k_u = args.batch_uniform
        inst = [workloads.Instance(streams=n_u, iterations=t_u, seed=k) for k in range(k_u)]
        name = f"batched: {k_u} instances of {n_u} streams x {t_u} iterations, seeds 0..{k_u - 1}, one CUDA-graph launch"
    else:
        inst = workloads.batched_instances(cap_bytes=int(args.batch_cap_gib * GIB))
        name = BATCHED_NAME.format(cap=args.batch_cap_gib)
    total = sum(i.nbytes for i in inst)
    b = rng.Batch([i.streams for i in inst], [i.iterations for i in inst], [i.seed for i in inst],
                  values_per_thread=args.batch_vpt, mode=args.batch_mode,
                  stores=args.batch_stores)
    cfg = b.config()
    s = b.stream
    for _ in range(args.warmup):
        b.run()
    b.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    e0.record(s)
    for _ in range(args.steps):
        b.run()
    e1.record(s)
    e1.synchronize()
    t1 = time.time()
    batched_s = e0.elapsed_time(e1) * 1e-3 / args.steps
    clk = clocks.window(t0, t1) if clocks else None
    # Plain form: one generator per instance, launched one after another.
    plain_stream = torch.cuda.Stream()
    gens = [rng.Generator(i.streams, i.seed, compute_stream=plain_stream, profiling=False, init=False)
            for i in inst]

    def plain_step():
        for g, o, i in zip(gens, b.outputs, inst):
            g.init()
            g.generate_to(i.iterations, o.data_ptr())

    for _ in range(args.warmup):
        plain_step()
    plain_stream.synchronize()
    e0.record(plain_stream)
    for _ in range(args.steps):
        plain_step()
    e1.record(plain_stream)
    e1.synchronize()
    plain_s = e0.elapsed_time(e1) * 1e-3 / args.steps
    for g in gens:
        g.close()
    b.close()
    d = {"config": {"workload": name, "instances": len(inst),
                    "bytes_per_step": total, "tuned": cfg,
                    "l2": f"output {total / GIB:.1f} GiB per step > L2: no flush needed"},
         "value": total / batched_s / 1e9, "unit": "GB/s", "ms_per_step": batched_s * 1e3,
         "plain_form_GBps": total / plain_s / 1e9, "plain_form_ms": plain_s * 1e3,
         "batched_over_plain_form": plain_s / batched_s, "steps": args.steps, "warmup": args.warmup}
    if write_ceiling:
        d["frac_write_ceiling"] = d["value"] / write_ceiling
    if clocks:
        d["clocks"] = clk
    return d


def run_batched(args):
    d = batched_leg(args)
    _json_line({"workload": d["config"]["workload"], "bytes_per_step": d["config"]["bytes_per_step"],
                "batched_GBps": d["value"], "batched_ms": d["ms_per_step"], "plain_GBps": d["plain_form_GBps"],
                "plain_ms": d["plain_form_ms"], "tuned": d["config"]["tuned"], "steps": args.steps,
                "warmup": args.warmup})
    return 0


def served_leg(args, clocks=None):
    """Served form: Poisson arrivals (2000/s) for `args.duration` seconds,
    continuous batching, 64 GiB budget; latency from submission to the
    output being complete on the device."""
    sys.path.insert(0, ROOT)
    import paper_1609_01257_gb300 as rng
    import workloads

    reqs = workloads.served_requests(duration_s=args.duration)
    offered = sum(r.nbytes for r in reqs)
    with rng.Server(hbm_budget_bytes=64 << 30, step_bytes=args.step_bytes,
                    max_steps_in_flight=args.steps_in_flight, values_per_thread=args.server_vpt,
                    mode=args.server_mode) as srv:
        warm = workloads.served_requests(duration_s=0.5, seed_start=5, arrival_start=6, size_start=7)
        rng.run_load(srv, warm)
        t0 = time.time()
        res = rng.run_load(srv, reqs)
        t1 = time.time()
        st = srv.stats()
    d = {"config": {"workload": SERVED_NAME.format(dur=args.duration), "window_s": args.duration,
                    "server": {"step_bytes": args.step_bytes, "steps_in_flight": args.steps_in_flight,
                               "values_per_thread": args.server_vpt, "mode": args.server_mode}},
         "requests": len(reqs), "p50_ms": res.percentile(50) * 1e3, "p99_ms": res.percentile(99) * 1e3,
         "max_ms": max(res.latencies_s.values()) * 1e3,
         "aggregate_GBps": res.bytes / res.wall_s / 1e9, "offered_GBps": offered / args.duration / 1e9,
         "wall_s": res.wall_s, "worst_submit_lag_ms": res.submit_lag_s * 1e3,
         "steps": st["steps"], "peak_active": st["peak_active"], "peak_bytes_in_use": st["peak_bytes_in_use"]}
    if clocks:
        d["clocks"] = clocks.window(t0, t1)
    return d


def run_served(args):
    d = served_leg(args)
    line = {"workload": d["config"]["workload"]}
    line.update({k: v for k, v in d.items() if k != "config"})
    line["server"] = d["config"]["server"]
    _json_line(line)
    return 0


def checksum_leg(args, wl, clocks=None):
    """Generate-and-checksum mode on the streaming workload: every value is
    produced and folded into its row's XOR and wrapping sum; nothing is
    stored.  Bound by integer issue on the ALU pipe, not memory."""
    import torch
    sys.path.insert(0, ROOT)
    import paper_1609_01257_gb300 as rng

    n, T, seed = wl["streams"], wl["iterations"], wl["seed"]
    g = rng.Generator(n, seed, output_mode=args.output_mode, init=False)
    rx = torch.empty(T, dtype=torch.uint64, device="cuda")
    rs = torch.empty(T, dtype=torch.uint64, device="cuda")
    torch.cuda.synchronize()

    def step():
        g.init()
        g.generate_checksum(T, rx, rs)

    own = clocks is None
    if own:
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
    for _ in range(args.warmup):
        step()
    g.sync()
    g.profile_reset()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s = g.stream
    t_start = time.time()
    e0.record(s)
    for _ in range(args.steps):
        step()
    e1.record(s)
    e1.synchronize()
    t_end = time.time()
    secs = e0.elapsed_time(e1) * 1e-3
    clk = clocks.stop(t_start, t_end) if own else clocks.window(t_start, t_end)
    c, t = g.profile_stat("CHECKSUM_KERNEL")
    g.close()
    props = torch.cuda.get_device_properties(0)
    vps = n * T * args.steps / secs
    # Integer-ALU roofline: the ALU pipe retires 64 lane-ops per SM per clock
    # (half a warp instruction per cycle per sub-partition); the ops per
    # value come from the kernel's ncu capture (ALU-pipe share x pipe peak x
    # duration / values).
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0  # nominal maximum when nvidia-smi gave no sample
    peak = props.multi_processor_count * 64 * sm_mhz * 1e6 / 1e12
    ops = CHECKSUM_ALU_OPS_PER_VALUE[args.output_mode]
    achieved = vps * ops / 1e12
    return {"config": {"workload": wl["name"] + " (generate-and-checksum mode)" + _mode_label(args),
                       "streams": n, "iterations": T, "seed": seed},
            "values_per_s": vps,
            "equiv_GBps": 8 * vps / 1e9, "kernel_avg_ms": 1e3 * t / max(c, 1), "steps": args.steps,
            "sms": props.multi_processor_count,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s (ALU-pipe lane ops)",
                         "frac": achieved / peak, "alu_ops_per_value": ops,
                         "peak_source": "SMs x 64 ALU-pipe lanes x median SM clock during the timed region"},
            "clocks": clk}


def run_checksum(args, wl):
    line = checksum_leg(args, wl)
    line = dict(line, workload=line["config"]["workload"])
    del line["config"]
    if not args.skip_cpu_baseline:
        sys.path.insert(0, ROOT)
        import oracle  # test infrastructure: the CPU baseline leg only
        oracle.build()
        n, T, seed = wl["streams"], wl["iterations"], wl["seed"]
        rows = min(T, args.cpu_rows or T)
        t0 = time.perf_counter()
        oracle.row_checksums(n, seed, rows, output_mode=args.output_mode)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": n * rows / dt, "unit": "values/s", "cores": 1, "kind": "oracle",
                                "sample": f"{n} streams x first {rows} iterations, row checksums, "
                                          f"single-threaded C oracle, {dt:.1f} s"}
    _json_line(line)
    return 0


def plain_leg(args, clocks=None, write_ceiling=None, peak=None):
    """The plain method (2^16 streams x 100 iterations, seed 0, 52 MB,
    device-resident): L2 flushed before every timed step, outside its events."""
    import torch
    sys.path.insert(0, ROOT)
    import paper_1609_01257_gb300 as rng

    wl = WORKLOADS["plain"]
    n, T, seed = wl["streams"], wl["iterations"], wl["seed"]
    g = rng.Generator(n, seed, init=False)
    out = torch.empty((T, n), dtype=torch.uint64, device="cuda")
    flush = L2Flush(torch)
    torch.cuda.synchronize()

    def step():
        g.init()
        g.generate_to(T, out.data_ptr())

    steps = max(args.steps, 100)
    for _ in range(args.warmup):
        flush(g.stream)
        step()
    g.sync()
    g.profile_reset()
    t0 = time.time()
    secs = timed_steps(torch, g.stream, step, steps, flush)
    t1 = time.time()
    c, kt = g.profile_stat("RNG_KERNEL")
    ran = g.last_launch()
    vpt, block, grid = ran["values_per_thread"], ran["block"], ran["grid"]
    g.close()
    k_avg = kt / max(c, 1)
    nbytes = 8 * n * T
    d = {"config": {"workload": wl["name"], "streams": n, "iterations": T, "seed": seed,
                    "bytes_per_step": nbytes, "values_per_thread": vpt, "block": block, "grid": grid,
                    "kernel": ran["kernel"], "l2": flush.label()},
         "value": nbytes * steps / secs / 1e9, "unit": "GB/s", "us_per_step": 1e6 * secs / steps,
         "kernel_us": 1e6 * k_avg, "kernel_GBps": nbytes / k_avg / 1e9, "steps": steps, "warmup": args.warmup}
    if write_ceiling:
        d["kernel_frac_write_ceiling"] = d["kernel_GBps"] / write_ceiling
    if peak:
        d["kernel_frac_hbm_peak"] = d["kernel_GBps"] / peak
    if clocks:
        d["clocks"] = clocks.window(t0, t1)
    del flush
    return d


def sweep_leg(args, clocks=None):
    """Compact roofline sweep for the default line: at each stream count 2^16
    .. 2^28 (powers of 4), the library's default shape in full-write mode
    (4 GiB ring per launch, four launches) and in generate-and-checksum
    mode (16 GiB worth of values).  Each full-write launch also reads and
    writes every stream's state once (16 B per stream), which weighs as
    much as the output at 2^28 streams (two rows per launch); the DRAM rate
    including it is reported beside the output rate.  One call through the
    ring would keep the states in registers, but then every block rewrites
    its own few ring rows while its earlier stores still sit in L2, so L2
    absorbs part of the output and the rate no longer measures HBM."""
    import torch
    sys.path.insert(0, ROOT)
    import paper_1609_01257_gb300 as rng

    ring = torch.empty(GIB // 2, dtype=torch.uint64, device="cuda")  # 2 x 2 GiB
    points = {}
    t0 = time.time()
    for e in range(16, 29, 2):
        n = 1 << e
        rows = (4 * GIB) // (8 * n)
        g = rng.Generator(n, 1, init=False)
        g.init()
        g.generate_to(rows, ring.data_ptr())
        g.sync()
        g.profile_reset()
        for _ in range(4):
            g.generate_to(rows, ring.data_ptr())
        c, t = g.profile_stat("RNG_KERNEL")
        ran = g.last_launch()
        g.close()
        T = max(1, (16 * GIB) // (8 * n))
        ck = rng.Generator(n, 1, init=False)
        ck.init()
        ck.generate_checksum(T)
        ck.sync()
        ck.init()
        ck.profile_reset()
        ck.generate_checksum(T)
        ck.sync()
        cc, ct = ck.profile_stat("CHECKSUM_KERNEL")
        ck.close()
        points[f"2^{e}"] = {"rows_per_launch": rows, "kernel": ran["kernel"],
                            "values_per_thread": ran["values_per_thread"],
                            "write_GBps": round(8 * n * rows * c / t / 1e9, 1),
                            "dram_GBps_incl_state": round((8 * n * rows + 16 * n) * c / t / 1e9, 1),
                            "checksum_values_per_s": float(f"{n * T * cc / ct:.4g}")}
    t1 = time.time()
    del ring
    torch.cuda.empty_cache()
    d = {"config": {"workload": "roofline sweep: streams 2^16..2^28 (powers of 4), seed 1, default shape; "
                                "full-write into a 2 x 2 GiB ring vs generate-and-checksum",
                    "l2": "4 GiB written per launch > L2: no flush needed"},
         "points": points}
    if clocks:
        d["clocks"] = clocks.window(t0, t1)
    return d


def run_skip(args):
    """Jump-ahead (rng_skip): every stream advanced by k = 2^40 + 12345
    iterations, one GF(2) matrix-vector product per state; 8 bytes read and
    8 written per stream.  Kernel time from the library's events."""
    import torch
    sys.path.insert(0, ROOT)
    import paper_1609_01257_gb300 as rng

    peaks, src = _peaks()
    k = (1 << 40) + 12345
    points = []
    for n in args.skip_streams:
        g = rng.Generator(n, 1)
        g.skip(1)  # materialises the states from the hash
        for _ in range(args.warmup):
            g.skip(k)
        g.sync()
        # States smaller than L2 would stay there between calls: flush it
        # before each timed call (outside the call's events).
        flush = L2Flush(torch) if L2Flush.needed(torch, 8 * n) else None
        g.profile_reset()
        call_s = timed_steps(torch, g.stream, lambda: g.skip(k), args.steps, flush)
        c, kt = g.profile_stat("SKIP_KERNEL")
        g.close()
        kern = kt / max(c, 1)
        gbs = 16 * n / kern / 1e9
        points.append({"streams": n, "call_ms": 1e3 * call_s / args.steps, "kernel_ms": 1e3 * kern,
                       "states_per_s": n / kern, "GBps": gbs, "frac_hbm": gbs / peaks["hbm_gbs"],
                       "l2": flush.label() if flush else "state > 4 x L2: no flush needed"})
        del flush
    _json_line({"workload": "jump-ahead by 2^40 + 12345 iterations", "unit": "GB/s of state read + written",
                "peak": peaks["hbm_gbs"], "peak_source": f"{src}: hbm_gbs (copy) from MEASURED_PEAKS.json",
                "points": points, "steps": args.steps})
    return 0


def run_consumer(args, wl):
    """Host consumer threads of the streamed path: per-row XOR/sum folding
    (rng_generate_host_checksum) and copies into pageable memory through the
    staging slots, against the number of consumer threads, on the streaming
    workload's shape (2^22 streams, 32 MiB rows); with `--consumer-chunks-mib`
    the fold is also timed with smaller chunks (device buffers and staging
    slots of that size, so that the slots' total footprint can fit in the
    host's last-level cache) and `--consumer-slots` staging slots (0 = one per
    consumer thread plus two); one JSON line."""
    import numpy as np
    import torch
    sys.path.insert(0, ROOT)
    import paper_1609_01257_gb300 as rng

    n, T, seed = wl["streams"], wl["iterations"], wl["seed"]
    link = measure_host_link(torch)

    def best_fold(k, chunk, slots, host_path=0):
        g = rng.Generator(n, seed, device_buffer_bytes=chunk, profiling=False, host_consumers=k,
                          host_slots=slots, host_path=host_path)
        g.generate_host_checksum(T)
        best = float("inf")
        for _ in range(args.steps):
            g.init()
            t0 = time.perf_counter()
            g.generate_host_checksum(T)
            best = min(best, time.perf_counter() - t0)
        stats = g.host_stats()
        g.close()
        return 8 * n * T / best / 1e9, stats

    fold, copy, by_chunk = {}, {}, {}
    for k in args.consumers:
        fold[k], _ = best_fold(k, wl["device_buffer_bytes"], 0)
    paths = {0: "copy engine", 2: "kernel stores into the slots", 3: "copy kernel"}
    for hp, mib, slots in ((hp, mib, slots) for hp in args.consumer_host_paths
                           for mib in args.consumer_chunks_mib for slots in args.consumer_slots):
        gbs, stats = best_fold(0, mib << 20, slots, hp)
        by_chunk[f"{paths.get(hp, hp)}: {mib} MiB x {stats['slots']} slots"] = {
            "GBps": round(gbs, 1), "slot_footprint_MiB": mib * stats["slots"], "consumers": stats["consumers"],
            "producer_wait_frac": round(stats["producer_wait_s"] / stats["wall_s"], 3)}
    rows = min(T, 128)  # 4 GiB of pageable memory, touched before timing
    out = np.ones((rows, n), dtype=np.uint64)
    for k in args.consumers:
        g = rng.Generator(n, seed, device_buffer_bytes=wl["device_buffer_bytes"], profiling=False,
                          host_path=1, host_consumers=k)
        g.generate_to_host(rows, out)
        best = float("inf")
        for _ in range(args.steps):
            g.init()
            t0 = time.perf_counter()
            g.generate_to_host(rows, out)
            best = min(best, time.perf_counter() - t0)
        g.close()
        copy[k] = 8 * n * rows / best / 1e9
    _json_line({"workload": f"host consumers: {n} streams, 32 MiB rows; fold {T} rows, "
                            f"pageable copy {rows} rows; best of {args.steps}",
                "unit": "GB/s", "host_link_GBps": link, "host_cores": os.cpu_count(),
                "fold_xor_sum": fold, "fold_default_consumers_by_chunk": by_chunk, "pageable_copy": copy})
    return 0


def run_host_dest(args, wl):
    """Host output into three kinds of page-locked destination of the full
    streaming step (32 GiB): rng_host_alloc with transparent huge pages,
    cudaHostAlloc (torch pin_memory, 64 KiB pages) and rng_host_alloc with
    base pages only.  For each: the double buffer with copy-engine reads
    (per-chunk read times from the profiler; a chunk read below 150 GB/s
    counts as stalled), the double buffer with copy-kernel reads and the
    direct path, `steps` timed steps each after one warm-up step."""
    import tempfile
    import torch
    sys.path.insert(0, ROOT)
    import paper_1609_01257_gb300 as rng

    n, T, seed = wl["streams"], wl["iterations"], wl["seed"]
    nbytes = 8 * n * T
    chunk = wl["device_buffer_bytes"]
    link = measure_host_link(torch)
    kinds = {}
    for kind in ("rng_host_alloc, huge pages", "cudaHostAlloc (torch pin_memory)", "rng_host_alloc, base pages"):
        t0 = time.perf_counter()
        if kind.startswith("cudaHostAlloc"):
            host = torch.empty((T, n), dtype=torch.uint64).pin_memory().numpy()
        else:
            host = rng.host_empty((T, n), huge_pages="huge" in kind)
        alloc_s = time.perf_counter() - t0
        res = {"alloc_s": round(alloc_s, 2), "huge_page_share": huge_page_share(host)}
        for label, hp in (("double_buffer", 1), ("double_buffer_copy_kernel", 3), ("direct", 0)):
            g = rng.Generator(n, seed, device_buffer_bytes=chunk, host_path=hp, profiling=(hp == 1), init=False)
            g.init()
            g.generate_to_host(T, host)
            rates, stalled = [], []
            for _ in range(args.steps):
                g.init()
                g.profile_reset()
                t1 = time.perf_counter()
                g.generate_to_host(T, host)
                rates.append(round(nbytes / (time.perf_counter() - t1) / 1e9, 1))
                if hp == 1:
                    with tempfile.NamedTemporaryFile("r", suffix=".tsv") as f:
                        g.profile_export(f.name)
                        reads = [(float(a), float(b)) for q, a, b, nm in
                                 (line.rstrip("\n").split("\t") for line in open(f.name)) if nm == "READ_BUFFER"]
                    # exported times are in nanoseconds
                    stalled.append(sum(1 for a, b in reads if chunk / max(b - a, 1.0) < 150.0))
            g.close()
            res[label] = {"GBps": rates}
            if hp == 1:
                res[label]["stalled_chunks"] = stalled
                res[label]["chunks_per_step"] = (nbytes + chunk - 1) // chunk
        kinds[kind] = res
        del host
        if hasattr(torch._C, "_host_emptyCache"):
            torch._C._host_emptyCache()
    _json_line({"workload": wl["name"] + ": host output into three kinds of page-locked destination",
                "unit": "GB/s", "host_link_GBps": link, "chunk_bytes": chunk,
                "stall_threshold_GBps": 150.0, "steps": args.steps, "destinations": kinds})
    return 0


def run_queue_chart(args):
    """The run the paper charts (Section 4.2, queue utilisation figure): 2^24
    values per iteration, 8 iterations, the double buffer with one 128 MiB row
    per device buffer; prints every profiled event (queue, start, end, name)."""
    import tempfile
    import torch
    sys.path.insert(0, ROOT)
    import paper_1609_01257_gb300 as rng

    n, T = 1 << 24, 8
    host = torch.empty((T, n), dtype=torch.uint64).pin_memory()
    g = rng.Generator(n, 0, device_buffer_bytes=8 * n, host_path=1, init=False)
    for _ in range(args.warmup):
        g.init()
        g.generate_to_host(T, host)
    g.init()
    g.profile_reset()
    g.generate_to_host(T, host)
    with tempfile.NamedTemporaryFile("r", suffix=".tsv") as f:
        g.profile_export(f.name)
        events = [line.rstrip("\n").split("\t") for line in open(f.name)]
    summary = g.profile_summary()
    g.close()
    _json_line({"workload": "queue chart: 2^24 values per iteration x 8 iterations, double buffer",
                "events": [[q, int(float(a)), int(float(b)), nm] for q, a, b, nm in events],
                "summary": summary})
    return 0


def run_sweep(args):
    """Roofline sweep: streams 2^16..2^28 (powers of 4) x values per thread
    1..64 (register stores) and 4, 8, 16 (bulk copies, store_policy 2),
    full-write mode and generate-and-checksum mode.

    Full-write mode: output goes to a ring of two 2 GiB device buffers; each
    launch writes the whole 4 GiB ring once (iterations = ring rows, no row
    written twice in a launch, so L2 cannot absorb rewrites), four launches
    per point (16 GiB).  Launches carry the states through the state array
    (8 B read + 8 B written per stream per launch), reported separately as
    `dram_GBps_incl_state`.  Generate-and-checksum mode: 16 GiB worth of
    values per point (no stores; per-row XOR and sum), for each compiled
    values-per-thread shape.  The CPU-baseline leg times the oracle's row
    checksums over the same rows and reports whether the GPU's checksums
    (default shape) equal them bit for bit."""
    import torch
    sys.path.insert(0, ROOT)
    import paper_1609_01257_gb300 as rng

    ring = torch.empty(GIB // 2, dtype=torch.uint64, device="cuda")  # 2 x 2 GiB
    launches = 4
    for e in range(16, 29, 2):
        n = 1 << e
        rows = (4 * GIB) // (8 * n)
        out = ring[: rows * n]
        res, res_dram = {}, {}

        def point(**kw):
            g = rng.Generator(n, 1, init=False, **kw)
            g.init()
            g.generate_to(rows, out.data_ptr())
            g.sync()
            g.profile_reset()
            for _ in range(launches):
                g.generate_to(rows, out.data_ptr())
            c, t = g.profile_stat("RNG_KERNEL")
            ran = g.last_launch()
            cfg = (ran["values_per_thread"], ran["block"], ran["grid"], ran["kernel"])
            g.close()
            return 8 * n * rows * c / t / 1e9, (8 * n * rows + 16 * n) * c / t / 1e9, cfg

        for vpt in args.sweep_vpts:
            res[vpt], res_dram[vpt], _ = point(values_per_thread=vpt)
        bulk = {vpt: point(values_per_thread=vpt, store_policy=2)[0] for vpt in args.sweep_bulk_vpts}
        dflt, dflt_dram, cfg = point()
        T = max(1, (16 * GIB) // (8 * n))

        def checksum_point(**kw):
            ck = rng.Generator(n, 1, init=False, **kw)
            ck.init()
            ck.generate_checksum(T)
            ck.sync()
            ck.init()
            ck.profile_reset()
            rx, rs = ck.generate_checksum(T)  # iterations 0 .. T-1
            ck.sync()
            c, t = ck.profile_stat("CHECKSUM_KERNEL")
            ck.close()
            return n * T / t, rx, rs

        ck_vps = {}
        for vpt in args.sweep_checksum_vpts:
            ck_vps[vpt], _, _ = checksum_point(values_per_thread=vpt)
        ck_default, rx, rs = checksum_point()
        cpu = None
        if not args.skip_cpu_baseline:
            # The oracle on the same rows: its row checksums, timed on one
            # host core, and compared with the GPU's.
            import oracle  # test infrastructure: the CPU baseline leg only
            oracle.build()
            t0 = time.perf_counter()
            wx, ws_, _ = oracle.row_checksums(n, 1, T)
            dt = time.perf_counter() - t0
            same = bool(np.array_equal(rx.cpu().numpy(), wx) and np.array_equal(rs.cpu().numpy(), ws_))
            cpu = {"value": n * T / dt, "unit": "values/s", "cores": 1, "kind": "oracle",
                   "sample": f"{n} streams x {T} iterations, row checksums, single-threaded C oracle, {dt:.1f} s",
                   "checksums_equal_gpu": same}
        _json_line({"sweep_streams": n, "rows_per_launch": rows, "launches": launches,
                    "write_GBps_by_vpt": {str(k): round(v, 1) for k, v in res.items()},
                    "dram_GBps_incl_state_by_vpt": {str(k): round(v, 1) for k, v in res_dram.items()},
                    "write_GBps_bulk_by_vpt": {str(k): round(v, 1) for k, v in bulk.items()},
                    "default_shape": {"kernel": cfg[3], "vpt": cfg[0], "grid": cfg[2], "GBps": round(dflt, 1),
                                      "dram_GBps_incl_state": round(dflt_dram, 1)},
                    "checksum_iterations": T,
                    "checksum_values_per_s_by_vpt": {str(k): float(f"{v:.4g}") for k, v in ck_vps.items()},
                    "checksum_values_per_s": ck_default,
                    "checksum_equiv_GBps": 8 * ck_default / 1e9,
                    "cpu_baseline": cpu})
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batched", "served", "sweep", "checksum", "queue-chart", "consumer", "skip", "host-dest"],
                    default="streaming")
    ap.add_argument("--duration", type=float, default=60.0, help="served workload length in seconds")
    ap.add_argument("--batch-cap-gib", type=float, default=8.0, help="batched: total output cap")
    ap.add_argument("--batch-vpt", type=int, default=0, help="batched: values per thread (0 = autotune)")
    ap.add_argument("--batch-mode", type=int, default=0, help="batched: 0 autotune, 1 per block, 2 persistent")
    ap.add_argument("--batch-uniform", type=int, nargs=3, metavar=("STREAMS", "ITERATIONS", "COUNT"),
                    help="batched: COUNT instances of STREAMS x ITERATIONS instead of the drawn 512-instance mix")
    ap.add_argument("--batch-stores", type=int, default=0,
                    help="batched: 0 autotune, 1 register/staged stores, 2 bulk copies for units of 16+ rows")
    ap.add_argument("--step-bytes", type=int, default=2 << 30, help="served: output bytes per step")
    ap.add_argument("--steps-in-flight", type=int, default=2, help="served: launched, unfinished steps")
    ap.add_argument("--server-vpt", type=int, default=4, help="served: values per thread")
    ap.add_argument("--server-mode", type=int, default=1, help="served: 1 one unit per block, 2 persistent")
    ap.add_argument("--sweep-vpts", type=int, nargs="+", default=[1, 2, 4, 6, 8, 12, 16, 24, 32, 48, 64])
    ap.add_argument("--sweep-checksum-vpts", type=int, nargs="+", default=[1, 2, 4, 8, 16, 32, 64])
    ap.add_argument("--sweep-bulk-vpts", type=int, nargs="+", default=[4, 8, 16],
                    help="sweep: values per thread of the bulk-copy row kernel (store_policy 2)")
    ap.add_argument("--skip-streams", type=int, nargs="+", default=[1 << 22, 1 << 26, 1 << 28],
                    help="skip: stream counts")
    ap.add_argument("--consumers", type=int, nargs="+", default=[1, 2, 4, 8, 16],
                    help="consumer: host consumer thread counts")
    ap.add_argument("--consumer-chunks-mib", type=int, nargs="+", default=[32],
                    help="consumer: chunk (device buffer and staging slot) sizes for the default-thread fold")
    ap.add_argument("--consumer-host-paths", type=int, nargs="+", default=[0],
                    help="consumer: host paths for the chunk sweep (0 copy engine, 2 kernel into the slots, 3 copy kernel)")
    ap.add_argument("--consumer-slots", type=int, nargs="+", default=[0],
                    help="consumer: staging slot counts for the chunk sweep (0 = consumers + 2)")
    ap.add_argument("--output-mode", type=int, choices=[0, 1], default=0,
                    help="streaming/checksum: 0 the paper's output, 1 xorshift64* scrambled values")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--skip-configs", action="store_true",
                    help="default workload: leave out the plain, batched, checksum, sweep and served objects")
    ap.add_argument("--cpu-rows", type=int, default=0,
                    help="iterations in the CPU-baseline sample (0 = the whole workload)")
    ap.add_argument("--reference-rows", type=int, default=128, help="iterations per reference step")
    ap.add_argument("--values-per-thread", type=int, default=0,
                    help="streaming/plain device leg: streams per thread of the row kernel (0 = the library's choice)")
    ap.add_argument("--block-threads", type=int, default=0,
                    help="streaming/plain device leg: threads per block of the row kernel (0 = 256)")
    ap.add_argument("--store-width", type=int, default=0, choices=[0, 1, 2, 4],
                    help="streaming/plain device leg: widest store in values (0 = per shape)")
    ap.add_argument("--grid-blocks", type=int, default=0,
                    help="streaming/plain device leg: row-kernel grid (0 = one block per tile; fewer: "
                         "persistent blocks striding over the tiles)")
    ap.add_argument("--store-policy", type=int, default=1, choices=[0, 1, 2],
                    help="streaming/plain device leg: 1 = streaming stores (st.global.cs), with bulk copies where measured faster; 0 = default stores; 2 = TMA bulk copies for every row")
    ap.add_argument("--iterations", type=int, default=0,
                    help="override the workload's iteration count (profiling captures of a smaller case)")
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)  # at least three untimed warm-up steps
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "queue-chart":
        return run_queue_chart(args)
    if args.workload == "skip":
        return run_skip(args)
    wl = dict(WORKLOADS["streaming" if args.workload in ("checksum", "consumer", "host-dest") else args.workload])
    if args.iterations:
        wl["iterations"] = args.iterations
        wl["name"] = re.sub(r"x \d+ iterations", f"x {args.iterations} iterations", wl["name"])
    if args.workload == "checksum":
        return run_checksum(args, wl)
    if args.workload == "consumer":
        return run_consumer(args, wl)
    if args.workload == "host-dest":
        return run_host_dest(args, wl)
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_gpu(args, wl)


if __name__ == "__main__":
    sys.exit(main())
