"""Host-side pieces of bench.py: clock-sample parsing, the traffic lookup
(reported only while the kernel sources match the capture), peaks, and the
step timing with an L2 flush outside each step's events."""
import os

import bench


def test_parse_clock_samples():
    text = """0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active
0, 1980, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active
0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active
garbage line
"""
    c = bench.parse_clock_samples(text)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.parse_clock_samples("") is None


def test_clock_samples_inside_the_timed_region():
    warm = "0, 1500, 2070, 300.0, 0x1, Not Active, Not Active, Not Active, Not Active\n"
    busy = "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Active\n"
    lines = [(1.0, warm), (2.0, busy), (2.1, busy), (3.0, warm)]
    c = bench.clocks_in_window(lines, 1.9, 2.2)
    assert c["sm_mhz"] == 2070.0 and c["samples"] == 2 and c["window"] == "timed region"
    assert c["reasons"] == ["sw_power_cap"]
    c = bench.clocks_in_window(lines, 2.5, 2.6)  # no sample inside: all of them
    assert c["samples"] == 4 and c["window"].startswith("warm-up")
    assert bench.clocks_in_window([], 0, 1) is None


def test_traffic_lookup_tracks_kernel_sources(tmp_path, monkeypatch):
    f = tmp_path / "rows_bulk_kernel_traffic.md"
    f.write_text(f"kernel_source_sha256_16: {bench._kernel_source_hash()}\n"
                 "traffic_bytes_per_launch[streaming]: 3.5e+10\n")
    monkeypatch.setattr(bench, "PROFILES_DIR", str(tmp_path))
    assert bench._traffic_per_launch("streaming", "rows_bulk_kernel") == 3.5e10
    assert bench._traffic_per_launch("plain", "rows_bulk_kernel") is None
    assert bench._traffic_per_launch("streaming", "rows_kernel") is None  # no summary for that kernel
    f.write_text("kernel_source_sha256_16: 0000000000000000\ntraffic_bytes_per_launch[streaming]: 3.5e+10\n")
    assert bench._traffic_per_launch("streaming", "rows_bulk_kernel") is None


def test_committed_traffic_summary_matches_the_kernel_sources():
    # The streaming workload's device leg runs the bulk-copy row kernel; its
    # committed ncu summary must be taken on the current kernel sources.
    assert bench._traffic_per_launch("streaming", "rows_bulk_kernel") is not None


class _FakeEvent:
    """Stand-in for torch.cuda.Event: the clock advances by one unit per
    record, so elapsed times count the records between two events."""
    clock = 0.0

    def __init__(self, enable_timing=True):
        self.t = None

    def record(self, stream):
        _FakeEvent.clock += 1.0
        self.t = _FakeEvent.clock

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return other.t - self.t


def test_timed_steps_flush_outside_the_step_events():
    import types
    fake = types.SimpleNamespace(cuda=types.SimpleNamespace(Event=_FakeEvent))
    log = []
    # One event pair around all steps: 2 records 1 unit apart (ms -> s).
    assert bench.timed_steps(fake, None, lambda: log.append("step"), 4) == 1e-3
    log.clear()
    # With a flush: each step has its own pair, the flush runs before it and
    # outside it, and the result sums the steps (3 x 1 unit).
    t = bench.timed_steps(fake, None, lambda: log.append("step"), 3, flush=lambda s: log.append("flush"))
    assert t == 3e-3
    assert log == ["flush", "step"] * 3


def test_peaks_file_is_read():
    peaks, src = bench._peaks()
    assert peaks["hbm_gbs"] > 0
    if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        assert src == "measured"


def test_reference_arm_prints_one_json_line(capsys):
    # The reference arm times the CPU oracle; it needs no GPU.
    rc = bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3", "--reference-rows", "1"])
    assert rc == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    import json
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GB/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["higher_is_better"] is True


def test_all_cores_oracle_baseline_covers_every_stream():
    # One process per host core on contiguous stream-id blocks: together they
    # produce exactly the workload's bytes.
    nbytes, secs, procs = bench.cpu_oracle_all_cores(10_007, 3, 5)
    assert nbytes == 8 * 10_007 * 5 and secs > 0 and 1 <= procs <= (os.cpu_count() or 1)
