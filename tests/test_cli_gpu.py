"""The paper's program interface: raw uint64 values to a file descriptor /
stdout (Section 5), and the queue-utilisation export of the double-buffer
run the paper charts (2^24 values per iteration, 8 iterations)."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
import paper_1609_01257_gb300 as rng

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_generate_fd_writes_raw_values(tmp_path):
    n, T = 3000, 9
    path = tmp_path / "out.bin"
    with open(path, "wb") as f:
        g = rng.Generator(n, 12, device_buffer_bytes=8 * n * 2)
        g.generate_fd(T, f.fileno())
        g.close()
    got = np.fromfile(path, dtype=np.uint64)
    assert got.size == n * T
    assert np.array_equal(got.reshape(T, n), oracle.generate(n, 12, T))


def test_cli_stdout_matches_oracle():
    n, T = 1000, 7
    r = subprocess.run([sys.executable, "-m", "paper_1609_01257_gb300", str(n), str(T), "--seed", "5",
                        "--profile"], cwd=ROOT, capture_output=True, timeout=300)
    assert r.returncode == 0, r.stderr.decode()
    assert len(r.stdout) == 8 * n * T   # Eq. 1
    got = np.frombuffer(r.stdout, dtype=np.uint64).reshape(T, n)
    assert np.array_equal(got, oracle.generate(n, 5, T))
    assert b"Aggregate times by event" in r.stderr


def test_cli_output_mode_1():
    n, T = 777, 4
    r = subprocess.run([sys.executable, "-m", "paper_1609_01257_gb300", str(n), str(T), "--seed", "5",
                        "--output-mode", "1"], cwd=ROOT, capture_output=True, timeout=300)
    assert r.returncode == 0, r.stderr.decode()
    got = np.frombuffer(r.stdout, dtype=np.uint64).reshape(T, n)
    assert np.array_equal(got, oracle.generate(n, 5, T, output_mode=1))


def test_c_example_program_matches_oracle():
    # The paper's program as a plain C client of the library (built by build()).
    from paper_1609_01257_gb300 import builder
    n, T = 2000, 5
    r = subprocess.run([builder.EXAMPLE, str(n), str(T), "7"], capture_output=True, timeout=300)
    assert r.returncode == 0, r.stderr.decode()
    got = np.frombuffer(r.stdout, dtype=np.uint64)
    assert got.size == n * T
    assert np.array_equal(got.reshape(T, n), oracle.generate(n, 7, T))
    assert b"Time spent in device" in r.stderr
    assert b"objects left alive" not in r.stderr


def test_queue_chart_export_of_the_papers_run(tmp_path):
    # One 128 MiB row per device buffer: each iteration is one kernel on the
    # main queue and one read on the comms queue, the reads of one buffer
    # overlapping the generation into the other.
    n, T = 1 << 24, 8
    host = torch.empty((T, n), dtype=torch.uint64).pin_memory()
    g = rng.Generator(n, 0, device_buffer_bytes=8 * n, host_path=1)
    g.profile_reset()
    g.generate_to_host(T, host)
    path = tmp_path / "events.tsv"
    g.profile_export(str(path))
    prof = g.profile()
    g.close()
    rows = [line.split("\t") for line in path.read_text().splitlines()]
    kern = [r for r in rows if r[3] == "RNG_KERNEL"]
    read = [r for r in rows if r[3] == "READ_BUFFER"]
    assert len(kern) == T and len(read) == T
    assert all(r[0] == "Main" for r in kern) and all(r[0] == "Comms" for r in read)
    assert all(float(r[1]) <= float(r[2]) for r in rows)
    # read k starts after kernel k ends; kernel k+1 runs while read k runs
    for k in range(T):
        assert float(read[k][1]) >= float(kern[k][2])
    assert prof["overlaps"].get(("RNG_KERNEL", "READ_BUFFER"), 0) > 0
    assert np.array_equal(host.numpy()[::7], oracle.generate(n, 0, T)[::7])
