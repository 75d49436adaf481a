"""The seeded workload generators: draw rules and the shapes the workload
definitions ask for (no generator arithmetic lives here)."""
import math

import numpy as np
import pytest

import workloads


def test_splitmix64_sequence_is_deterministic_and_distinct():
    a = [workloads.SplitMix64(7).next() for _ in range(1)]
    s1, s2 = workloads.SplitMix64(7), workloads.SplitMix64(7)
    xs = [s1.next() for _ in range(1000)]
    assert xs == [s2.next() for _ in range(1000)]
    assert len(set(xs)) == 1000 and a[0] == xs[0]
    assert all(0 <= x < 1 << 64 for x in xs)


def test_uniform_and_log_uniform_ranges():
    s = workloads.SplitMix64(1)
    u = np.array([s.uniform() for _ in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    v = np.array([s.log_uniform_int(1 << 8, 1 << 20) for _ in range(20000)])
    assert v.min() >= 1 << 8 and v.max() <= 1 << 20
    # log-uniform: log2 of the draws is close to uniform on [8, 20]
    assert abs(np.log2(v).mean() - 14.0) < 0.1


def test_batched_instances_shape_and_cap():
    inst = workloads.batched_instances()
    assert len(inst) == 512
    assert sum(i.nbytes for i in inst) <= 8 * workloads.GIB
    assert all((1 << 8) <= i.streams <= (1 << 20) and 1 <= i.iterations <= 4096 for i in inst)
    assert len({i.seed for i in inst}) == 512
    assert inst == workloads.batched_instances()  # seeded


def test_batched_cap_binds_only_when_needed():
    small = workloads.batched_instances(count=4, streams_hi=1 << 9, iters_hi=4)
    assert sum(i.nbytes for i in small) < 8 * workloads.GIB
    capped = workloads.batched_instances(count=64, cap_bytes=1 << 30)
    assert sum(i.nbytes for i in capped) <= 1 << 30


def test_served_requests_poisson_shape():
    reqs = workloads.served_requests(duration_s=5.0)
    assert abs(len(reqs) - 10000) < 4 * math.sqrt(10000)   # 2000/s for 5 s
    t = np.array([r.arrival_s for r in reqs])
    assert (np.diff(t) > 0).all() and t[-1] < 5.0
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 2000) < 0.05 / 2000 * 4
    assert all((1 << 10) <= r.streams <= (1 << 22) and 1 <= r.iterations <= 512 for r in reqs)


def test_sweep_points_write_at_least_16_gib():
    for n, v, t in workloads.sweep_points():
        assert 8 * n * t >= 16 * workloads.GIB
