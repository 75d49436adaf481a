"""Served form: continuous batching, admission against a memory budget,
resident states across steps; results bit-exact against the oracle and the
same alone as in a mix."""
import time

import numpy as np
import pytest

import oracle
import paper_1609_01257_gb300 as rng
import workloads
from paper_1609_01257_gb300 import _capi as C

pytestmark = pytest.mark.gpu


def _collect(srv, n, timeout=60.0):
    got = {}
    t_end = time.time() + timeout
    while len(got) < n and time.time() < t_end:
        for t, addr, lat in srv.poll(64, 50):
            got[t] = (addr, lat)
    assert len(got) == n, f"only {len(got)} of {n} completed"
    return got


def _full(srv, ticket, n, T):
    return srv.read(ticket, 0, n * T).reshape(T, n)


@pytest.mark.parametrize("vpt,mode", [(0, 0), (2, 1), (4, 2), (8, 1), (8, 2), (32, 2)])
def test_mix_of_sizes_bit_exact(vpt, mode):
    # (0, 0): the defaults (4 values per thread, one unit per block).
    rs = np.random.default_rng(3)
    reqs = [(int(rs.integers(0, 2**63)), int(rs.integers(1, 70_000)), int(rs.integers(1, 40))) for _ in range(60)]
    reqs += [(5, 1, 1), (6, 2, 3), (7, 257, 1), (8, 4096, 17)]
    kw = {"values_per_thread": vpt, "mode": mode} if mode else {}
    with rng.Server(hbm_budget_bytes=2 << 30, step_bytes=4 << 20, **kw) as srv:
        tickets = {srv.submit(s, n, T): (s, n, T) for s, n, T in reqs}
        got = _collect(srv, len(reqs))
        for t, (s, n, T) in tickets.items():
            assert np.array_equal(_full(srv, t, n, T), oracle.generate(n, s, T)), (s, n, T)
            srv.release(t)
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["released"] == len(reqs)
        assert st["bytes_in_use"] == 0


def test_alone_equals_in_mix():
    target = (424242, 5001, 33)
    with rng.Server(hbm_budget_bytes=1 << 30, step_bytes=1 << 20) as srv:
        t = srv.submit(*target)
        _collect(srv, 1)
        alone = _full(srv, t, target[1], target[2])
        srv.release(t)
    rs = np.random.default_rng(9)
    with rng.Server(hbm_budget_bytes=1 << 30, step_bytes=1 << 20) as srv:
        others = [srv.submit(int(rs.integers(0, 2**63)), int(rs.integers(1, 20000)), int(rs.integers(1, 30)))
                  for _ in range(40)]
        t = srv.submit(*target)
        others += [srv.submit(int(rs.integers(0, 2**63)), int(rs.integers(1, 20000)), int(rs.integers(1, 30)))
                   for _ in range(40)]
        _collect(srv, 81)
        mixed = _full(srv, t, target[1], target[2])
        assert srv.stats()["peak_active"] > 1
    assert np.array_equal(alone, mixed)
    assert np.array_equal(alone, oracle.generate(target[1], target[0], target[2]))


def test_request_spanning_many_steps_continues_from_resident_state():
    n, T, seed = 30_000, 50, 77
    with rng.Server(hbm_budget_bytes=1 << 30, step_bytes=8 * n * 3) as srv:
        t = srv.submit(seed, n, T)
        _collect(srv, 1)
        assert srv.stats()["steps"] >= T // 3
        assert np.array_equal(_full(srv, t, n, T), oracle.generate(n, seed, T))


def test_small_requests_overtake_a_large_one():
    # Continuous batching: requests that arrive while a large one is on the
    # GPU are admitted and finish before it does.
    # The large request (32 GiB) needs at least 1024 steps of one 32 MiB row.
    with rng.Server(hbm_budget_bytes=40 << 30, step_bytes=16 << 20) as srv:
        big = srv.submit(1, 1 << 22, 1024)
        small = [srv.submit(100 + k, 1024, 4) for k in range(10)]
        order = []
        t_end = time.time() + 60
        while len(order) < 11 and time.time() < t_end:
            order += [t for t, _, _ in srv.poll(64, 50)]
        assert len(order) == 11
        assert order[-1] == big, order
        for k, t in enumerate(small):
            assert np.array_equal(_full(srv, t, 1024, 4), oracle.generate(1024, 100 + k, 4))
        got = srv.read(big, (1023 << 22) + 12345, 3)
        for j in range(3):
            assert int(got[j]) == oracle.value(12345 + j, 1, 1023)


def test_budget_admission_and_release():
    n, T = 1 << 16, 16   # 8 MiB of output + 512 KiB of state per request
    with rng.Server(hbm_budget_bytes=10 << 20, step_bytes=64 << 20) as srv:
        with pytest.raises(rng.RngError) as e:
            srv.submit(1, 1 << 20, 16)  # 128 MiB > budget
        assert e.value.code == C.RNG_EBUDGET
        t1 = srv.submit(1, n, T)
        t2 = srv.submit(2, n, T)
        first = _collect(srv, 1)
        assert list(first) == [t1]
        assert srv.poll(8, 200) == []          # t2 waits for memory
        assert srv.stats()["pending"] == 1
        srv.release(t1)
        second = _collect(srv, 1)
        assert list(second) == [t2]
        assert np.array_equal(_full(srv, t2, n, T), oracle.generate(n, 2, T))
        with pytest.raises(rng.RngError):
            srv.release(t1)                     # already released


def test_continuations_use_resident_states():
    n, seed = 5000, 31
    with rng.Server(hbm_budget_bytes=1 << 30, step_bytes=1 << 20) as srv:
        a = srv.submit_ex(seed, n, 7, keep_state=True)
        b = srv.submit_ex(0, 0, 5, keep_state=True, continue_ticket=a)  # queued behind its parent
        c = srv.submit_ex(0, 0, 3, continue_ticket=b)
        _collect(srv, 3)
        want = oracle.generate(n, seed, 15)
        assert np.array_equal(_full(srv, a, n, 7), want[:7])
        srv.release(a)
        assert np.array_equal(_full(srv, b, n, 5), want[7:12])
        assert np.array_equal(_full(srv, c, n, 3), want[12:15])
        with pytest.raises(rng.RngError) as e:
            srv.submit_ex(0, 0, 1, continue_ticket=c)  # c did not keep its states
        assert e.value.code == C.RNG_ESTATE
        with pytest.raises(rng.RngError):
            srv.submit_ex(0, 0, 1, continue_ticket=a)  # a was continued already
        srv.release(b)
        srv.release(c)
        assert srv.stats()["bytes_in_use"] == 0


def test_kept_state_freed_on_release_without_continuation():
    with rng.Server(hbm_budget_bytes=1 << 30) as srv:
        t = srv.submit_ex(4, 4096, 3, keep_state=True)
        _collect(srv, 1)
        assert srv.stats()["bytes_in_use"] > 8 * 4096 * 3
        srv.release(t)
        assert srv.stats()["bytes_in_use"] == 0


def test_invalid_requests():
    with rng.Server(hbm_budget_bytes=1 << 20) as srv:
        for args in [(1, 0, 5), (1, 5, 0), (1, (1 << 32) + 1, 1)]:
            with pytest.raises(rng.RngError) as e:
                srv.submit(*args)
            assert e.value.code == C.RNG_EINVAL
        with pytest.raises(rng.RngError):
            srv.read(12345, 0, 1)


def test_poisson_load_sampled():
    # One second of the served workload (Poisson arrivals at 2000/s, streams
    # log-uniform in [2^10, 2^22], iterations in [1, 512]); sampled requests
    # checked value by value.
    reqs = workloads.served_requests(duration_s=1.0)
    rs = np.random.default_rng(5)
    picked = set(rs.choice(len(reqs), size=min(40, len(reqs)), replace=False).tolist())
    checks = {}

    def on_complete(idx, ticket, addr):
        if idx in picked:
            r = reqs[idx]
            i = int(rs.integers(0, r.iterations))
            g = int(rs.integers(0, r.streams))
            checks[idx] = (i, g, int(srv.read(ticket, i * r.streams + g, 1)[0]),
                           srv.read(ticket, 0, min(r.streams, 4096)))

    with rng.Server(hbm_budget_bytes=64 << 30) as srv:
        res = rng.run_load(srv, reqs, on_complete=on_complete)
        assert len(res.latencies_s) == len(reqs)
        assert srv.stats()["bytes_in_use"] == 0
    for idx, (i, g, v, row0) in checks.items():
        r = reqs[idx]
        assert v == oracle.value(g, r.seed, i), idx
        assert np.array_equal(row0, oracle.generate(min(r.streams, 4096), r.seed, 1)[0]), idx
    assert res.percentile(99) < 1.0
