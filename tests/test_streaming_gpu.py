"""Paper-shaped streaming run at full size: 2^22 streams x 1024 iterations,
seed 12345, through two 32 MiB device buffers into 32 GiB of page-locked host
memory -- the launch configuration the benchmark's end-to-end leg times.
Every 16th iteration is compared in full with the oracle, and every
iteration's XOR and wrapping sum over all 2^22 values."""
import numpy as np
import pytest
import torch

import oracle
import paper_1609_01257_gb300 as rng
import workloads

pytestmark = pytest.mark.gpu


def _row_checksums(block: np.ndarray):
    x = np.bitwise_xor.reduce(block, axis=1)
    s = block.sum(axis=1, dtype=np.uint64)  # numpy wraps modulo 2^64 for uint64
    return x, s


def test_streaming_full_size_sampled_rows_and_checksums():
    cfg = workloads.STREAMING
    n, T, seed = cfg["streams"], cfg["iterations"], cfg["seed"]
    host = torch.empty((T, n), dtype=torch.uint64).pin_memory()
    g = rng.Generator(n, seed, device_buffer_bytes=cfg["device_buffer_bytes"], host_path=1)
    g.profile_reset()
    g.generate_to_host(T, host)
    prof = g.profile()
    cnt_k, _ = g.profile_stat("RNG_KERNEL")
    cnt_r, _ = g.profile_stat("READ_BUFFER")
    g.close()
    out = host.numpy()
    wx, ws, samples = oracle.row_checksums(n, seed, T, sample_every=16)
    for j, i in enumerate(range(0, T, 16)):
        assert np.array_equal(out[i], samples[j]), f"row {i} differs"
    for i0 in range(0, T, 64):
        x, s = _row_checksums(out[i0:i0 + 64])
        assert np.array_equal(x, wx[i0:i0 + 64]), f"xor checksum differs in rows {i0}..{i0 + 63}"
        assert np.array_equal(s, ws[i0:i0 + 64]), f"sum checksum differs in rows {i0}..{i0 + 63}"
    # One row per 32 MiB buffer: one kernel and one read per iteration, and
    # generation overlaps the reads.
    assert cnt_k == T and cnt_r == T
    assert prof["overlaps"], "no kernel/transfer overlap recorded"
    assert prof["aggregate"]["READ_BUFFER"][0] > prof["aggregate"]["RNG_KERNEL"][0]


def test_copy_kernel_double_buffer_full_size():
    # The double buffer with its reads done by a copy kernel (host_path 3),
    # into the same 32 GiB of page-locked memory.
    cfg = workloads.STREAMING
    n, T, seed = cfg["streams"], cfg["iterations"], cfg["seed"]
    host = torch.empty((T, n), dtype=torch.uint64).pin_memory()
    g = rng.Generator(n, seed, device_buffer_bytes=cfg["device_buffer_bytes"], host_path=3)
    g.generate_to_host(T, host)
    cnt_r, _ = g.profile_stat("READ_BUFFER")
    g.close()
    out = host.numpy()
    wx, ws, samples = oracle.row_checksums(n, seed, T, sample_every=64)
    for j, i in enumerate(range(0, T, 64)):
        assert np.array_equal(out[i], samples[j]), f"row {i} differs"
    for i0 in range(0, T, 64):
        x, s = _row_checksums(out[i0:i0 + 64])
        assert np.array_equal(x, wx[i0:i0 + 64]) and np.array_equal(s, ws[i0:i0 + 64]), i0
    assert cnt_r == T


def test_direct_to_host_full_size_checksums():
    # The same run with the kernel storing straight into host memory.
    cfg = workloads.STREAMING
    n, T, seed = cfg["streams"], cfg["iterations"], cfg["seed"]
    host = torch.empty((T, n), dtype=torch.uint64).pin_memory()
    g = rng.Generator(n, seed, host_path=2)
    g.generate_to_host(T, host)
    g.close()
    out = host.numpy()
    wx, ws, samples = oracle.row_checksums(n, seed, T, sample_every=64)
    for j, i in enumerate(range(0, T, 64)):
        assert np.array_equal(out[i], samples[j]), f"row {i} differs"
    for i0 in range(0, T, 64):
        x, s = _row_checksums(out[i0:i0 + 64])
        assert np.array_equal(x, wx[i0:i0 + 64]) and np.array_equal(s, ws[i0:i0 + 64]), i0


def test_host_checksum_full_size():
    # The same run folded on the host: the consumer threads reduce each
    # 32 MiB row as it arrives over the link, in the configuration the
    # benchmark's host-consumer leg times.
    cfg = workloads.STREAMING
    n, T, seed = cfg["streams"], cfg["iterations"], cfg["seed"]
    g = rng.Generator(n, seed, device_buffer_bytes=cfg["device_buffer_bytes"])
    rx, rs = g.generate_host_checksum(T)
    g.close()
    wx, ws, _ = oracle.row_checksums(n, seed, T)
    assert np.array_equal(rx, wx) and np.array_equal(rs, ws)


def test_checksum_mode_largest_sweep_point():
    # The sweep's largest point: 2^28 streams x 8 iterations in
    # generate-and-checksum mode, in the launch shape the sweep times.  XOR
    # against its closed form (the update is linear: XOR of row i is M^i
    # applied to the XOR of the initial states), sum against the oracle.
    from oracle import gf2
    n, T, seed = 1 << 28, 8, 1
    g = rng.Generator(n, seed)
    rx, rs = g.generate_checksum(T)
    g.sync()
    rx, rs = rx.cpu().numpy(), rs.cpu().numpy()
    g.close()
    wx, ws, _ = oracle.row_checksums(n, seed, T)
    assert np.array_equal(rx, wx) and np.array_equal(rs, ws)
    m = gf2.xorshift_matrix()
    for i in range(T):
        assert int(rx[i]) == gf2.apply(gf2.power(m, i), int(wx[0]))


def test_ring_largest_sweep_point():
    # Ring output at the sweep's largest stream count: 2^28 streams, 8
    # iterations in one call through a ring of two 2 GiB rows (ring row j
    # ends holding iteration 6 + j).  Both rows' XOR and sum against the
    # oracle, sampled values one by one, then the next call continuing from
    # the states the ring launch stored.
    n, T, R, seed = 1 << 28, 8, 2, 1
    g = rng.Generator(n, seed)
    ring = torch.zeros((R, n), dtype=torch.int64, device="cuda").view(torch.uint64)
    g.generate_ring(T, ring)
    x9, s9 = g.generate_checksum(1)   # iteration 8, from the stored states
    g.sync()
    host = ring.cpu().numpy()
    x9, s9 = x9.cpu().numpy(), s9.cpu().numpy()
    del ring
    g.close()
    wx, ws, _ = oracle.row_checksums(n, seed, T + 1)
    x, s = _row_checksums(host)
    assert np.array_equal(x, wx[T - R:T]) and np.array_equal(s, ws[T - R:T])
    assert int(x9[0]) == int(wx[T]) and int(s9[0]) == int(ws[T])
    rs = np.random.default_rng(5)
    for j, gg in zip(rs.integers(0, R, 16), rs.integers(0, n, 16)):
        assert int(host[j, gg]) == oracle.value(int(gg), seed, T - R + int(j)), (j, gg)


def test_device_resident_full_size_every_row():
    # The benchmark's device leg (2^22 x 1024 into device memory, default
    # shape): sampled values one by one, and every row's XOR and wrapping sum
    # over all 2^22 values against the oracle's.
    cfg = workloads.STREAMING
    n, T, seed = cfg["streams"], cfg["iterations"], cfg["seed"]
    g = rng.Generator(n, seed)
    out = g.generate(T)
    g.sync()
    host = torch.empty((T, n), dtype=torch.uint64).pin_memory()
    host.copy_(out)
    del out
    g.close()
    h = host.numpy()
    rs = np.random.default_rng(1)
    for i, gg in zip(rs.integers(0, T, 24), rs.integers(0, n, 24)):
        assert int(h[i, gg]) == oracle.value(int(gg), seed, int(i)), (i, gg)
    wx, ws, _ = oracle.row_checksums(n, seed, T)
    for i0 in range(0, T, 64):
        x, s = _row_checksums(h[i0:i0 + 64])
        assert np.array_equal(x, wx[i0:i0 + 64]) and np.array_equal(s, ws[i0:i0 + 64]), i0
