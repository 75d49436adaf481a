"""Host consumer threads of the streamed path (Section 5, "out" block):
per-row XOR / wrapping-sum folding on the host, several threads draining the
staging slots, and pageable copies split across them.  Every result is
compared with the oracle."""
import threading

import numpy as np
import pytest

import oracle
import paper_1609_01257_gb300 as rng

pytestmark = pytest.mark.gpu


# (streams, iterations, device buffer bytes): whole rows per chunk, a ragged
# last chunk, and rows split into column slabs (buffer smaller than a row,
# odd widths) so that several threads fold parts of one row.
CASES = [
    (1, 9, 64),
    (1000, 37, 8 * 1000 * 5),
    (4097, 20, 8 * 4097 * 3 + 8),  # device buffers are multiples of 16 bytes
    (30_001, 7, 8 * 4096),
    (262_147, 5, 8 * 65_536),
]


@pytest.mark.parametrize("n,T,buf", CASES)
@pytest.mark.parametrize("consumers,host_path", [(1, 0), (3, 0), (8, 0), (3, 3), (1, 2), (3, 2)])
def test_host_checksum_matches_oracle(n, T, buf, consumers, host_path):
    # host_path 3: the slots are filled by a copy kernel instead of the copy
    # engine; host_path 2: the kernel stores each chunk straight into its slot.
    g = rng.Generator(n, 21, device_buffer_bytes=buf, host_consumers=consumers, host_path=host_path)
    rx, rs = g.generate_host_checksum(T)
    tail = g.generate(2).cpu().numpy()  # the streams advanced by T
    g.close()
    wx, ws, _ = oracle.row_checksums(n, 21, T)
    assert np.array_equal(rx, wx) and np.array_equal(rs, ws)
    assert np.array_equal(tail, oracle.generate(n, 21, 2, p0=T))


def test_host_checksum_equals_device_checksum_after_position():
    # Started mid-stream: both checksum forms cover the same iterations.
    n = 50_000
    g = rng.Generator(n, 3, device_buffer_bytes=8 * n * 2)
    g.generate(11)
    hx, hs = g.generate_host_checksum(13)
    g.close()
    g = rng.Generator(n, 3)
    g.generate(11)
    dx, ds = g.generate_checksum(13)
    g.sync()
    dx, ds = dx.cpu().numpy(), ds.cpu().numpy()
    g.close()
    assert np.array_equal(hx, dx) and np.array_equal(hs, ds)
    wx, ws, _ = oracle.row_checksums(n, 3, 13, p0=11)
    assert np.array_equal(hx, wx) and np.array_equal(hs, ws)


def test_host_checksum_zero_iterations_and_not_initialised():
    g = rng.Generator(100, 1, init=False)
    with pytest.raises(rng.RngError) as e:
        g.generate_host_checksum(3)
    assert e.value.code == 4
    g.init()
    rx, rs = g.generate_host_checksum(0)
    assert rx.size == 0 and rs.size == 0
    assert np.array_equal(g.generate(1).cpu().numpy(), oracle.generate(100, 1, 1))
    g.close()


def test_concurrent_sink_sees_every_chunk_once():
    n, T = 3000, 40
    g = rng.Generator(n, 6, device_buffer_bytes=8 * n * 3, host_consumers=4)
    got = np.zeros((T, n), dtype=np.uint64)
    seen = []
    lock = threading.Lock()

    def sink(first_it, block, first_stream):
        with lock:
            seen.append(first_it)
        got[first_it:first_it + block.shape[0], first_stream:first_stream + block.shape[1]] = block

    g.generate_sink(T, sink)
    g.close()
    assert sorted(seen) == list(range(0, T, 3))
    assert np.array_equal(got, oracle.generate(n, 6, T))


@pytest.mark.parametrize("consumers,host_path", [(1, 1), (4, 1), (4, 3)])
def test_pageable_copy_with_consumers(consumers, host_path):
    # Double buffer into pageable memory: copies out of the staging slots
    # are spread over the consumer threads.
    n, T = 70_001, 9
    g = rng.Generator(n, 8, device_buffer_bytes=8 * 20_000, host_path=host_path, host_consumers=consumers)
    out = np.zeros((T, n), dtype=np.uint64)
    g.generate_to_host(T, out)
    g.close()
    assert np.array_equal(out, oracle.generate(n, 8, T))


@pytest.mark.parametrize("host_path", [0, 2, 3])
def test_fd_output_in_order_with_consumers(tmp_path, host_path):
    # rng_generate_fd keeps one consumer whatever host_consumers says: the
    # bytes reach the file in stream order.
    n, T = 5000, 12
    g = rng.Generator(n, 4, device_buffer_bytes=8 * n, host_consumers=6, host_path=host_path)
    path = tmp_path / "out.bin"
    with open(path, "wb") as f:
        g.generate_fd(T, f.fileno())
    g.close()
    got = np.fromfile(path, dtype=np.uint64).reshape(T, n)
    assert np.array_equal(got, oracle.generate(n, 4, T))


@pytest.mark.parametrize("consumers", [1, 4])
def test_sink_with_chunks_stored_straight_into_the_slots(consumers):
    # host_path 2: no device buffer and no copy -- one kernel per chunk
    # writes the slot over the host link, then a consumer hands it on.
    n, T = 4099, 31
    g = rng.Generator(n, 17, device_buffer_bytes=8 * n * 4, host_path=2, host_consumers=consumers)
    got = np.zeros((T, n), dtype=np.uint64)
    order = []

    def sink(first_it, block, first_stream):
        order.append(first_it)
        got[first_it:first_it + block.shape[0], first_stream:first_stream + block.shape[1]] = block

    g.profile_reset()
    g.generate_sink(T, sink)
    kernels, _ = g.profile_stat("RNG_KERNEL")
    reads, _ = g.profile_stat("READ_BUFFER")
    g.close()
    assert (kernels, reads) == (8, 0)
    if consumers == 1:
        assert order == list(range(0, T, 4))
    assert sorted(order) == list(range(0, T, 4))
    assert np.array_equal(got, oracle.generate(n, 17, T))


def test_host_consumers_bound():
    with pytest.raises(rng.RngError) as e:
        rng.Generator(16, 1, host_consumers=65)
    assert e.value.code == 1


def test_host_stats_show_a_slow_consumer():
    # A sink slower than the link: the issuing thread spends most of the call
    # waiting for free slots, and the consumer's time covers the sleeps.
    # Of 20 chunks, the last 17 each wait for the consumer to free a slot.
    import time
    n, T = 4096, 40
    g = rng.Generator(n, 2, device_buffer_bytes=8 * n * 2)

    def slow(first_it, block, first_stream):
        time.sleep(0.02)

    g.generate_sink(T, slow)
    s = g.host_stats()
    g.close()
    assert s["chunks"] == 20 and s["consumers"] == 1 and s["slots"] == 3
    assert s["consume_s"] >= 20 * 0.02 * 0.9
    assert s["producer_wait_s"] > 0.6 * s["wall_s"] and s["wall_s"] >= s["consume_s"] * 0.9


def test_host_stats_of_a_fold_and_of_a_page_locked_copy():
    import torch
    n, T = 8192, 10
    g = rng.Generator(n, 2, device_buffer_bytes=8 * n, host_consumers=4)
    g.generate_host_checksum(T)
    s = g.host_stats()
    assert s["chunks"] == T and s["consumers"] == 4 and s["slots"] == 6
    assert s["wall_s"] > 0 and s["consume_s"] > 0 and s["copy_wait_s"] >= 0
    g.close()
    # Page-locked destination on the double buffer: copies land in place, no
    # staging slots and no consumer threads.
    host = torch.empty((T, n), dtype=torch.uint64).pin_memory()
    g = rng.Generator(n, 2, device_buffer_bytes=8 * n * 5, host_path=1)
    g.generate_to_host(T, host)
    s = g.host_stats()
    g.close()
    assert s["chunks"] == 2 and s["consumers"] == 0 and s["slots"] == 0
    assert np.array_equal(host.numpy(), oracle.generate(n, 2, T))
