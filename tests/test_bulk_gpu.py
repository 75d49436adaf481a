"""Row kernel whose rows are staged in shared memory and written by TMA bulk
copies (cp.async.bulk), against the CPU oracle element by element: forced
(store_policy 2) and as the default shape chooses it, odd and even row
pitches, outputs off 16-byte and 128-byte boundaries, banded launches, rings,
output mode 1, continuation from the stored states, and host destinations
(which keep the register-store kernels)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1609_01257_gb300 as rng

pytestmark = pytest.mark.gpu

BULK_VPTS = [0, 4, 8, 16]


@pytest.mark.parametrize("vpt", BULK_VPTS)
@pytest.mark.parametrize("n", [1, 2, 5, 300, 2049, 4097, 65_537, 100_002, 250_001])
def test_forced_bulk_copies(vpt, n):
    T = 7
    g = rng.Generator(n, 31, store_policy=2, values_per_thread=vpt)
    a = g.generate(T).cpu().numpy()
    info = g.last_launch()
    b = g.generate(2).cpu().numpy()  # from the states the bulk launch stored
    g.close()
    want = oracle.generate(n, 31, T + 2)
    assert info["kernel"] == "bulk" and info["values_per_thread"] == (vpt or 8)
    assert np.array_equal(a, want[:T]) and np.array_equal(b, want[T:])


@pytest.mark.parametrize("off", [1, 2, 3, 15, 16])
@pytest.mark.parametrize("n", [64, 4097, 100_000])
def test_unaligned_outputs_and_canaries(off, n):
    # Outputs that start 8 bytes off a 16-byte boundary or off a 128-byte
    # line: odd heads and tails go out as 8-byte stores, nothing outside the
    # output changes.
    T = 5
    buf = torch.full((T * n + off + 8,), -1, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()  # generate_to launches on the library's stream
    g = rng.Generator(n, 8, store_policy=2)
    g.generate_to(T, buf.data_ptr() + 8 * off)
    g.sync()
    g.close()
    got = buf.cpu().numpy().view(np.uint64)
    assert np.array_equal(got[off:off + T * n], oracle.generate(n, 8, T).reshape(-1))
    assert (got[:off] == np.uint64(2**64 - 1)).all() and (got[off + T * n:] == np.uint64(2**64 - 1)).all()


@pytest.mark.parametrize("vpt", [4, 8, 16])
@pytest.mark.parametrize("n,T", [(5, 3000), (300, 2049), (4096, 1000), (70_001, 300)])
def test_banded_bulk_copies(vpt, n, T):
    # Too few tiles to fill the GPU: rows split into bands whose blocks jump
    # their states ahead over GF(2) before staging.
    g = rng.Generator(n, 17, store_policy=2, values_per_thread=vpt)
    a = g.generate(T).cpu().numpy()
    info = g.last_launch()
    b = g.generate(3).cpu().numpy()
    g.close()
    want = oracle.generate(n, 17, T + 3)
    assert info["kernel"] == "bulk" and info["band_rows"] > 0
    assert np.array_equal(a, want[:T]) and np.array_equal(b, want[T:])


@pytest.mark.parametrize("n,T,R", [(3001, 23, 4), (4096, 9, 9), (65_537, 10, 3), (7, 50, 1)])
def test_bulk_copies_into_a_ring(n, T, R):
    g = rng.Generator(n, 21, store_policy=2)
    ring = torch.zeros((R, n), dtype=torch.int64, device="cuda").view(torch.uint64)
    g.generate_ring(T, ring)
    info = g.last_launch()
    after = g.generate(2).cpu().numpy()
    got = ring.cpu().numpy()
    g.close()
    want = oracle.generate(n, 21, T + 2)
    assert info["kernel"] == "bulk"
    for j in range(R):
        its = [i for i in range(T) if i % R == j]
        assert np.array_equal(got[j], want[its[-1]]) if its else (got[j] == 0).all(), j
    assert np.array_equal(after, want[T:])


@pytest.mark.parametrize("vpt", BULK_VPTS)
@pytest.mark.parametrize("n,T", [(1, 5), (4097, 20), (262_147, 3), (70_001, 300)])
def test_bulk_copies_output_mode_1(vpt, n, T):
    g = rng.Generator(n, 41, store_policy=2, values_per_thread=vpt, output_mode=1)
    a = g.generate(T).cpu().numpy()
    g.close()
    assert np.array_equal(a, oracle.generate(n, 41, T, output_mode=1))


@pytest.mark.parametrize("n", [65_537, 250_001, 1_000_003, 3_000_017, (1 << 22) + 1])
def test_default_shape_takes_bulk_copies_for_rows_off_the_lines(n):
    # From 128 rows per launch; fewer rows keep the register or staged kernels.
    g = rng.Generator(n, 4)
    a = g.generate(128).cpu().numpy()
    info = g.last_launch()
    b = g.generate(3).cpu().numpy()
    few = g.last_launch()
    g.close()
    want = oracle.generate(n, 4, 131)
    assert info["kernel"] == "bulk" and few["kernel"] != "bulk"
    assert np.array_equal(a, want[:128]) and np.array_equal(b, want[128:])


def test_default_shape_for_lined_rows():
    # Rows on 128-byte lines: bulk copies from 3.5 M streams (and 128 rows),
    # register stores below.
    for n, T, kernel in ((1 << 22, 128, "bulk"), (1 << 22, 2, "register"), (1 << 20, 128, "register"),
                         (1 << 16, 128, "register")):
        g = rng.Generator(n, 6)
        a = g.generate(T).cpu().numpy()
        info = g.last_launch()
        g.close()
        assert info["kernel"] == kernel, (n, T, info)
        assert np.array_equal(a, oracle.generate(n, 6, T))


@pytest.mark.parametrize("host_path", [1, 2])
def test_host_destinations_keep_register_stores(host_path):
    n, T = 250_001, 6
    g = rng.Generator(n, 9, store_policy=2, host_path=host_path, device_buffer_bytes=8 * n * 2)
    host = torch.zeros((T, n), dtype=torch.int64).pin_memory()
    g.generate_to_host(T, host.view(torch.uint64))
    info = g.last_launch()
    g.close()
    assert info["kernel"] != "bulk"
    assert np.array_equal(host.numpy().view(np.uint64), oracle.generate(n, 9, T))


def test_last_launch_before_any_launch_is_a_state_error():
    g = rng.Generator(1000, 1)
    with pytest.raises(rng.RngError):
        g.last_launch()
    g.generate(2)
    assert g.last_launch()["kernel"] in ("register", "staged", "bulk")
    g.close()


@pytest.mark.parametrize("off", [123_456, (1 << 32) - 4097])
def test_bulk_copies_with_a_stream_offset(off):
    # A shard of a larger generator: ids off .. off + n - 1, up to the
    # 32-bit id limit.
    n, T = 4097, 9
    g = rng.Generator(n, 77, stream_offset=off, store_policy=2)
    a = g.generate(T).cpu().numpy()
    g.close()
    assert np.array_equal(a, oracle.generate(n, 77, T, g0=off))


@pytest.mark.parametrize("grid", [1, 3, 7])
@pytest.mark.parametrize("n,T", [(70_001, 9), (20_000, 40), (4096 * 5 + 3, 17)])
def test_bulk_copies_with_blocks_striding_over_tiles(grid, n, T):
    # A grid smaller than the tile count: each block runs several tiles one
    # after another, its row buffers rotating across them.
    g = rng.Generator(n, 13, store_policy=2, grid_blocks=grid)
    a = g.generate(T).cpu().numpy()
    info = g.last_launch()
    b = g.generate(2).cpu().numpy()
    g.close()
    want = oracle.generate(n, 13, T + 2)
    assert info["kernel"] == "bulk" and info["grid"] == grid
    assert np.array_equal(a, want[:T]) and np.array_equal(b, want[T:])
