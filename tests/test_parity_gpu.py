"""GPU path against the CPU oracle, element by element (bit-exact: all of
the generator's arithmetic is integer)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1609_01257_gb300 as rng
import workloads

pytestmark = pytest.mark.gpu


def dev_gen(n, seed, T, **kw):
    g = rng.Generator(n, seed, **kw)
    out = g.generate(T)
    g.sync()
    res = out.cpu().numpy()
    g.close()
    return res


def test_plain_method_full_compare():
    # 2^16 streams x 100 iterations, seed 0, device-resident: every value.
    cfg = workloads.PLAIN
    got = dev_gen(cfg["streams"], cfg["seed"], cfg["iterations"])
    want = oracle.generate(cfg["streams"], cfg["seed"], cfg["iterations"])
    assert got.shape == want.shape
    assert np.array_equal(got, want)
    assert (got != 0).all()


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 31, 33, 255, 257, 1023, 1025, 4095, 4097, 65535, 65537])
@pytest.mark.parametrize("T", [1, 3, 17])
def test_ragged_sizes(n, T):
    got = dev_gen(n, 12345, T)
    assert np.array_equal(got, oracle.generate(n, 12345, T))


VPTS = [1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16, 20, 24, 28, 32, 48, 64]


@pytest.mark.parametrize("vpt", VPTS)
@pytest.mark.parametrize("n", [4096 * 3 + 4, 100_001, 100_002])
def test_values_per_thread_variants(vpt, n):
    want = oracle.generate(n, 99, 9)
    for width in (1, 2, 4):
        got = dev_gen(n, 99, 9, values_per_thread=vpt, store_width=width)
        assert np.array_equal(got, want), (vpt, width)


@pytest.mark.parametrize("policy", [0, 1])
def test_store_policies(policy):
    got = dev_gen(70_000, 3, 11, store_policy=policy)
    assert np.array_equal(got, oracle.generate(70_000, 3, 11))


@pytest.mark.parametrize("seed", [0, 1, 12345, 2**64 - 1, 0x9E3779B97F4A7C15])
def test_seeds(seed):
    assert np.array_equal(dev_gen(5000, seed, 4), oracle.generate(5000, seed, 4))


def test_continuation_equals_single_call():
    g = rng.Generator(3001, 7)
    a = g.generate(5).cpu().numpy()
    b = g.generate(1).cpu().numpy()
    c = g.generate(13).cpu().numpy()
    assert g.position == 19
    g.close()
    want = oracle.generate(3001, 7, 19)
    assert np.array_equal(np.concatenate([a, b, c]), want)


def test_separate_init_kernel_equals_fused():
    for fuse in (True, False):
        g = rng.Generator(4099, 5, fuse_init=fuse)
        st = g.state()  # initial states (iteration-0 values)
        assert np.array_equal(st, oracle.generate(4099, 5, 1)[0])
        out = g.generate(6).cpu().numpy()
        assert np.array_equal(out, oracle.generate(4099, 5, 6))
        assert np.array_equal(g.state(), oracle.generate(4099, 5, 1, p0=6)[0])
        g.close()


def test_reinit_restarts():
    g = rng.Generator(1000, 11)
    first = g.generate(4).cpu().numpy()
    g.generate(3)
    g.init()
    again = g.generate(4).cpu().numpy()
    g.close()
    assert np.array_equal(first, again)


def test_stream_offset_is_a_column_block():
    n, off, T = 2000, 123_456, 5
    got = dev_gen(n, 77, T, stream_offset=off)
    assert np.array_equal(got, oracle.generate(n, 77, T, g0=off))


def test_ids_up_to_the_32_bit_limit():
    # The last ids a generator can own: stream_offset + streams == 2^32.
    n = 1000
    got = dev_gen(n, 5, 4, stream_offset=(1 << 32) - n)
    assert np.array_equal(got, oracle.generate(n, 5, 4, g0=(1 << 32) - n))
    with pytest.raises(rng.RngError):
        rng.Generator(n, 5, stream_offset=(1 << 32) - n + 1)


@pytest.mark.parametrize("policy", [1, 2])
def test_maximum_stream_count(policy):
    # 2^32 streams (the id width): 2 iterations = 64 GiB of output plus a
    # 32 GiB state array; sampled values one by one.  Policy 2 runs the
    # bulk-copy row kernel (2^21 blocks, 64-bit row offsets).
    n, T, seed = 1 << 32, 2, 3
    g = rng.Generator(n, seed, store_policy=policy)
    out = g.generate(T)
    g.sync()
    o64 = out.view(torch.int64).view(-1)
    rs = np.random.default_rng(4)
    idx = [0, 1, n - 1, n, 2 * n - 1] + [int(i) for i in rs.integers(0, 2 * n, 40)]
    vals = o64[torch.tensor(idx, device="cuda")].cpu().numpy().view(np.uint64)
    ran = g.last_launch()["kernel"]
    del out, o64
    g.close()
    assert ran == ("bulk" if policy == 2 else "register")
    for k, v in zip(idx, vals):
        i, gg = divmod(k, n)
        assert int(v) == oracle.value(gg, seed, i), (i, gg)


def test_generate_before_init_is_an_error():
    g = rng.Generator(10, 1, init=False)
    with pytest.raises(rng.RngError) as e:
        g.generate(2)
    assert e.value.code == 4
    g.close()


def test_both_or_no_output_is_an_error():
    import ctypes
    from paper_1609_01257_gb300 import _capi as C
    g = rng.Generator(10, 1)
    L = C.load()
    buf = torch.empty(40, dtype=torch.uint64, device="cuda")
    host = np.empty(40, dtype=np.uint64)
    assert L.rng_generate(g._h, 2, None, None, None) == C.RNG_EINVAL
    assert L.rng_generate(g._h, 2, ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(host.ctypes.data), None) == C.RNG_EINVAL
    assert L.rng_generate(g._h, 0, ctypes.c_void_p(buf.data_ptr()), None, None) == C.RNG_OK
    g.close()


def test_unaligned_device_output():
    # 8-byte aligned but not 16: scalar-store path.
    n, T = 1000, 7
    g = rng.Generator(n, 2)
    raw = torch.zeros(n * T + 1, dtype=torch.int64, device="cuda")
    g.generate_to(T, raw.data_ptr() + 8)
    g.sync()
    got = raw.cpu().numpy().view(np.uint64)
    g.close()
    assert got[0] == 0
    assert np.array_equal(got[1:].reshape(T, n), oracle.generate(n, 2, T))


def test_no_write_outside_output():
    # Canary words around the output region stay untouched.
    n, T = 5003, 9
    g = rng.Generator(n, 8)
    pad = 64
    raw = torch.full((n * T + 2 * pad,), 0xA5A5A5A5, dtype=torch.int64, device="cuda")
    g.generate_to(T, raw.data_ptr() + pad * 8)
    g.sync()
    r = raw.cpu().numpy()
    g.close()
    assert (r[:pad] == 0xA5A5A5A5).all() and (r[-pad:] == 0xA5A5A5A5).all()
    assert np.array_equal(r[pad:-pad].view(np.uint64).reshape(T, n), oracle.generate(n, 8, T))


@pytest.mark.parametrize("host_path", [0, 1, 3])
@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("n,T,buf", [(4096, 40, 1 << 16), (3001, 7, 8 * 3001 * 2), (5000, 3, 4096), (7, 100, 64)])
def test_host_output(host_path, pinned, n, T, buf):
    # host_path 1: the double buffer; buf smaller than one row (5000 streams x
    # 8 B > 4096) exercises column slabs.  host_path 3: the same with the
    # reads done by a copy kernel (odd widths: 8-byte aligned destinations).
    # host_path 0: direct stores where the GPU can reach the destination.
    g = rng.Generator(n, 4, device_buffer_bytes=buf, host_path=host_path)
    out = torch.empty((T, n), dtype=torch.uint64)
    if pinned:
        out = out.pin_memory()
    g.generate_to_host(T, out)
    first = out.numpy().copy()
    second = g.generate_to_host(2)
    assert g.position == T + 2
    g.close()
    want = oracle.generate(n, 4, T + 2)
    assert np.array_equal(first, want[:T])
    assert np.array_equal(second, want[T:])


@pytest.mark.parametrize("host_path", [0, 1, 3])
def test_device_then_host_then_device(host_path):
    g = rng.Generator(2048, 9, device_buffer_bytes=8 * 2048 * 3, host_path=host_path)
    a = g.generate(4).cpu().numpy()
    b = g.generate_to_host(10)
    c = g.generate(2).cpu().numpy()
    g.close()
    assert np.array_equal(np.concatenate([a, b, c]), oracle.generate(2048, 9, 16))


def test_sink_receives_every_chunk_in_order():
    n, T = 3000, 25
    g = rng.Generator(n, 6, device_buffer_bytes=8 * n * 4, host_slots=3)
    got = np.zeros((T, n), dtype=np.uint64)
    seen = []

    def sink(first_it, block, first_stream):
        seen.append((first_it, block.shape[0], first_stream))
        got[first_it:first_it + block.shape[0], first_stream:first_stream + block.shape[1]] = block

    g.generate_sink(T, sink)
    g.close()
    assert [s[0] for s in seen] == sorted(s[0] for s in seen)
    assert np.array_equal(got, oracle.generate(n, 6, T))


def test_sink_error_stops_run():
    g = rng.Generator(1000, 6, device_buffer_bytes=8 * 1000)
    calls = []

    def sink(first_it, block, first_stream):
        calls.append(first_it)
        return 1 if first_it == 3 else 0

    with pytest.raises(rng.RngError) as e:
        g.generate_sink(20, sink)
    assert e.value.code == 7
    assert calls[-1] == 3
    # The run failed part-way: the generator must be re-initialised.
    with pytest.raises(rng.RngError):
        g.generate(1)
    g.init()
    assert np.array_equal(g.generate(2).cpu().numpy(), oracle.generate(1000, 6, 2))
    g.close()


def test_stalled_consumer_times_out():
    import time
    g = rng.Generator(512, 6, device_buffer_bytes=8 * 512, host_slots=2, host_wait_ms=200)

    def slow(first_it, block, first_stream):
        time.sleep(0.6)

    with pytest.raises(rng.RngError) as e:
        g.generate_sink(8, slow)
    assert e.value.code == 5
    g.close()


@pytest.mark.parametrize("n,T", [(1, 5), (33, 7), (4097, 20), (262_147, 6)])
def test_checksum_mode(n, T):
    g = rng.Generator(n, 12)
    rx, rs = g.generate_checksum(T)
    g.sync()
    rx, rs = rx.cpu().numpy(), rs.cpu().numpy()
    tail = g.generate(2).cpu().numpy()  # state advanced by T
    g.close()
    wx, ws, _ = oracle.row_checksums(n, 12, T)
    assert np.array_equal(rx, wx) and np.array_equal(rs, ws)
    assert np.array_equal(tail, oracle.generate(n, 12, 2, p0=T))


def test_profiler_names_and_overlap():
    n = 1 << 18
    g = rng.Generator(n, 1, device_buffer_bytes=8 * n, fuse_init=False, host_path=1)
    g.profile_reset()
    g.init()
    g.generate_to_host(8)
    p = g.profile()
    s = g.profile_summary()
    cnt_k, t_k = g.profile_stat("RNG_KERNEL")
    cnt_r, t_r = g.profile_stat("READ_BUFFER")
    g.close()
    assert set(p["aggregate"]) == {"INIT_KERNEL", "RNG_KERNEL", "READ_BUFFER"}
    assert cnt_k == 8 and cnt_r == 8 and t_k > 0 and t_r > 0
    assert p["effective"] <= p["total"] + 1e-12
    assert p["effective"] <= p["elapsed"]
    assert "Aggregate times by event" in s and "Time spent in device" in s


def test_direct_path_records_one_kernel_and_no_copy():
    n = 1 << 16
    host = torch.empty((6, n), dtype=torch.uint64).pin_memory()
    g = rng.Generator(n, 3, host_path=2)
    g.profile_reset()
    g.generate_to_host(6, host)
    cnt_k, _ = g.profile_stat("RNG_KERNEL")
    cnt_r, _ = g.profile_stat("READ_BUFFER")
    g.close()
    assert (cnt_k, cnt_r) == (1, 0)
    assert np.array_equal(host.numpy(), oracle.generate(n, 3, 6))


@pytest.mark.parametrize("n,T,R", [(1000, 10, 3), (4096, 7, 7), (4097, 5, 8), (100_001, 9, 2)])
def test_ring_output_holds_the_last_rows(n, T, R):
    g = rng.Generator(n, 21)
    ring = torch.zeros((R, n), dtype=torch.int64, device="cuda").view(torch.uint64)
    g.generate_ring(T, ring)
    after = g.generate(2).cpu().numpy()      # the state advanced by T
    got = ring.cpu().numpy()
    g.close()
    want = oracle.generate(n, 21, T + 2)
    for j in range(R):
        its = [i for i in range(T) if i % R == j]
        if its:
            assert np.array_equal(got[j], want[its[-1]]), (j, its[-1])
        else:
            assert (got[j] == 0).all()
    assert np.array_equal(after, want[T:])


@pytest.mark.parametrize("n,T", [(1, 5000), (5, 3000), (300, 2049), (4096, 1000), (10_000, 700), (70_001, 300)])
def test_few_streams_many_rows_split_into_bands(n, T):
    # Too few tiles to fill the GPU: rows are split into bands whose blocks
    # jump ahead over GF(2); values and the final states must not change.
    g = rng.Generator(n, 17)
    a = g.generate(T).cpu().numpy()
    b = g.generate(3).cpu().numpy()           # continues from the banded launch's states
    g.close()
    want = oracle.generate(n, 17, T + 3)
    assert np.array_equal(a, want[:T])
    assert np.array_equal(b, want[T:])


def test_generate_returns_a_tensor_ready_on_the_current_stream():
    # generate() launches on the generator's own stream; the tensor it hands
    # back must be readable at once on torch's current stream.  The memory is
    # dirtied first (torch's allocator hands the same block back), so a read
    # that ran ahead of the kernel would see the old values.
    for T in (257, 300, 1000):
        for _ in range(3):
            junk = torch.full((T, 1), -1, dtype=torch.int64, device="cuda")
            del junk
            g = rng.Generator(1, 17)
            got = g.generate(T).cpu().numpy()
            g.close()
            assert np.array_equal(got, oracle.generate(1, 17, T)), T


@pytest.mark.parametrize("vpt", [24, 32, 64])
def test_few_streams_many_rows_shapes_without_banded_variant(vpt):
    # Shapes compiled without a banded variant run unbanded.
    n, T = 3000, 600
    got = dev_gen(n, 29, T, values_per_thread=vpt)
    assert np.array_equal(got, oracle.generate(n, 29, T))


# Up to 2^18 streams the default shape holds 32 values per thread (8192 is the
# smallest such run: one tile); 200,003 ends on a ragged tile.
@pytest.mark.parametrize("n,T", [(1, 3000), (100, 1000), (4097, 700), (8192, 500), (1 << 16, 300),
                                 (200_003, 60)])
def test_checksum_mode_banded(n, T):
    g = rng.Generator(n, 31)
    rx, rs = g.generate_checksum(T)
    g.sync()
    tail = g.generate(2).cpu().numpy()
    g.close()
    wx, ws, _ = oracle.row_checksums(n, 31, T)
    assert np.array_equal(rx.cpu().numpy(), wx) and np.array_equal(rs.cpu().numpy(), ws)
    assert np.array_equal(tail, oracle.generate(n, 31, 2, p0=T))


@pytest.mark.parametrize("host_path", [1, 2, 3])
def test_few_streams_many_rows_to_host(host_path):
    n, T = 1000, 3000
    g = rng.Generator(n, 23, host_path=host_path)
    host = torch.empty((T, n), dtype=torch.uint64).pin_memory()
    g.generate_to_host(T, host)
    nxt = g.generate(2).cpu().numpy()
    g.close()
    want = oracle.generate(n, 23, T + 2)
    assert np.array_equal(host.numpy(), want[:T]) and np.array_equal(nxt, want[T:])


def test_allocation_failure_is_reported_and_recoverable():
    # A device buffer far larger than the GPU: cudaMalloc fails, the call
    # returns RNG_ENOMEM, and the generator still works for device output
    # after rng_init.
    n = 1000
    g = rng.Generator(n, 2, device_buffer_bytes=1 << 50, host_path=1)
    with pytest.raises(rng.RngError) as e:
        g.generate_to_host(3)
    assert e.value.code == 2
    g.init()
    assert np.array_equal(g.generate(3).cpu().numpy(), oracle.generate(n, 2, 3))
    g.close()


def test_server_arena_allocation_failure():
    from paper_1609_01257_gb300 import _capi as C
    with pytest.raises(rng.RngError) as e:
        rng.Server(hbm_budget_bytes=1 << 50)
    assert e.value.code == C.RNG_ENOMEM


def test_on_torch_current_stream_without_sync():
    # Launched on torch's current stream, the output can feed torch ops with
    # no explicit synchronisation in between.
    n, T = 50_000, 20
    g = rng.Generator(n, 8, compute_stream=torch.cuda.current_stream())
    out = g.generate(T)
    lo32 = (out.view(torch.int64) & 0xFFFFFFFF).sum(dim=1)   # queued right behind the kernel
    got = lo32.cpu().numpy()
    g.close()
    want = (oracle.generate(n, 8, T) & np.uint64(0xFFFFFFFF)).astype(np.int64).sum(axis=1)
    assert np.array_equal(got, want)


def test_live_objects_balance():
    before = rng.live_objects()
    gs = [rng.Generator(100, k) for k in range(3)]
    assert rng.live_objects() == before + 3
    for g in gs:
        g.close()
    assert rng.live_objects() == before


def test_launch_counter_counts_kernels():
    g = rng.Generator(1000, 1)
    c0 = rng.launch_count()
    g.generate(3)
    g.generate(3)
    g.sync()
    assert rng.launch_count() == c0 + 2
    g.close()
