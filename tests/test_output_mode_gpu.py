"""Alternative output mode (xorshift64* scrambled values of the paper's state
sequence): every path that emits values, against the oracle's mode 1."""
import numpy as np
import pytest
import torch

import oracle
import paper_1609_01257_gb300 as rng
import workloads

pytestmark = pytest.mark.gpu


def _dev(n, seed, T, **kw):
    g = rng.Generator(n, seed, output_mode=1, **kw)
    out = g.generate(T)
    g.sync()
    res = out.cpu().numpy()
    g.close()
    return res


@pytest.mark.parametrize("vpt", [0, 1, 2, 4, 8, 16, 24, 32])
@pytest.mark.parametrize("n,T", [(1, 5), (33, 7), (4097, 20), (262_147, 3)])
def test_device_output(vpt, n, T):
    assert np.array_equal(_dev(n, 41, T, values_per_thread=vpt), oracle.generate(n, 41, T, output_mode=1))


def test_differs_from_mode_0_and_unscrambles_to_it():
    n, T = 5000, 6
    star = _dev(n, 2, T)
    g = rng.Generator(n, 2)
    plain = g.generate(T).cpu().numpy()
    g.close()
    inv = pow(0x2545F4914F6CDD1D, -1, 1 << 64)
    assert not np.array_equal(star, plain)
    assert np.array_equal((star * np.uint64(inv)), plain)  # wraps modulo 2^64


def test_unaligned_output_and_offsets():
    # Odd stream count: every other row starts 8-byte aligned only.
    n, T = 3001, 9
    got = _dev(n, 5, T, stream_offset=123)
    assert np.array_equal(got, oracle.generate(n, 5, T, g0=123, output_mode=1))


def test_few_streams_many_rows_banded():
    n, T = 1000, 3000
    g = rng.Generator(n, 23, output_mode=1)
    out = g.generate(T)
    nxt = g.generate(2)
    g.sync()
    got, nxt = out.cpu().numpy(), nxt.cpu().numpy()
    g.close()
    want = oracle.generate(n, 23, T + 2, output_mode=1)
    assert np.array_equal(got, want[:T]) and np.array_equal(nxt, want[T:])


@pytest.mark.parametrize("n,T", [(1, 5), (4097, 20), (262_147, 6), (1 << 16, 600)])
def test_checksum_mode(n, T):
    g = rng.Generator(n, 12, output_mode=1)
    rx, rs = g.generate_checksum(T)
    g.sync()
    rx, rs = rx.cpu().numpy(), rs.cpu().numpy()
    tail = g.generate(2).cpu().numpy()
    g.close()
    wx, ws, _ = oracle.row_checksums(n, 12, T, output_mode=1)
    assert np.array_equal(rx, wx) and np.array_equal(rs, ws)
    assert np.array_equal(tail, oracle.generate(n, 12, 2, p0=T, output_mode=1))


@pytest.mark.parametrize("host_path", [0, 1, 3])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_output(host_path, pinned):
    n, T = 5000, 7
    g = rng.Generator(n, 4, output_mode=1, host_path=host_path, device_buffer_bytes=4096)
    out = torch.empty((T, n), dtype=torch.uint64)
    if pinned:
        out = out.pin_memory()
    g.generate_to_host(T, out)
    g.close()
    assert np.array_equal(out.numpy(), oracle.generate(n, 4, T, output_mode=1))


def test_sink_fd_and_host_checksum(tmp_path):
    n, T = 4096, 12
    g = rng.Generator(n, 9, output_mode=1, device_buffer_bytes=8 * n * 5)
    got = np.zeros((T, n), dtype=np.uint64)

    def sink(first_it, block, first_stream):
        got[first_it:first_it + block.shape[0], first_stream:first_stream + block.shape[1]] = block

    g.generate_sink(T, sink)
    path = tmp_path / "out.bin"
    with open(path, "wb") as f:
        g.generate_fd(T, f.fileno())
    hx, hs = g.generate_host_checksum(T)
    g.close()
    want = oracle.generate(n, 9, 3 * T, output_mode=1)
    assert np.array_equal(got, want[:T])
    assert np.array_equal(np.fromfile(path, dtype=np.uint64).reshape(T, n), want[T:2 * T])
    wx, ws, _ = oracle.row_checksums(n, 9, T, p0=2 * T, output_mode=1)
    assert np.array_equal(hx, wx) and np.array_equal(hs, ws)


def test_states_skip_and_checkpoint_are_shared_with_mode_0():
    # The state sequence is the paper's in both modes: checkpoints taken in
    # one mode resume in the other, and rng_skip lands on the same states.
    n = 2048
    a = rng.Generator(n, 3, output_mode=1)
    a.generate(10)
    a.skip(5000)
    s_star = a.state()
    b = rng.Generator(n, 3)
    b.generate(10)
    b.skip(5000)
    s_plain = b.state()
    assert np.array_equal(s_star, s_plain)
    b.close()
    nxt = a.generate(3).cpu().numpy()
    a.close()
    assert np.array_equal(nxt, oracle.generate(n, 3, 3, p0=10 + 5000, output_mode=1))
    c = rng.Generator(n, 3)  # mode 0, resumed from the mode-1 checkpoint
    c.set_state(s_star, 10 + 5000)
    resumed = c.generate(3).cpu().numpy()
    c.close()
    assert np.array_equal(resumed, oracle.generate(n, 3, 3, p0=10 + 5000))


@pytest.mark.parametrize("kw", [dict(output_mode=2), dict(output_mode=1, values_per_thread=12),
                                dict(output_mode=1, block_threads=512, values_per_thread=8)])
def test_unsupported_configurations(kw):
    with pytest.raises(rng.RngError) as e:
        rng.Generator(64, 1, **kw)
    assert e.value.code == 1


def test_streaming_full_size_sampled():
    # The paper-shaped run (2^22 streams x 1024 iterations) in mode 1,
    # device-resident in the benchmark's launch shape: every 64th row in full
    # and every row's checksums (generate-and-checksum mode) against the oracle.
    cfg = workloads.STREAMING
    n, T, seed = cfg["streams"], cfg["iterations"], cfg["seed"]
    g = rng.Generator(n, seed, output_mode=1)
    out = g.generate(T)
    g.sync()
    rows = out[::64].cpu().numpy()
    del out
    g.init()
    rx, rs = g.generate_checksum(T)
    g.sync()
    rx, rs = rx.cpu().numpy(), rs.cpu().numpy()
    g.close()
    wx, ws, samples = oracle.row_checksums(n, seed, T, sample_every=64, output_mode=1)
    assert np.array_equal(rows, samples)
    assert np.array_equal(rx, wx) and np.array_equal(rs, ws)
