"""Batched form against the oracle, instance by instance."""
import numpy as np
import pytest
import torch

import oracle
import paper_1609_01257_gb300 as rng
import workloads

pytestmark = pytest.mark.gpu


def test_small_batch_fixed_vpt_all_values():
    streams = [1, 2, 3, 255, 256, 257, 1000, 4099, 70_000]
    iters = [1, 5, 2, 7, 3, 1, 9, 4, 2]
    seeds = [0, 1, 2, 3, 4, 5, 6, 7, 2**64 - 1]
    want = [oracle.generate(streams[k], seeds[k], iters[k]) for k in range(len(streams))]
    for mode in (1, 2):          # one unit per block / persistent blocks with a counter
        for vpt in (1, 2, 4, 6, 8, 12, 16, 24, 32):
            b = rng.Batch(streams, iters, seeds, values_per_thread=vpt, mode=mode)
            b.run()
            b.sync()
            assert b.config()["one_unit_per_block"] == (mode == 1)
            for k in range(len(streams)):
                got = b.outputs[k].cpu().numpy()
                assert np.array_equal(got, want[k]), (mode, vpt, k)
            b.close()


def test_replay_is_identical_and_autotuned():
    streams = [3000, 5, 1 << 16]
    iters = [3, 40, 6]
    seeds = [10, 11, 12]
    b = rng.Batch(streams, iters, seeds)
    cfg = b.config()
    assert cfg["values_per_thread"] in (1, 2, 4, 6, 8, 12, 16, 24, 32) and cfg["tuned_ms"] > 0
    for o in b.outputs:
        o.view(torch.int64).zero_()
    torch.cuda.synchronize()
    b.run()
    b.sync()
    first = [o.cpu().numpy().copy() for o in b.outputs]
    b.run()
    b.sync()
    for k, o in enumerate(b.outputs):
        assert np.array_equal(o.cpu().numpy(), first[k])
        assert np.array_equal(first[k], oracle.generate(streams[k], seeds[k], iters[k]))
    b.close()


def test_unaligned_instance_outputs():
    # One shared buffer with instances at 8-byte (not 16-byte) offsets.
    streams, iters, seeds = [6, 10, 4], [3, 2, 5], [1, 2, 3]
    sizes = [n * t for n, t in zip(streams, iters)]
    buf = torch.zeros(sum(sizes) + 1, dtype=torch.int64, device="cuda").view(torch.uint64)
    outs, off = [], 1
    for s, n, t in zip(sizes, streams, iters):
        outs.append(buf[off:off + s].view(t, n))
        off += s
    b = rng.Batch(streams, iters, seeds, outputs=outs, values_per_thread=4)
    b.run()
    b.sync()
    for k in range(3):
        assert np.array_equal(outs[k].cpu().numpy(), oracle.generate(streams[k], seeds[k], iters[k]))
    assert int(buf.view(torch.int64)[0].item()) == 0
    b.close()


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("vpt", [1, 2, 4, 6, 8])
def test_rows_off_the_cache_lines_are_staged(vpt, mode):
    # Row pitches that are not multiples of 16 values and outputs that start
    # off a 128-byte line: these rows go through the shared-memory staging.
    # Several tiles per instance, ragged last tiles, every output surrounded
    # by canary values that must stay untouched.
    streams = [2049, 4097, 70_001, 1000, 4103, 16, 5000]
    iters = [5, 3, 2, 9, 4, 7, 3]
    seeds = [3, 1, 4, 1, 5, 9, 2]
    offsets = [1, 3, 5, 7, 16, 9, 2]     # 8-byte words from a line boundary
    total = sum(o + n * t + 3 for o, n, t in zip(offsets, streams, iters))
    buf = torch.full((total + 16,), 0x5A5A, dtype=torch.int64, device="cuda").view(torch.uint64)
    outs, spans, pos = [], [], 0
    for o, n, t in zip(offsets, streams, iters):
        pos += o
        outs.append(buf[pos:pos + n * t].view(t, n))
        spans.append((pos, pos + n * t))
        pos += n * t + 3
    b = rng.Batch(streams, iters, seeds, outputs=outs, values_per_thread=vpt, mode=mode)
    b.run()
    b.sync()
    for k in range(len(streams)):
        assert np.array_equal(outs[k].cpu().numpy(), oracle.generate(streams[k], seeds[k], iters[k])), k
    host = buf.view(torch.int64).cpu().numpy()
    mask = np.ones(host.size, dtype=bool)
    for a, e in spans:
        mask[a:e] = False
    assert (host[mask] == 0x5A5A).all()
    b.close()


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("vpt", [4, 8])
def test_bulk_copies_for_long_units(vpt, mode):
    # stores = 2: units of 16 or more rows are written by TMA bulk copies,
    # shorter ones by the register and staged stores, in one kernel (with
    # persistent blocks a block moves between the two paths).  Odd and even
    # pitches, outputs off 16-byte and 128-byte boundaries, canaries around
    # every output.
    streams = [2049, 4097, 70_001, 1000, 4103, 16, 5000, 1, 300, 65_536]
    iters = [20, 3, 16, 40, 15, 33, 2, 50, 17, 18]
    seeds = [3, 1, 4, 1, 5, 9, 2, 6, 5, 3]
    offsets = [1, 3, 5, 7, 16, 9, 2, 1, 4, 0]
    total = sum(o + n * t + 3 for o, n, t in zip(offsets, streams, iters))
    buf = torch.full((total + 16,), 0x5A5A, dtype=torch.int64, device="cuda").view(torch.uint64)
    outs, spans, pos = [], [], 0
    for o, n, t in zip(offsets, streams, iters):
        pos += o
        outs.append(buf[pos:pos + n * t].view(t, n))
        spans.append((pos, pos + n * t))
        pos += n * t + 3
    b = rng.Batch(streams, iters, seeds, outputs=outs, values_per_thread=vpt, mode=mode, stores=2)
    cfg = b.config()
    assert cfg["stores"] == "bulk" and cfg["row_buffers"] > 0
    for _ in range(2):  # a replay rewrites the same values
        b.run()
        b.sync()
        for k in range(len(streams)):
            assert np.array_equal(outs[k].cpu().numpy(), oracle.generate(streams[k], seeds[k], iters[k])), k
    host = buf.view(torch.int64).cpu().numpy()
    mask = np.ones(host.size, dtype=bool)
    for a, e in spans:
        mask[a:e] = False
    assert (host[mask] == 0x5A5A).all()
    b.close()


def test_autotune_over_both_store_paths():
    # stores = 0 tunes over register/staged and bulk-copy shapes; stores = 1
    # keeps the first.  Either way every value matches the oracle.
    streams, iters, seeds = [70_001, 3000, 257], [40, 20, 5], [7, 8, 9]
    for stores in (0, 1, 2):
        b = rng.Batch(streams, iters, seeds, stores=stores)
        cfg = b.config()
        if stores:
            assert cfg["stores"] == ("bulk" if stores == 2 else "register")
        b.run()
        b.sync()
        for k in range(3):
            assert np.array_equal(b.outputs[k].cpu().numpy(), oracle.generate(streams[k], seeds[k], iters[k]))
        b.close()


def _row_checksums(block):
    return np.bitwise_xor.reduce(block, axis=1), block.sum(axis=1, dtype=np.uint64)


def test_paper_shaped_batch_every_row_checksummed():
    # 512 instances, 8 GiB: every row of every instance reduced to its XOR and
    # wrapping sum on the host and compared with the oracle's.
    inst = workloads.batched_instances()
    b = rng.Batch([i.streams for i in inst], [i.iterations for i in inst], [i.seed for i in inst])
    b.run()
    b.sync()
    for k, ins in enumerate(inst):
        out = b.outputs[k].cpu().numpy()
        x, s = _row_checksums(out)
        wx, ws, _ = oracle.row_checksums(ins.streams, ins.seed, ins.iterations)
        assert np.array_equal(x, wx) and np.array_equal(s, ws), k
    b.close()


def test_paper_shaped_batch_sampled():
    # 512 instances, log-uniform sizes, 8 GiB total: every instance checked on
    # its first row and sampled values, small instances in full.
    inst = workloads.batched_instances()
    b = rng.Batch([i.streams for i in inst], [i.iterations for i in inst], [i.seed for i in inst])
    b.run()
    b.sync()
    rs = np.random.default_rng(0)
    for k, ins in enumerate(inst):
        out = b.outputs[k]
        if ins.streams * ins.iterations <= 200_000:
            assert np.array_equal(out.cpu().numpy(), oracle.generate(ins.streams, ins.seed, ins.iterations)), k
            continue
        row0 = out[0].cpu().numpy()
        assert np.array_equal(row0, oracle.generate(ins.streams, ins.seed, 1)[0]), k
        last = out[ins.iterations - 1].cpu().numpy()
        gs = rs.integers(0, ins.streams, 16)
        for g in gs:
            assert int(last[g]) == oracle.value(int(g), ins.seed, ins.iterations - 1)
    b.close()
