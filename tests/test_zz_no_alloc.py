"""The allocation-free batched entry point, through the C ABI.

``rng_batch_generate_noalloc`` is for callers that must not allocate device
memory: code inside a framework whose memory pool owns the whole device and
forbids allocations beside it, or latency-bound code that cannot pay for a
cudaMalloc (and the device-wide synchronisation of a cudaFree) on every call.
Its scratch is a fixed array in device global memory instead.

These tests check, on consecutive calls on one stream:
  * every output value against the CPU oracle, and against the regular
    batched entry point (``rng_batch_create`` / ``rng_batch_run``);
  * batches at exactly the instance limit and exactly the work-unit limit;
  * that device free memory is the same before and after each call that
    follows the first (the first call may load the library's device code
    and its scratch array).
The file is named so that pytest collects it last; every test starts with a
small warm-up call, so each also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1609_01257_gb300 as rng
from paper_1609_01257_gb300 import _capi as C

pytestmark = pytest.mark.gpu

U64 = ctypes.c_uint64
MAX_INSTANCES = 4096       # RNG_NOALLOC_MAX_INSTANCES in include/rng.h
MAX_UNITS = 262_144        # RNG_NOALLOC_MAX_UNITS
TILE = 2048                # streams per work unit


def _flat_outputs(streams, iterations, misalign_odd=False):
    """One device buffer holding every instance's output; returns the buffer
    and a uint64 view (iterations, streams) per instance.  Offsets are kept
    16-byte aligned unless ``misalign_odd`` shifts every odd instance by one
    value (8-byte aligned outputs take the kernel's narrow-store path)."""
    offs, o = [], 0
    for k, (n, t) in enumerate(zip(streams, iterations)):
        if misalign_odd and k % 2 == 1:
            o += 1
        offs.append(o)
        o += n * t
        o += o % 2
    buf = torch.zeros(o + 2, dtype=torch.int64, device="cuda").view(torch.uint64)
    views = [buf[a:a + n * t].view(t, n) for a, n, t in zip(offs, streams, iterations)]
    return buf, views


def _call(L, streams, iterations, seeds, views, stream):
    """One call of the entry point; returns after the stream has finished it.
    Also returns the device free memory just before and just after the call."""
    k = len(streams)
    ptrs = (ctypes.c_void_p * k)(*[v.data_ptr() for v in views])
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    err = ctypes.POINTER(C.RngErr)()
    rc = L.rng_batch_generate_noalloc(k, (U64 * k)(*streams), (U64 * k)(*iterations),
                                      (U64 * k)(*[s & (2**64 - 1) for s in seeds]), ptrs,
                                      ctypes.c_void_p(stream.cuda_stream), ctypes.byref(err))
    msg = err.contents.msg.decode() if err else ""
    L.rng_err_clear(ctypes.byref(err))
    assert rc == C.RNG_OK, msg
    stream.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    return free_before, free_after


@pytest.fixture
def lib_and_stream():
    L = C.load()
    stream = torch.cuda.Stream()
    # Warm-up: the first call on a device looks up the scratch array's
    # address, which may make the driver load the library's device code.
    _, views = _flat_outputs([3], [2])
    _call(L, [3], [2], [1], views, stream)
    return L, stream


def _check_oracle(views, streams, iterations, seeds):
    host = [v.cpu().numpy() for v in views]
    for k, (got, n, t, s) in enumerate(zip(host, streams, iterations, seeds)):
        want = oracle.generate(n, s & (2**64 - 1), t)
        assert np.array_equal(got, want), f"instance {k} ({n} streams x {t} iterations, seed {s}) differs"


def test_noalloc_matches_oracle_and_regular_batch_on_two_calls(lib_and_stream):
    L, stream = lib_and_stream
    first = ([1, 2, 3, 257, 4096, 70_001, 65_536], [1, 5, 2, 9, 3, 4, 2], [0, 1, 2, 3, 4, 5, 2**64 - 1])
    second = ([5000, 9, 131_072, 2047, 2049], [7, 300, 2, 11, 1], [12345, 99, 7, 8, 9])
    buf1, out1 = _flat_outputs(*first[:2], misalign_odd=True)
    buf2, out2 = _flat_outputs(*second[:2])
    f0, f1 = _call(L, *first, out1, stream)
    g0, g1 = _call(L, *second, out2, stream)   # the second call reuses the same scratch
    assert f0 == f1 and g0 == g1, "device free memory changed across a call"
    _check_oracle(out1, *first)
    _check_oracle(out2, *second)
    # The regular batched entry point writes the same values.
    for views, (streams, iterations, seeds) in ((out1, first), (out2, second)):
        b = rng.Batch(streams, iterations, seeds, values_per_thread=8)
        b.run()
        b.sync()
        for got, want in zip(views, b.outputs):
            assert torch.equal(got.view(torch.int64), want.view(torch.int64))
        b.close()


def test_noalloc_at_the_instance_limit(lib_and_stream):
    L, stream = lib_and_stream
    r = np.random.default_rng(4096)
    streams = [int(x) for x in r.integers(1, 3000, MAX_INSTANCES)]
    iterations = [int(x) for x in r.integers(1, 5, MAX_INSTANCES)]
    seeds = [int(x) for x in r.integers(0, 2**63, MAX_INSTANCES)]
    _, views = _flat_outputs(streams, iterations, misalign_odd=True)
    before, after = _call(L, streams, iterations, seeds, views, stream)
    assert before == after, "device free memory changed across a call"
    _check_oracle(views, streams, iterations, seeds)
    # One instance more is refused, before anything is launched.
    k = MAX_INSTANCES + 1
    err = ctypes.POINTER(C.RngErr)()
    rc = L.rng_batch_generate_noalloc(k, (U64 * k)(*([1] * k)), (U64 * k)(*([1] * k)), (U64 * k)(*([1] * k)),
                                      (ctypes.c_void_p * k)(*([views[0].data_ptr()] * k)),
                                      ctypes.c_void_p(stream.cuda_stream), ctypes.byref(err))
    assert rc == C.RNG_EINVAL and b"at most 4096" in err.contents.msg
    L.rng_err_clear(ctypes.byref(err))


def test_noalloc_at_the_work_unit_limit(lib_and_stream):
    L, stream = lib_and_stream
    # 131,073 + 131,071 = 262,144 work units, both instances with a ragged last tile.
    streams = [(1 << 28) + 5, 131_071 * TILE - 100]
    iterations = [1, 2]
    seeds = [31, 2**64 - 3]
    assert sum((n + TILE - 1) // TILE for n in streams) == MAX_UNITS
    _, views = _flat_outputs(streams, iterations)
    before, after = _call(L, streams, iterations, seeds, views, stream)
    assert before == after, "device free memory changed across a call"
    block = 1 << 25
    for k, (v, n, t, s) in enumerate(zip(views, streams, iterations, seeds)):
        for a in range(0, n, block):
            b = min(n, a + block)
            want = oracle.generate(b - a, s, t, g0=a)
            for row in range(t):
                got = v[row, a:b].cpu().numpy()
                assert np.array_equal(got, want[row]), f"instance {k}, row {row}, streams {a}..{b} differ"
    # One unit more is refused, before anything is launched.
    err = ctypes.POINTER(C.RngErr)()
    ptrs = (ctypes.c_void_p * 2)(views[0].data_ptr(), views[1].data_ptr())
    rc = L.rng_batch_generate_noalloc(2, (U64 * 2)(streams[0], streams[1] + 100 + 1), (U64 * 2)(*iterations),
                                      (U64 * 2)(*seeds), ptrs, ctypes.c_void_p(stream.cuda_stream),
                                      ctypes.byref(err))
    assert rc == C.RNG_EINVAL and b"work units" in err.contents.msg
    L.rng_err_clear(ctypes.byref(err))
