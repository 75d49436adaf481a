"""The allocation-free batched entry point against the regular batched form.

``rng_batch_generate_noalloc`` serves callers that cannot call cudaMalloc
(for example code running during someone else's stream capture, or inside a
framework whose memory pool owns the device).  It keeps its scratch in a
fixed device array instead of allocating it.  This test calls it through the
C ABI twice in a row, with different batches on one stream, and requires
each output to equal, value for value, what the regular batched entry point
(``rng_batch_create`` / ``rng_batch_run``) writes for the same instances.
The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_1609_01257_gb300 as rng
from paper_1609_01257_gb300 import _capi as C

pytestmark = pytest.mark.gpu

U64 = ctypes.c_uint64


def _noalloc(L, streams, iterations, seeds, stream):
    k = len(streams)
    outs = [torch.zeros((t, n), dtype=torch.int64, device="cuda").view(torch.uint64)
            for n, t in zip(streams, iterations)]
    torch.cuda.synchronize()  # outputs allocated and cleared before the library writes them
    ptrs = (ctypes.c_void_p * k)(*[o.data_ptr() for o in outs])
    err = ctypes.POINTER(C.RngErr)()
    rc = L.rng_batch_generate_noalloc(k, (U64 * k)(*streams), (U64 * k)(*iterations), (U64 * k)(*seeds),
                                      ptrs, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(err))
    msg = err.contents.msg.decode() if err else ""
    L.rng_err_clear(ctypes.byref(err))
    assert rc == C.RNG_OK, msg
    return outs


def _regular(streams, iterations, seeds):
    b = rng.Batch(streams, iterations, seeds, values_per_thread=8)
    b.run()
    b.sync()
    res = [o.cpu().numpy().copy() for o in b.outputs]
    b.close()
    return res


def test_noalloc_matches_regular_batch_on_two_calls():
    L = C.load()
    stream = torch.cuda.Stream()
    first = ([1, 2, 3, 257, 4096, 70_001, 65_536], [1, 5, 2, 9, 3, 4, 2], [0, 1, 2, 3, 4, 5, 2**64 - 1])
    second = ([5000, 9, 131_072, 2047, 2049], [7, 300, 2, 11, 1], [12345, 99, 7, 8, 9])
    out1 = _noalloc(L, *first, stream)
    out2 = _noalloc(L, *second, stream)   # second call reuses the same scratch
    stream.synchronize()
    for got, want in zip(out1, _regular(*first)):
        assert np.array_equal(got.cpu().numpy(), want)
    for got, want in zip(out2, _regular(*second)):
        assert np.array_equal(got.cpu().numpy(), want)


def test_noalloc_rejects_batches_beyond_its_scratch():
    L = C.load()
    k = 1
    big = [(1 << 32)]                 # 2^32 / 2048 = 2^21 units > the limit
    out = torch.empty(8, dtype=torch.int64, device="cuda")
    ptrs = (ctypes.c_void_p * k)(out.data_ptr())
    err = ctypes.POINTER(C.RngErr)()
    rc = L.rng_batch_generate_noalloc(k, (U64 * k)(*big), (U64 * k)(1), (U64 * k)(1), ptrs, None,
                                      ctypes.byref(err))
    assert rc == C.RNG_EINVAL and b"at most" in err.contents.msg
    L.rng_err_clear(ctypes.byref(err))
