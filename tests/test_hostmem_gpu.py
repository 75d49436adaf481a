"""Page-locked host memory from the library's allocator (rng_host_alloc) as
the destination of host output: every host path writes the oracle's values
into it, the range starts on a huge-page boundary, and the full-size
streaming run through the double buffer (the benchmark's end-to-end
destination) is checked against the oracle."""
import numpy as np
import pytest

import oracle
import paper_1609_01257_gb300 as rng
import workloads

pytestmark = pytest.mark.gpu


def _huge_page_bytes():
    try:
        with open("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size") as f:
            return int(f.read())
    except (OSError, ValueError):
        return 2 << 20


@pytest.mark.parametrize("huge", [True, False])
@pytest.mark.parametrize("host_path", [0, 1, 2, 3])
def test_every_host_path_into_allocator_memory(huge, host_path):
    n, T, seed = 70_001, 37, 99
    live0 = rng.live_objects()
    out = rng.host_empty((T, n), huge_pages=huge)
    if huge:
        assert out.ctypes.data % _huge_page_bytes() == 0
    # Small device buffers: many chunks per call (whole rows, 4 per buffer).
    g = rng.Generator(n, seed, device_buffer_bytes=8 * n * 4, host_path=host_path)
    g.generate_to_host(T, out)
    g.close()
    assert np.array_equal(out, oracle.generate(n, seed, T))
    del out
    assert rng.live_objects() == live0


def test_allocator_memory_starts_zeroed_and_views_keep_it_alive():
    a = rng.host_empty(1 << 20)
    assert a.dtype == np.uint64 and not a.any()
    view = a[5:9]
    del a
    view[:] = 7                      # the range is still mapped through the view
    assert view.sum() == 28
    with pytest.raises(ValueError):
        rng.host_empty(0)


def test_streaming_full_size_double_buffer_into_huge_pages():
    # The benchmark's end-to-end destination: 32 GiB from rng_host_alloc,
    # written by the paper's double buffer (copy-engine reads); every 16th
    # row in full and every row's XOR / wrapping sum against the oracle.
    cfg = workloads.STREAMING
    n, T, seed = cfg["streams"], cfg["iterations"], cfg["seed"]
    host = rng.host_empty((T, n))
    g = rng.Generator(n, seed, device_buffer_bytes=cfg["device_buffer_bytes"], host_path=1)
    g.generate_to_host(T, host)
    g.close()
    wx, ws, samples = oracle.row_checksums(n, seed, T, sample_every=16)
    for j, i in enumerate(range(0, T, 16)):
        assert np.array_equal(host[i], samples[j]), f"row {i} differs"
    for i0 in range(0, T, 64):
        blk = host[i0:i0 + 64]
        assert np.array_equal(np.bitwise_xor.reduce(blk, axis=1), wx[i0:i0 + 64])
        assert np.array_equal(blk.sum(axis=1, dtype=np.uint64), ws[i0:i0 + 64])
